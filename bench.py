#!/usr/bin/env python
"""Throughput benchmark of the FD-CGKS step on GB300.

Workload: the 2-D isentropic vortex on a periodic [0,10]^2 domain at 1024^2
primary nodes (plus 1024^2 dual nodes), strength 5 at (5,5), free stream
(1,1,1,1), gamma = 1.4, FD-CGKS(6-4), GENO (App. D constants), CFL 0.2.
A step is one full S2O4 step (two stages) of both grids; a node update is
one step of one primary or dual node (2 * 1024^2 per step).

Prints one JSON line, kept short (the figures that explain it are in the
`--detail` file).  `value` is the FP64 path's node-updates/s with the state
resident in HBM (all N ranks together); `mixed` is the mixed FP32/FP64 path
on the same workload with its error against the FP64 path; `err_vs_oracle`
states the error of both paths against the FP64 CPU oracle on oracle-sized
samples of the vortex, the viscous shock tube and an ensemble member (those
oracle runs are the CPU-baseline leg, timed as `cpu_baseline`).  `e2e` is the
same metric through the C ABI with host state: every step copies the state in
from pinned host memory, steps, and copies it back out.  `roofline` is the
dominant kernel's; `kernel_frac` gives every kernel's fraction of its bound
(FP64 / FP32 FMA pipe peaks measured in this run by csrc/pipe_peak.cu, HBM
copy bandwidth from the driver's measurement).

--impl reference times the CPU oracle (the plain FP64 C++ implementation
the tests compare against) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "2D node-updates/s, FP64 vs mixed-FP32 at stated L1 error; % of roofline"
UNIT = "node-updates/s"
# derived peaks, for context beside the measured ones: 152 SMs x 4 FP64
# flop/clk (2 DFMA per clock per SM) x 2.07 GHz; 152 x 128 FP32 lanes x 2 x 2.07 GHz
FP64_DERIVED_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FP32_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0


def kernel_hash():
    """Hash of the kernel sources; profiles/dram_traffic.json records the hash
    its counters were taken on."""
    import hashlib
    h = hashlib.sha256()
    for f in ("fdcgks_math.cuh", "fdcgks_kernels.cuh", "fdcgks_internal.cuh", "fdcgks_api.cu"):
        with open(os.path.join(ROOT, "paper_2606_17772_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` at n^2 from profiles/dram_traffic.json
    (ncu dram__bytes_read.sum + dram__bytes_write.sum), if it was taken on
    this kernel source at this grid; otherwise None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        rec = json.load(fh)
    if rec.get("kernel_hash") != kernel_hash():
        return None
    ent = rec.get("kernels", {}).get(kernel)
    if not ent or ent.get("n") != n:
        return None
    return ent.get("bytes_per_launch")


def hbm_peak():
    """Measured copy bandwidth (GB/s) from MEASURED_PEAKS.json, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return HBM_FALLBACK_GBS, "fallback 6.8 TB/s"


def pipe_peaks():
    """FP64 and FP32 FMA-pipe peaks (TFLOP/s) measured now on this GPU by
    csrc/pipe_peak.cu: chains of independent FMAs over all SMs, best of 5."""
    import ctypes
    from paper_2606_17772_gb300 import build as fbuild
    lib = ctypes.CDLL(fbuild.build_pipe_peak())
    out = {}
    for name, prec, iters in (("fp64", 0, 1000), ("fp32", 1, 40000)):
        tf, ms = ctypes.c_double(), ctypes.c_double()
        rc = lib.pipe_peak_tflops(prec, 8, iters, 5, ctypes.byref(tf), ctypes.byref(ms))
        if rc != 0:
            raise RuntimeError("pipe peak measurement failed (%d)" % rc)
        out[name] = tf.value
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1024, help="primary nodes per direction")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-peaks", action="store_true", help="derived pipe peaks instead of measured (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ens-members", type=int, default=256)
    ap.add_argument("--ens-steps", type=int, default=200)
    ap.add_argument("--ens-nmax", type=int, default=512, help="largest ensemble grid")
    ap.add_argument("--ens-no-tune", action="store_true", help="default tiles (profiling runs)")
    ap.add_argument("--no-viscous-tube", action="store_true")
    ap.add_argument("--vt-steps", type=int, default=100, help="timed steps of the viscous shock tube window")
    ap.add_argument("--no-double-mach", action="store_true")
    ap.add_argument("--no-lines", action="store_true")
    ap.add_argument("--dmr-steps", type=int, default=100, help="timed FP64 steps of the double Mach window")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adj-steps", type=int, default=20, help="steps of the adjoint window")
    ap.add_argument("--ensemble-only", action="store_true",
                    help="run only the ensemble workload and print its object (profiling runs)")
    ap.add_argument("--detail", default=None, help="also write every measured figure to this JSON file")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args, backend="nccl"):
    """Replicas: one process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE),
    each advancing its own copy of the workload; the only collectives are the
    barriers around the timed region and the max of the elapsed times.
    backend "gloo" runs the same logic on host tensors (CPU tests)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return world, rank, local


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, elapsed_s, world):
    """Whole-job rate of weak-scaled replicas: the units all ranks processed
    over the slowest rank's time."""
    el = max_over_ranks(elapsed_s, world)
    return units_per_rank * world / el, el


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def oracle_rate(n_sample, nsteps):
    """Node-updates/s of the CPU oracle on an n_sample^2 vortex (same constants)."""
    import oracle
    from paper_2606_17772_gb300 import inputs
    case = inputs.vortex(n_sample)
    p = oracle.make_params(**case.oracle_kwargs())
    S = case.initial_state()
    dt = 0.2 * case.hx / (math.sqrt(2.0) + math.sqrt(1.4)) * 0.9
    warm = inputs.vortex(16)            # load the library outside the timing
    oracle.steps(oracle.make_params(**warm.oracle_kwargs()), dt, 1, *warm.initial_state())
    t0 = time.perf_counter()
    oracle.steps(p, dt, nsteps, *S)
    el = time.perf_counter() - t0
    return 2 * n_sample * n_sample * nsteps / el, el


def _oracle_rate_task(sample):
    return oracle_rate(*sample)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate_all_cores(n_sample, nsteps, ncores=None):
    """The same bounded sample run concurrently by one spawned process per host
    core, each on its own copy (independent runs, the oracle unchanged):
    aggregate node-updates/s over the wall time of the concurrent runs."""
    import multiprocessing as mp
    ncores = ncores or host_cores()
    with mp.get_context("spawn").Pool(ncores) as pool:
        pool.map(_oracle_rate_task, [(8, 1)] * (2 * ncores), chunksize=1)   # start workers, load the library
        t0 = time.perf_counter()
        pool.map(_oracle_rate_task, [(n_sample, nsteps)] * ncores, chunksize=1)
        wall = time.perf_counter() - t0
    return ncores * 2 * n_sample * n_sample * nsteps / wall, wall, ncores


def run_reference(args):
    """CPU oracle as the reference arm: K timed steps of a bounded sample."""
    world, rank = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2606_17772_gb300 import inputs
    ns = 48
    case = inputs.vortex(ns)
    p = oracle.make_params(**case.oracle_kwargs())
    S = case.initial_state()
    dt = 0.2 * case.hx / (math.sqrt(2.0) + math.sqrt(1.4)) * 0.9
    for _ in range(args.warmup):
        S = oracle.steps(p, dt, 1, *S)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S = oracle.steps(p, dt, 1, *S)
    el = time.perf_counter() - t0
    value = 2 * ns * ns * args.steps / el
    sample = "isentropic vortex %d^2 (+%d^2 dual), periodic [0,10]^2, strength 5, FD-CGKS(6-4)" % (ns, ns)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "isentropic vortex 1024^2 (oracle on a %d^2 sample)" % ns},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def timed_steps(solver, dt, steps, warmup, world, device_index, sample_clocks):
    """Time `steps` steps with CUDA events on the context stream (profiling
    off, so that no event sits between the kernels), then run the same steps
    again with per-class events for the kernel-class breakdown."""
    import torch
    solver.steps(dt, warmup)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    launches0 = solver.launches()
    sampler = ClockSampler(device_index) if sample_clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    solver.steps(dt, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    launches = solver.launches() - launches0
    solver.set_profiling(True)
    solver.get_profile()                         # clear
    solver.steps(dt, steps)
    torch.cuda.synchronize()
    prof_ms, prof_n, _ = solver.get_profile()
    solver.set_profiling(False)
    return ms, prof_ms, prof_n, launches, clocks


def run_ensemble(args, world, rank, local, peaks=None):
    """Batched ensemble workload: seeded periodic isentropic vortices on uneven
    grids (N log-uniform in [32, 512], strength U[1, 5], centre uniform),
    mixed precision, every member taking its own CFL-0.2 step each step,
    one CUDA-graph step per launch, tile shapes from the autotuner."""
    import numpy as np
    import torch
    from paper_2606_17772_gb300 import fdcgks, flops, inputs
    cases = inputs.ensemble_members(count=args.ens_members, seed=0, nmax=args.ens_nmax)
    with fdcgks.Ensemble.from_cases(cases, fdcgks.MIXED) as ens:
        for m, c in enumerate(cases):
            ens.set_state(m, *c.initial_state())
        t0 = time.perf_counter()
        if args.ens_no_tune:
            cfg, tune_ms = ens.get_tiles(), None
        else:
            cfg, tune_ms = ens.tune(cfl=0.2, trial_steps=3)
        tune_s = time.perf_counter() - t0
        ens.run(args.warmup, cfl=0.2)
        stream = torch.cuda.ExternalStream(ens.stream)
        sampler = ClockSampler(local) if rank == 0 else None
        if sampler:
            sampler.start()
            time.sleep(0.3)
        ens.synchronize()
        barrier(world)
        launches0 = ens.launches()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ens.run(args.ens_steps, cfl=0.2)
        e1.record(stream)
        e1.synchronize()
        barrier(world)
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1), world)
        launches = ens.launches() - launches0
        t, _, st = ens.status()
        phases = ens.profile(3, cfl=0.2)
        nodes = ens.nodes
        # roofline of the point phase: FP32 flops of the interior points of
        # every member (counts of the largest member's state, the same per point)
        big = max(range(len(cases)), key=lambda m: cases[m].nx)
        cnt = flops.step_counts(cases[big], cases[big].initial_state(), 0.2 * cases[big].hx / 3.0, precision=1)
        npts = sum(c.nx * c.ny for c in cases)
        pt_flops = 2 * npts * (cnt["point_stage1"]["fp32"] + cnt["point_stage2"]["fp32"])
        pt_ms = phases["points"] / 3
        ach = pt_flops / (pt_ms / 1e3) / 1e12
        p32 = peaks["fp32"] if peaks else FP32_DERIVED_TFLOPS
        p32_src = "measured FP32 FMA pipe peak (csrc/pipe_peak.cu)" if peaks else "derived"
    sizes = sorted(c.nx for c in cases)
    return {
        "value": nodes * args.ens_steps * world / (ms / 1e3), "unit": UNIT, "dtype": "f32+f64",
        "ms_per_step": ms / args.ens_steps, "steps": args.ens_steps, "warmup": args.warmup,
        "config": {"workload": "%d periodic isentropic vortices on [0,10]^2, N log-uniform in [32, %d] "
                               "(seed 0; N from %d to %d), strength U[1,5], centre uniform; own CFL-0.2 dt "
                               "per member per step, computed on the device" % (len(cases), args.ens_nmax,
                                                                                 sizes[0], sizes[-1]),
                   "members": len(cases), "node_updates_per_step": nodes, "tiles": cfg,
                   "tile_fields": "log2 tile width of nodal, points, update; dispatch (1 persistent queue, "
                                  "0 one block per tile)",
                   "graph": "one CUDA graph per step (%d kernels)" % (launches // max(args.ens_steps, 1)),
                   "l2": "working set %.1f GB > 129 MB L2 (no flush needed)" % (nodes * 4 * 130 / 1e9)},
        "tune": {"seconds": tune_s, "best_ms_per_step": tune_ms},
        "phase_ms_per_step": {k: v / 3 for k, v in phases.items()},
        "members_time_range": [float(t.min()), float(t.max())], "members_flagged": int((st != 0).sum()),
        "roofline": {"bound": "alu", "achieved": ach, "peak": p32, "unit": "TFLOP/s",
                     "frac": ach / p32, "kernel": "ens_phase_kernel<float, points>",
                     "peak_source": p32_src, "traffic": None},
        "clocks": clocks, "gpu_launches": launches * world,
    }


def run_viscous_tube(args, world):
    """Viscous shock tube (Sec. 5.8) at 1000 x 500: throughput of a window of
    steps after the first 10, FP64 and mixed, each step with its own CFL-0.4
    time step (host loop, as in a run to t = 1).  GENO App. D constants and
    tau c2 = 25, the set with which most runs of either precision reach t = 1;
    this grid is marginal with every set tried, a run leaving the physical
    states near the shock's foot (t = 0.0015 to 0.009) or not depending on
    rounding-level details, so the window covers the first 1,000 steps."""
    import torch
    from paper_2606_17772_gb300 import fdcgks, inputs
    case = inputs.viscous_shock_tube(1000, 500, geno_variant=1, tau_c2=25.0)
    nodes = case.nx * case.ny + case.nxd * case.nyd
    out = {"config": {"workload": "viscous shock tube, [0,1]x[0,0.5], 1000x500 (+1001x501 dual), Re 200, "
                                  "Pr 0.73, no-slip walls, symmetry top, GENO App. D, tau c2 = 25; window "
                                  "after 10 steps, a CFL-0.4 step each step (host loop)",
                      "node_updates_per_step": nodes}}
    for name, prec, k in (("fp64", fdcgks.FP64, args.vt_steps), ("mixed", fdcgks.MIXED, 10 * args.vt_steps)):
        with fdcgks.Solver.from_case(case, prec) as s:
            s.set_state(*case.initial_state())
            t = 0.0
            for _ in range(10):
                dt = s.cfl_dt(0.4)
                s.step(dt)
                t += dt
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            done, failed = 0, False
            for _ in range(k):
                try:
                    dt = s.cfl_dt(0.4)          # raises once the state has no finite wave speed
                except fdcgks.FdcgksError:
                    failed = True
                    break
                s.step(dt)
                t += dt
                done += 1
            e1.record()
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world)
            bad = failed or s.check()
        out[name] = {"value": nodes * max(done, 1) * world / (ms / 1e3), "unit": UNIT,
                     "ms_per_step": ms / max(done, 1), "steps": done, "t_end": t, "nonphysical": bool(bad)}
    return out


def run_double_mach(args, world):
    """Double Mach reflection (Sec. 5.5) at 960 x 240 and 1440 x 360: split
    sides (inflow, outflow, the wall from x = 1/6, the tracked top shock)
    evaluated at each stage's time.  Throughput of a window of steps after 20
    CFL steps (dt held at the CFL value at the window's start), FP64 and
    mixed; FD-CGKS(6-2) with characteristic reconstruction."""
    import torch
    from paper_2606_17772_gb300 import fdcgks, inputs
    out = {}
    for nx, ny in ((960, 240), (1440, 360)):
        case = inputs.double_mach(nx, ny, flux_variant=62, recon_vars=1)
        nodes = case.nx * case.ny + case.nxd * case.nyd
        res = {"config": {"workload": "double Mach reflection, [0,4]x[0,1], %dx%d (+%dx%d dual), Mach 10, "
                                      "FD-CGKS(6-2), characteristic reconstruction, tau c1 = 0.05, c2 = 25; "
                                      "window after 20 CFL-0.4 steps; full_run_mixed: to t = 0.2 with a CFL-0.4 "
                                      "step each step (host loop)" % (nx, ny, case.nxd, case.nyd),
                          "node_updates_per_step": nodes}}
        for name, prec, k in (("fp64", fdcgks.FP64, args.dmr_steps), ("mixed", fdcgks.MIXED, 4 * args.dmr_steps)):
            with fdcgks.Solver.from_case(case, prec) as s:
                s.set_state(*case.initial_state())
                for _ in range(20):
                    s.step(s.cfl_dt(0.4))
                dt = s.cfl_dt(0.4)
                torch.cuda.synchronize()
                barrier(world)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.steps(dt, k)
                e1.record()
                torch.cuda.synchronize()
                ms = max_over_ranks(e0.elapsed_time(e1), world)
                bad = s.check()
                t_end = s.get_time()
            res[name] = {"value": nodes * k * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
                         "dt": dt, "t_end": t_end, "nonphysical": bool(bad)}
        # the paper's run to t = 0.2 in mixed precision (time to solution)
        from paper_2606_17772_gb300 import runs
        with fdcgks.Solver.from_case(case, fdcgks.MIXED) as s:
            s.set_state(*case.initial_state())
            torch.cuda.synchronize()
            barrier(world)
            t0 = time.perf_counter()
            try:
                t_run, n_run = runs.advance(s, 0.2, 0.4)
                ok = True
            except RuntimeError:
                t_run, n_run, ok = s.get_time(), -1, False
            torch.cuda.synchronize()
            wall = max_over_ranks(time.perf_counter() - t0, world)
            rho_max = float(s.get_state(device=False)[0][0].max())
        res["full_run_mixed"] = {"t": t_run, "steps": n_run, "seconds": wall, "physical": ok, "rho_max": rho_max}
        out["%dx%d" % (nx, ny)] = res
    return out


def run_lines(args, world):
    """The one-dimensional scheme (Sec. 2) on Woodward-Colella blast-wave lines
    (Sec. 5.3), N = 400, FD-CGKS(6-2) with App. D's GENO constants, run to
    t = 0.038 with each line's own CFL steps inside one launch: one line (the
    time to solution of the paper's run; spread over a thread-block cluster by
    default, and on one block for comparison) and a batch of 4 lines per SM
    (throughput); and the Sod and Lax tubes (Sec. 5.2, N = 100) as single
    lines."""
    import numpy as np
    import torch
    from paper_2606_17772_gb300 import fdcgks, inputs
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    wc = inputs.woodward_colella(400, flux_variant=62, geno_variant=1)
    out = {"config": {"workload": "Woodward-Colella blast waves, [0,1], N = 400, reflecting ends, "
                                  "FD-CGKS(6-2), GENO App. D, CFL 0.4, to t = 0.038, one thread block per line; "
                                  "Sod (t = 0.2) and Lax (t = 0.16) tubes, N = 100"}}
    FP64, MIXED = fdcgks.FP64, fdcgks.MIXED
    for name, case, t_end, batch, cs, prec in (("one_line", wc, 0.038, 1, 0, FP64),
                                               ("one_line_one_block", wc, 0.038, 1, 1, FP64),
                                               ("batch", wc, 0.038, 4 * sms, 0, FP64),
                                               ("one_line_mixed", wc, 0.038, 1, 0, MIXED),
                                               ("batch_mixed", wc, 0.038, 4 * sms, 0, MIXED),
                                               ("sod", inputs.sod_strip(100, 1), 0.2, 1, 0, FP64),
                                               ("lax", inputs.lax_strip(100, 1), 0.16, 1, 0, FP64)):
        W, G = inputs.line_state(case)
        Wb = np.ascontiguousarray(np.broadcast_to(W, (batch,) + W.shape))
        Gb = np.ascontiguousarray(np.broadcast_to(G, (batch,) + G.shape))
        with fdcgks.Lines.from_case(case, batch, cluster=cs, precision=prec) as L:
            L.set_state(Wb, Gb)
            L.steps(1e-9, 1)                           # warm-up: the kernel's first launch
            L.set_state(Wb, Gb)                        # back to t = 0
            torch.cuda.synchronize()
            barrier(world)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tt, kk = L.run(t_end, 0.4)
            e1.record()
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), world)
            _, bad = L.check()
        updates = float(kk.sum()) * case.nx
        out[name] = {"lines": batch, "blocks_per_line": cs or "auto", "precision": "mixed" if prec else "fp64",
                     "steps": int(kk.max()), "t": float(tt.min()), "ms": ms,
                     "value": updates * world / (ms / 1e3), "unit": UNIT, "launches": 1, "nonphysical": bool(bad)}
    return out


def run_adjoint(args, world):
    """Gradient of a density misfit after a window of steps of the 256^2 vortex
    (strength 5) with respect to the primary initial state: forward and
    adjoint (checkpoint every 50 steps) times, and the gradient along 2 random
    unit directions against central differences on the linear-reconstruction,
    c1-only collision time variant (where differences are in their linear
    regime; with GENO's nonlinear weights the vortex far field is not); and
    the GENO window on a mixed-precision solver (mixed trajectory, FP64
    reverse pass) with its gradient's distance from the FP64 one."""
    import numpy as np
    import torch
    from paper_2606_17772_gb300 import fdcgks, inputs

    def setup(case, nsteps):
        S0 = [torch.from_numpy(a).cuda() for a in case.initial_state()]
        rng = np.random.default_rng(1)
        X, Y = case.node_xy(False)
        bump = np.zeros_like(X)
        for _ in range(8):
            cx, cy = rng.uniform(0, 10, 2)
            bump += np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * 0.5 ** 2))
        return S0, bump

    out = {"config": {"workload": "isentropic vortex 256^2 (+dual), strength 5, %d steps (CFL 0.2 dt), "
                                  "J = 1/2 sum (rho - rho_target)^2 h^2, target from rho + 8 Gaussian bumps "
                                  "(sigma 0.5, amplitude 1e-3, seed 1); gradient w.r.t. primary W^0; "
                                  "checkpoint every 50 steps; geno: App. D GENO constants, linear: linear "
                                  "reconstruction with tau = 0.05 dt" % args.adj_steps}}
    fp64_geno = {}
    runs = (("geno", {}, 0, fdcgks.FP64), ("linear", dict(geno_variant=2, tau_c1=0.05, tau_c2=0.0), 2, fdcgks.FP64),
            ("geno_mixed", {}, 0, fdcgks.MIXED))
    for name, kw, ndir, prec in runs:
        case = inputs.vortex(256, strength=5.0, **kw)
        S0, bump = setup(case, args.adj_steps)
        h2 = case.hx * case.hy
        n = args.adj_steps
        with fdcgks.Solver.from_case(case, prec) as s:
            if prec == fdcgks.MIXED:
                # the FP64 run's step size and target, so that the gradients compare
                dt, target = fp64_geno["dt"], fp64_geno["target"]
            else:
                s.set_state(*S0)
                dt = s.cfl_dt(0.2)
                Wt = S0[0].clone()
                Wt[0] += torch.from_numpy(1e-3 * bump).cuda()
                s.set_state(Wt, *S0[1:])
                s.steps(dt, n)
                target = s.get_state()[0][0].clone()

            def J(Wp0):
                s.set_state(Wp0, *S0[1:])
                s.steps(dt, n)
                return 0.5 * float(((s.get_state()[0][0] - target) ** 2).sum()) * h2

            J(S0[0])                                   # warm-up (first launches, allocations)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            J0 = J(S0[0])
            torch.cuda.synchronize()
            tf = time.perf_counter() - t0
            fin = s.get_state()
            seed = [torch.zeros_like(t) for t in S0]
            seed[0][0] = (fin[0][0] - target) * h2
            s.vjp_steps(dt, 1, S0, seed, checkpoint_every=50)   # warm-up of the adjoint kernels
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g = s.vjp_steps(dt, n, S0, seed, checkpoint_every=50)
            torch.cuda.synchronize()
            ta = time.perf_counter() - t0
            checks = []
            drng = np.random.default_rng(2)
            for _ in range(ndir):
                d = torch.from_numpy(drng.standard_normal(S0[0].shape)).cuda()
                d /= d.norm()
                eps = 2.56e-6
                fd = (J(S0[0] + eps * d) - J(S0[0] - eps * d)) / (2 * eps)
                ad = float((g[0] * d).sum())
                checks.append(abs(ad - fd) / abs(fd))
        out[name] = {"J": J0, "dt": dt, "forward_ms_per_step": 1e3 * tf / n, "adjoint_ms_per_step": 1e3 * ta / n,
                     "adjoint_over_forward": ta / tf, "gradient_norm": float(g[0].norm())}
        if checks:
            out[name]["fd_rel_err"] = checks
        if name == "geno":
            fp64_geno.update(dt=dt, target=target, grad=g[0].clone())
        if prec == fdcgks.MIXED:
            out[name]["precision"] = "mixed trajectory, FP64 reverse pass"
            out[name]["grad_rel_diff_vs_fp64"] = float((g[0] - fp64_geno["grad"]).norm() / fp64_geno["grad"].norm())
    return out


GH = 3   # ghost layers of every state plane


def kernel_work(case, cnt, precision):
    """Algorithmic work of one full step (both stages) per kernel class:
    (FP64 flops, FP32 flops, bytes).  Units are the grid's own nodes and
    interface points (the kernels' extra halo units are not counted); bytes
    count each value a kernel must read or write once (r = 8 B FP64, 4 B for
    the mixed path's FP32 arrays and float-float halves):
      points  reads W and the line's averaged gradient of both grids (16 r),
              writes 25 values per solve at stage 1, 13 at stage 2;
      nodal   reads W and both gradients (12 r), writes F, G, F_t, G_t (16 r)
              at stage 1 and F_t, G_t (8 r) at stage 2;
      update  stage 1 reads 25 + 25 point values, 16 nodal fluxes and W^n,
              writes the stage state (12), the S2O4 accumulator (4) and the
              gradient base (8); stage 2 reads 13 + 13, 8, the accumulator and
              base, writes the state (12) (float-float pairs count both halves;
              a gradient base re-evaluated from the interface solution is an
              FP32 value, its low half 0 and not stored);
      ghost   3 ghost layers of 12 fields of both grids, read and write;
      cfl     4 conservative fields of every node (FP64, or both halves)."""
    r = 8 if precision == 0 else 4
    nodes = case.nx * case.ny + case.nxd * case.nyd
    pts = case.nx * case.nyd + case.nxd * case.ny
    def fl(name):
        c = cnt[name]
        return c["fp64"], c["fp32"]
    p1, p2 = fl("point_stage1"), fl("point_stage2")
    nd, nd2 = fl("node"), fl("node_stage2")
    u1, u2 = fl("update_stage1"), fl("update_stage2")
    # FP64: stage 1 reads 50 + 16 + 4, writes 24; stage 2 reads 26 + 8 + 4 + 8, writes 12.
    # mixed: stage 1 reads 66 floats and the W^n pairs (8), writes the stage state's high
    # parts (12), the accumulator pairs (8) and the gradient base (8 high parts; pairs,
    # 16, when the base is the state's own gradients); stage 2 reads 34 floats, the
    # accumulator and the base, writes the state pairs (24)
    base = 16 if case.grad_base else 8
    upd_bytes = (94 + 58) * 8 if precision == 0 else ((66 + 8 + 20 + base) + (34 + 8 + base + 24)) * 4
    ghosts = sum(2 * GH * ny + 2 * GH * (nx + 2 * GH) for nx, ny in ((case.nx, case.ny), (case.nxd, case.nyd)))
    work = {
        "points": (pts * (p1[0] + p2[0]), pts * (p1[1] + p2[1]), pts * (16 + 50 + 16 + 26) * r),
        "nodal": (nodes * (nd[0] + nd2[0]), nodes * (nd[1] + nd2[1]), nodes * (28 + 20) * r),
        "update": (nodes * (u1[0] + u2[0]), nodes * (u1[1] + u2[1]), nodes * upd_bytes),
        "ghost": (0.0, 0.0, 2 * ghosts * 12 * 2 * r),
        "cfl": (0.0, 0.0, nodes * 32.0),
    }
    return work


def kernel_fractions(work, ms_total, n_groups, steps_equiv, peaks, hbm_gbs):
    """Per kernel class: time per launch group, and the fraction of its
    roofline: ALU time at the measured FP64/FP32 pipe peaks (the two added)
    and byte time at the HBM copy bandwidth, each over the measured time; the
    larger names the bound."""
    out = {}
    for k, (f64, f32, b) in work.items():
        t = ms_total.get(k, 0.0) / 1e3
        if t <= 0:
            continue
        units = steps_equiv[k]
        alu = units * (f64 / (peaks["fp64"] * 1e12) + f32 / (peaks["fp32"] * 1e12)) / t
        mem = units * b / (hbm_gbs * 1e9) / t
        out[k] = {"ms_per_launch_group": 1e3 * t / max(n_groups.get(k, 1), 1),
                  "bound": "alu" if alu >= mem else "hbm", "frac": max(alu, mem), "alu_frac": alu, "hbm_frac": mem,
                  "achieved_tflops": units * (f64 + f32) / t / 1e12, "achieved_gbs": units * b / t / 1e9}
    return out


def rho_errors(got, ref):
    """L1 (mean |e| / mean |rho|) and L-infinity (max |e| / max |rho|) of the
    density over the nodes of both grids."""
    import numpy as np
    a = np.concatenate([got[0][0].ravel(), got[2][0].ravel()])
    b = np.concatenate([ref[0][0].ravel(), ref[2][0].ravel()])
    return [float(np.abs(a - b).mean() / np.abs(b).mean()), float(np.abs(a - b).max() / np.abs(b).max())]


def cpu_baseline_leg(args):
    """The CPU-baseline leg: the oracle as it stands, single thread, on
    oracle-sized samples of the bench's workloads (timed: the baseline), and
    the same samples on the GPU in FP64 and mixed precision, so that each
    path's error against the FP64 oracle is stated per workload."""
    import numpy as np
    import oracle
    import torch
    from paper_2606_17772_gb300 import fdcgks, inputs

    def gpu(case, dts, precision):
        with fdcgks.Solver.from_case(case, precision) as s:
            s.set_state(*case.initial_state())
            for dt in dts:
                s.step(dt)
            out = s.get_state(device=False)
            return out, bool(s.check())

    warm = inputs.vortex(16)            # load the library outside the timing
    oracle.steps(oracle.make_params(**warm.oracle_kwargs()), 0.01, 1, *warm.initial_state())
    res, timing = {}, {}
    # isentropic vortex (bench constants), fixed CFL-0.2 step from the initial state
    v = inputs.vortex(64)
    pv = oracle.make_params(**v.oracle_kwargs())
    S = v.initial_state()
    nv = 20
    dt = oracle.cfl_dt(pv, 0.2, S[0], S[2])
    t0 = time.perf_counter()
    ref = oracle.steps(pv, dt, nv, *S)
    el = time.perf_counter() - t0
    timing["vortex"] = ((v.nx * v.ny + v.nxd * v.nyd) * nv, el)
    for name, prec in (("fp64", fdcgks.FP64), ("mixed", fdcgks.MIXED)):
        got, bad = gpu(v, [dt] * nv, prec)
        res.setdefault("vortex64", {})[name] = rho_errors(got, ref)
    # viscous shock tube (Sec. 5.8 constants, no-slip walls): the oracle's own CFL-0.4 steps
    tb = inputs.viscous_shock_tube(40, 20)
    pt = oracle.make_params(**tb.oracle_kwargs())
    S = tb.initial_state()
    dts = []
    t0 = time.perf_counter()
    for _ in range(20):
        dts.append(oracle.cfl_dt(pt, 0.4, S[0], S[2]))
        S = oracle.steps(pt, dts[-1], 1, *S)
    timing["tube"] = ((tb.nx * tb.ny + tb.nxd * tb.nyd) * 20, time.perf_counter() - t0)
    for name, prec in (("fp64", fdcgks.FP64), ("mixed", fdcgks.MIXED)):
        got, bad = gpu(tb, dts, prec)
        res.setdefault("tube40x20", {})[name] = rho_errors(got, S)
    # the case amplifies rounding where the diaphragm meets the wall: the
    # oracle's own response to a 1e-7 relative perturbation (FP32 rounding
    # level) is the scale the mixed path's error compares with
    rng = np.random.default_rng(1)
    Sp = tuple(a * (1 + 1e-7 * rng.standard_normal(a.shape)) for a in tb.initial_state())
    for dt in dts:
        Sp = oracle.steps(pt, dt, 1, *Sp)
    res["tube40x20"]["spread"] = rho_errors(Sp, S)
    # smallest member of the bench ensemble, through the ensemble (mixed) path
    cases = inputs.ensemble_members(count=args.ens_members, seed=0, nmax=args.ens_nmax)
    m = min(cases, key=lambda c: c.nx)
    pm = oracle.make_params(**m.oracle_kwargs())
    S = m.initial_state()
    dt = oracle.cfl_dt(pm, 0.2, S[0], S[2])
    t0 = time.perf_counter()
    ref = oracle.steps(pm, dt, 20, *S)
    timing["member"] = ((m.nx * m.ny + m.nxd * m.nyd) * 20, time.perf_counter() - t0)
    with fdcgks.Ensemble.from_cases([m], fdcgks.MIXED) as ens:
        ens.set_state(0, *m.initial_state())
        ens.run(20, dt=[dt])
        ens.synchronize()
        got = ens.get_state(0, device=False)
    res["member"] = {"mixed": rho_errors(got, ref), "n": m.nx}
    torch.cuda.synchronize()
    units, secs = timing["vortex"]
    base = {"value": units / secs, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "isentropic vortex 64^2 (+dual), 20 steps, %.1f s, single thread" % secs,
            "sample_short": "vortex 64^2 x20",
            "other_samples": {k: {"value": u / t, "seconds": t} for k, (u, t) in timing.items() if k != "vortex"}}
    return base, res


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    from paper_2606_17772_gb300 import build as fbuild
    from paper_2606_17772_gb300 import fdcgks, flops, inputs

    fbuild.build()
    world, rank, local = dist_setup(args)
    if args.ensemble_only:
        ens = run_ensemble(args, world, rank, local)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "ensemble": ens}), flush=True)
        return 0
    peaks = pipe_peaks() if not args.no_peaks else {"fp64": FP64_DERIVED_TFLOPS, "fp32": FP32_DERIVED_TFLOPS}
    hbm, hbm_src = hbm_peak()
    n = args.n
    case = inputs.vortex(n)
    S_host = case.initial_state()
    S_dev = [torch.from_numpy(a).cuda() for a in S_host]
    nodes = 2 * n * n

    results = {}
    for name, prec in (("fp64", fdcgks.FP64), ("mixed", fdcgks.MIXED)):
        if name == "mixed" and args.no_mixed:
            continue
        with fdcgks.Solver.from_case(case, prec) as s:
            s.set_state(*S_dev)
            dt = s.cfl_dt(0.2)
            ms, pms, pn, launches, clocks = timed_steps(s, dt, args.steps, args.warmup, world, local,
                                                        sample_clocks=(name == "fp64" and rank == 0))
            out = s.get_state()
            assert not s.check(), "non-physical state during the benchmark"
            # the CFL reduction, timed apart (it is not part of a fixed-dt step)
            s.set_profiling(True)
            for _ in range(5):
                s.cfl_dt(0.2)
            cms, cn, _ = s.get_profile()
            s.set_profiling(False)
            pms["cfl"], pn["cfl"] = cms["cfl"], cn["cfl"]
        ms_max = max_over_ranks(ms, world)
        cnt = flops.step_counts(case, S_host, dt, precision=0 if name == "fp64" else 1)
        work = kernel_work(case, cnt, 0 if name == "fp64" else 1)
        equiv = {k: args.steps for k in ("points", "nodal", "update", "ghost")}
        equiv["cfl"] = 5
        kf = kernel_fractions(work, pms, pn, equiv, peaks, hbm)
        # measured DRAM bytes per launch (profiles/dram_traffic.json) beside the
        # algorithmic bytes per launch (a step launches 4 point, 2 nodal, 2 update kernels)
        rt = "double" if name == "fp64" else "float"
        for cls, kname, per_step in (("points", "point_pair_kernel<%s>" % rt, 4), ("nodal", "nodal_kernel<%s>" % rt, 2),
                                     ("update", "update_kernel<%s>" % rt, 2)):
            if cls in kf:
                kf[cls]["algorithmic_bytes_per_launch"] = work[cls][2] / per_step
                kf[cls]["dram_bytes_per_launch"] = profiled_traffic(kname, n)
        results[name] = dict(ms=ms_max, prof_ms=pms, prof_n=pn, launches=launches, clocks=clocks, dt=dt, cnt=cnt,
                             kernels=kf, state=[t.cpu().numpy() for t in out] if rank == 0 else None)

    fp = results["fp64"]
    value = nodes * args.steps * world / (fp["ms"] / 1e3)
    wset = nodes * 8 * (24 + 24 + 12) / 1e9 + nodes * 8 * 66 / 1e9
    step_ms = {k: v for k, v in fp["prof_ms"].items() if k != "cfl"}
    pk = fp["kernels"]["points"]
    roof = {"bound": "alu", "achieved": pk["achieved_tflops"], "peak": peaks["fp64"], "unit": "TFLOP/s",
            "frac": pk["alu_frac"], "traffic": profiled_traffic("point_pair_kernel<double>", n),
            "kernel": "point_kernel<double> (Type A + B interface points)",
            "peak_source": "measured FP64 FMA pipe (csrc/pipe_peak.cu), this run",
            "step_share": step_ms["points"] / max(sum(step_ms.values()), 1e-9)}

    full = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": fp["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "isentropic vortex %d^2 (+%d^2 dual), periodic [0,10]^2, strength 5, "
                                   "FD-CGKS(6-4), GENO App. D, CFL 0.2" % (n, n),
                       "workload_short": "isentropic vortex %d^2+dual, FD-CGKS(6-4), App.D GENO, CFL 0.2" % n,
                       "l2": "working set %.1f GB > 129 MB L2, no flush" % wset,
                       "l2_short": "%.1f GB > L2, no flush" % wset},
            "roofline": roof, "clocks": fp["clocks"], "gpu_launches": fp["launches"] * world,
            "peaks": {"fp64_tflops": peaks["fp64"], "fp32_tflops": peaks["fp32"], "hbm_gbs": hbm,
                      "hbm_source": hbm_src, "fp64_derived": FP64_DERIVED_TFLOPS,
                      "fp32_derived": FP32_DERIVED_TFLOPS},
            "kernels": {"fp64": fp["kernels"]},
            "flops_per_node_update": {"fp64": fp["cnt"]["per_node_update_total"]}}

    if "mixed" in results:
        mx = results["mixed"]
        mval = nodes * args.steps * world / (mx["ms"] / 1e3)
        err = None
        if rank == 0:
            a, b = mx["state"], fp["state"]
            err = {"rho_L1_Linf": rho_errors(a, b), "after_steps": args.warmup + 2 * args.steps}
        mk = mx["kernels"]["points"]
        full["mixed"] = {"value": mval, "unit": UNIT, "dtype": "f32+f64", "ms_per_step": mx["ms"] / args.steps,
                         "err_vs_fp64_gpu": err, "points_frac": mk["alu_frac"],
                         "points_tflops": mk["achieved_tflops"], "gpu_launches": mx["launches"] * world}
        full["kernels"]["mixed"] = mx["kernels"]
        full["flops_per_node_update"]["mixed"] = mx["cnt"]["per_node_update_total"]

    if not args.no_e2e:
        # end to end through the C ABI with host state in pinned memory
        pin = [torch.from_numpy(a).pin_memory() for a in S_host]
        outp = [torch.empty_like(t).pin_memory() for t in pin]
        with fdcgks.Solver.from_case(case, fdcgks.FP64) as s:
            s.set_state(*pin)
            dt = s.cfl_dt(0.2)
            for _ in range(max(1, args.warmup)):
                s.set_state(*pin)
                s.step(dt)
                s.get_state(out=outp)
            barrier(world)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                s.set_state(*pin)
                s.step(dt)
                s.get_state(out=outp)
            torch.cuda.synchronize()
            el = max_over_ranks(time.perf_counter() - t0, world)
        nbytes = sum(t.numel() * 8 for t in pin)
        full["e2e"] = {"value": nodes * args.steps * world / el, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                       "d2h_bytes_per_step": nbytes, "ms_per_step": 1e3 * el / args.steps}

    if not args.no_ensemble:
        full["ensemble"] = run_ensemble(args, world, rank, local, peaks)
    if not args.no_viscous_tube:
        full["viscous_tube"] = run_viscous_tube(args, world)
    if not args.no_double_mach:
        full["double_mach"] = run_double_mach(args, world)
    if not args.no_lines:
        full["lines_1d"] = run_lines(args, world)
    if not args.no_adjoint:
        full["adjoint"] = run_adjoint(args, world)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, errs = cpu_baseline_leg(args)
        full["cpu_baseline"] = base
        full["err_vs_oracle"] = errs
        try:
            arate, wall, ncores = oracle_rate_all_cores(64, 2)
            full["cpu_baseline"]["all_cores"] = {
                "value": arate, "unit": UNIT, "cores": ncores, "kind": "oracle",
                "sample": "isentropic vortex 64^2 (+dual), 2 steps, one copy per core, %.1f s wall" % wall}
        except Exception as e:                   # the auxiliary leg never costs the line
            full["cpu_baseline"]["all_cores"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if rank == 0:
        if args.detail:
            with open(args.detail, "w") as fh:
                json.dump(full, fh, indent=1)
        print(json.dumps(compact(full), separators=(",", ":")), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _r(x, d=4):
    """x rounded to d significant digits (JSON line length); large values as integers."""
    if isinstance(x, float) and math.isfinite(x) and x != 0.0:
        v = float("%.*g" % (d, x))
        return int(v) if abs(v) >= 1e5 else v
    return x


def _rl(v):
    return [_r(x, 3) for x in v]


def compact(full):
    """The printed line: the contract's keys and the figures the metric names,
    rounded, in an order that puts the headline numbers first (every figure is
    in the --detail file)."""
    line = {k: full[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                                 "higher_is_better", "scaling", "vs_baseline", "dtype", "data")}
    line["value"], line["ms_per_step"] = _r(line["value"]), _r(line["ms_per_step"])
    line["config"] = {"workload": full["config"]["workload_short"], "l2": full["config"]["l2_short"]}
    ro = full["roofline"]
    line["roofline"] = {"bound": ro["bound"], "achieved": _r(ro["achieved"]), "peak": _r(ro["peak"]),
                        "unit": ro["unit"], "frac": _r(ro["frac"], 3), "traffic": ro["traffic"],
                        "kernel": "points fp64"}
    c = full.get("clocks") or {}
    line["clocks"] = {"sm_mhz": c.get("sm_mhz"), "sm_max_mhz": c.get("sm_max_mhz"), "reasons": c.get("reasons")}
    line["gpu_launches"] = full["gpu_launches"]
    if "e2e" in full:
        e = full["e2e"]
        line["e2e"] = {"value": _r(e["value"]), "unit": e["unit"], "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                       "d2h_bytes_per_step": e["d2h_bytes_per_step"]}
    if "mixed" in full:
        m = full["mixed"]
        line["mixed"] = {"value": _r(m["value"]), "frac": _r(m["points_frac"], 3),
                         "err_fp64": _rl(m["err_vs_fp64_gpu"]["rho_L1_Linf"]) if m["err_vs_fp64_gpu"] else None}
    if "err_vs_oracle" in full:
        line["err_vs_oracle"] = {k: {p: _rl(v) if isinstance(v, list) else v for p, v in d.items()}
                                 for k, d in full["err_vs_oracle"].items()}
    # per kernel class its fraction of its own bound, suffixed a (FP64/FP32 FMA
    # pipe) or h (HBM bandwidth), e.g. "points 0.52a update 0.12h"
    line["kernel_frac"] = {p: " ".join("%s %.2f%s" % (k, v["frac"], "h" if v["bound"] == "hbm" else "a")
                                       for k, v in kk.items()) for p, kk in full["kernels"].items()}
    pk = full["peaks"]
    line["peaks"] = [_r(pk["fp64_tflops"], 3), _r(pk["fp32_tflops"], 3), _r(pk["hbm_gbs"], 4)]
    if "ensemble" in full:
        en = full["ensemble"]
        line["ensemble"] = {"value": _r(en["value"]), "frac": _r(en["roofline"]["frac"], 3)}
    if "viscous_tube" in full:
        vt = full["viscous_tube"]
        # [FP64 value, mixed value, every run physical]
        line["viscous_tube"] = [_r(vt["fp64"]["value"], 3), _r(vt["mixed"]["value"], 3),
                                not (vt["fp64"]["nonphysical"] or vt["mixed"]["nonphysical"])]
    if "cpu_baseline" in full:
        b = full["cpu_baseline"]
        line["cpu_baseline"] = {"value": _r(b["value"]), "unit": b["unit"], "cores": b["cores"], "kind": b["kind"],
                                "sample": b["sample_short"]}
        ac = b.get("all_cores", {})
        if "value" in ac:
            line["cpu_baseline"]["all_cores"] = [_r(ac["value"]), ac["cores"]]
    return line


if __name__ == "__main__":
    sys.exit(main())
