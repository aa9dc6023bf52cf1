"""Algorithmic flop counts of one FD-CGKS step per node update.

The device arithmetic (csrc/fdcgks_math.cuh) is instantiated on the host with
an operation-counting scalar (csrc/flop_count.cpp).  Counting convention:
add, sub, mul = 1 flop (a fused multiply-add = 2), div = 1, sqrt = 1 and one
call of exp, erfc, tanh or expm1 = 1; these kinds are also returned
separately.  Only the reconstruction has data-dependent branches (the GENO
path function skips the sub-stencil blend where chi = 1), so its counts are
averaged over lines sampled from the actual state; the kinetic solves and
the compact flux have fixed counts.

Per stage and per pair of nodes (one primary, one dual) on a periodic grid
the kernels process: one Type A and one Type B point (each 2 lines x 4
components of interface reconstruction + 2 interface solves + the W~
combination), two nodes (8 node reconstructions + 1 nodal flux each) and two
node updates (compact fluxes, the operator and the S2O4 stage combination).
Glue arithmetic outside the counted functions (combinations in the point
and update kernels) is tallied here by hand, per the kernel source.
"""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "flop_count.cpp")
LIB = os.path.join(HERE, "_build", "libflopcount.so")
KINDS = ["add", "mul", "div", "sqrt", "exp", "erfc", "tanh", "expm1"]
_lib = None


def _load():
    global _lib
    if _lib is None:
        hdr = os.path.join(HERE, "csrc", "fdcgks_math.cuh")
        if (not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC)
                or os.path.getmtime(LIB) < os.path.getmtime(hdr)):
            os.makedirs(os.path.dirname(LIB), exist_ok=True)
            tmp = LIB + ".tmp.%d" % os.getpid()
            subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-I", os.path.join(HERE, "csrc"),
                            "-o", tmp, SRC], check=True)
            os.replace(tmp, LIB)
        _lib = ctypes.CDLL(LIB)
    return _lib


def _count(what, precision, variant, gas, normal, h, inp):
    """Average counts per item: {'fp64': {kind: n}, 'fp32': {kind: n}}."""
    inp = np.ascontiguousarray(inp, dtype=np.float64)
    n = inp.shape[0]
    out = (ctypes.c_longlong * 16)()
    g = (ctypes.c_double * 6)(*gas)
    _load().flop_count(what, precision, variant, g, normal, ctypes.c_double(h), n,
                       inp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out)
    vals = np.array(list(out), dtype=np.float64) / max(n, 1)
    return {"fp64": dict(zip(KINDS, vals[:8])), "fp32": dict(zip(KINDS, vals[8:]))}


def _total(d):
    return float(sum(d.values()))


def _add(a, b, s=1.0):
    return {k: a.get(k, 0.0) + s * b.get(k, 0.0) for k in KINDS}


def _sample_lines(case, state, nsample, rng):
    """Interface-reconstruction inputs [Q(4), Qx(4)] of random lines of both grids, both directions."""
    Wp, Gp, Wd, Gd = state
    rows = []
    for W, G in ((Wp, Gp), (Wd, Gd)):
        ny, nx = W.shape[1:]
        for _ in range(nsample // 4):
            c = rng.integers(0, 4)
            i, j = rng.integers(0, nx), rng.integers(0, ny)
            d = rng.integers(0, 2)
            if d == 0:
                idx = [(i - 1 + m) % nx for m in range(4)]
                rows.append(np.concatenate([W[c, j, idx], G[0, c, j, idx]]))
            else:
                idx = [(j - 1 + m) % ny for m in range(4)]
                rows.append(np.concatenate([W[c, idx, i], G[1, c, idx, i]]))
    return np.array(rows)


def _sample_nodes(case, state, nsample, rng):
    Wp, Gp, Wd, Gd = state
    rows = []
    for W, G in ((Wp, Gp), (Wd, Gd)):
        ny, nx = W.shape[1:]
        for _ in range(nsample // 4):
            c = rng.integers(0, 4)
            i, j = rng.integers(0, nx), rng.integers(0, ny)
            if rng.integers(0, 2) == 0:
                idx = [(i - 1 + m) % nx for m in range(3)]
                rows.append(np.concatenate([W[c, j, idx], G[0, c, j, idx]]))
            else:
                idx = [(j - 1 + m) % ny for m in range(3)]
                rows.append(np.concatenate([W[c, idx, i], G[1, c, idx, i]]))
    return np.array(rows)


def step_counts(case, state, dt, precision=0, nsample=4000, seed=0):
    """Flops of one full S2O4 step, per node update and per point-kernel launch group.

    Returns a dict with 'per_node_update' (fp64 / fp32 kind dicts and totals),
    'point_stage1' / 'point_stage2' (flops of one interface point), 'node' /
    'node_stage2' (one node of the nodal kernel at stage 1 / 2),
    'update_stage1' / 'update_stage2' (one node of the update kernel), each split into fp64 / fp32, and the unit
    counts used.
    """
    rng = np.random.default_rng(seed)
    gas = (case.gamma, case.mu, case.Pr, case.tau_c1, case.tau_c2, dt)
    v, h = case.geno_variant, min(case.hx, case.hy)
    R = "fp32" if precision == 1 else "fp64"
    rec_i = _count(0, precision, v, gas, 0, h, _sample_lines(case, state, nsample, rng))
    rec_n = _count(1, precision, v, gas, 0, h, _sample_nodes(case, state, nsample, rng))
    W = np.array([1.0, 0.4, -0.3, 2.7])
    solve_in = np.concatenate([W, W * 1.01, 0.1 * np.ones(4), 0.12 * np.ones(4), 0.05 * np.ones(4)])[None]
    solve = _count(2, precision, v, gas, 0, h, solve_in)
    nodal = _count(3, precision, v, gas, 0, h, np.concatenate([W, 0.1 * np.ones(8)])[None])
    nodal_t = _count(5, precision, v, gas, 0, h, np.concatenate([W, 0.1 * np.ones(8)])[None])
    cflux = _count(4, precision, v, gas, case.flux_variant, h, np.array([[0.7, 1, 2, 3, 1.5, 2.5]]))

    def glue(n_r, n_64):
        d = {"fp64": {k: 0.0 for k in KINDS}, "fp32": {k: 0.0 for k in KINDS}}
        d[R]["add"] += n_r
        d["fp64"]["add"] += n_64
        return d

    def comb(*terms):
        out = {"fp64": {k: 0.0 for k in KINDS}, "fp32": {k: 0.0 for k in KINDS}}
        for t, s in terms:
            for p in ("fp64", "fp32"):
                out[p] = _add(out[p], t[p], s)
        return out

    # glue of the point kernel: tangential derivatives (16) + W~ combination
    # (12 per component for the time derivatives, 12 more for the values at stage 1)
    # + the positivity check of the four reconstructed states (5 each)
    point1 = comb((rec_i, 8), (solve, 2), (glue(16 + 4 * 24 + 20, 0), 1))
    point2 = comb((rec_i, 8), (solve, 2), (glue(16 + 4 * 12 + 20, 0), 1))
    node = comb((rec_n, 8), (nodal, 1))
    node2 = comb((rec_n, 8), (nodal_t, 1))       # second stage: F_t, G_t only
    # update kernel per node: stage 1 evaluates 8 compact fluxes per component
    # (F, F_t in x and y at both faces), 18 operator/gradient flops in the compute
    # type and 19 FP64 flops of the S2O4 combination; stage 2 evaluates 4 fluxes,
    # 9 + 8 flops; 6 FP64 flops of the positivity check per node
    if precision == 1:
        # mixed path: the S2O4 increments are formed in FP32 (stage 1: 5 + 5 per
        # component for W* and W_acc, 2 x 2 for the gradients; stage 2: 3 + 2 x 2)
        # and added to float-float pairs (8 flops per addition: 4 per component at
        # stage 1, 3 at stage 2); positivity check 6 flops per node, all FP32
        upd1 = comb((cflux, 32), (glue(4 * (18 + 14 + 32) + 6, 0), 1))
        upd2 = comb((cflux, 16), (glue(4 * (9 + 7 + 24) + 6, 0), 1))
    else:
        upd1 = comb((cflux, 32), (glue(4 * 18, 4 * 19 + 6), 1))
        upd2 = comb((cflux, 16), (glue(4 * 9, 4 * 8 + 6), 1))
    # per node pair per step: 2 points + 2 nodes + 2 updates in each stage
    pair = comb((point1, 2), (point2, 2), (node, 2), (node2, 2), (upd1, 2), (upd2, 2))
    per_node = {p: {k: pair[p][k] / 2.0 for k in KINDS} for p in ("fp64", "fp32")}
    return {
        "per_node_update": per_node,
        "per_node_update_total": {p: _total(per_node[p]) for p in per_node},
        "point_stage1": {p: _total(point1[p]) for p in point1},
        "point_stage2": {p: _total(point2[p]) for p in point2},
        "node": {p: _total(node[p]) for p in node},
        "node_stage2": {p: _total(node2[p]) for p in node2},
        "update_stage1": {p: _total(upd1[p]) for p in upd1},
        "update_stage2": {p: _total(upd2[p]) for p in upd2},
        "units": {"recon_interface": rec_i, "recon_node": rec_n, "iface_solve": solve, "nodal_flux": nodal,
                  "compact_flux": cflux},
    }
