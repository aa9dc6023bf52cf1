"""The bench's printed line: the contract's keys, and short enough that a
consumer keeping only the last ~1500 characters of the output still has it
whole (the detailed figures go to the --detail file).  Host logic only: a
`full` record with every section the bench fills, at realistic magnitudes."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402

KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "gpu_launches", "e2e", "cpu_baseline")


def _kernel(frac, bound):
    return {"ms_per_launch_group": 1.234567, "bound": bound, "frac": frac, "alu_frac": frac, "hbm_frac": 0.01,
            "achieved_tflops": 0.6543210, "achieved_gbs": 123.456789}


def _full():
    ks = {k: _kernel(0.523456789, "alu" if k in ("points", "nodal", "update") else "hbm")
          for k in ("points", "nodal", "update", "ghost", "cfl")}
    km = {k: _kernel(0.523456789, "alu" if k in ("points", "nodal") else "hbm")
          for k in ("points", "nodal", "update", "ghost", "cfl")}
    return {
        "metric": bench.METRIC, "value": 50538038.3899335, "unit": bench.UNIT, "n_gpus": 1, "steps": 20,
        "warmup": 5, "ms_per_step": 41.49650573730469, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "isentropic vortex 1024^2 (+1024^2 dual), periodic [0,10]^2, strength 5, "
                               "FD-CGKS(6-4), GENO App. D, CFL 0.2",
                   "l2": "working set 2.1 GB > 129 MB L2, no flush",
                   "workload_short": "isentropic vortex 1024^2+dual, FD-CGKS(6-4), App.D GENO, CFL 0.2",
                   "l2_short": "2.1 GB > L2, no flush"},
        "roofline": {"bound": "alu", "achieved": 0.658065915, "peak": 1.19123456, "unit": "TFLOP/s",
                     "frac": 0.5523456, "traffic": 527123456, "kernel": "x", "peak_source": "y",
                     "step_share": 0.7739228951473514},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 7},
        "gpu_launches": 240,
        "peaks": {"fp64_tflops": 1.19123, "fp32_tflops": 72.51234, "hbm_gbs": 6691.5, "hbm_source": "m",
                  "fp64_derived": 1.2, "fp32_derived": 80.5},
        "kernels": {"fp64": ks, "mixed": km},
        "mixed": {"value": 1.2412345e9, "ms_per_step": 1.7123456, "points_frac": 0.251234, "points_tflops": 20.1,
                  "err_vs_fp64_gpu": {"rho_L1_Linf": [8.412345e-8, 1.512345e-6], "after_steps": 25},
                  "gpu_launches": 240},
        "e2e": {"value": 48120321.95150462, "unit": bench.UNIT, "h2d_bytes_per_step": 201326592,
                "d2h_bytes_per_step": 201326592, "ms_per_step": 43.58},
        "err_vs_oracle": {"vortex64": {"fp64": [1.2345678e-14, 2.3456789e-13], "mixed": [3.4567e-8, 4.5678e-7]},
                          "tube40x20": {"fp64": [1.2345678e-14, 2.3456789e-13], "mixed": [3.4567e-8, 4.5678e-7],
                                        "spread": [3.4567e-8, 4.5678e-7]},
                          "member": {"mixed": [3.4567e-8, 4.5678e-7], "n": 33}},
        "ensemble": {"value": 1.1212345e9, "ms_per_step": 22.312345, "members_flagged": 0,
                     "roofline": {"frac": 0.2212345}},
        "viscous_tube": {"fp64": {"value": 4.9123456e7, "nonphysical": False},
                         "mixed": {"value": 7.1123456e8, "nonphysical": False}},
        "cpu_baseline": {"value": 12296.199277825262, "unit": bench.UNIT, "cores": 1, "kind": "oracle",
                         "sample": "s", "sample_short": "vortex 64^2, 20 steps",
                         "all_cores": {"value": 171234.5678, "cores": 16}},
        "double_mach": {"960x240": {"fp64": {"value": 4.0512345e7}, "mixed": {"value": 9.0123456e8}},
                        "1440x360": {"fp64": {"value": 4.3412345e7}, "mixed": {"value": 1.0612345e9}}},
        "adjoint": {"geno": {"adjoint_over_forward": 59.951234}},
    }


def test_line_has_contract_keys_and_fits_a_short_tail():
    line = bench.compact(_full())
    text = json.dumps(line)
    for k in KEYS:
        assert k in line, k
    assert line["roofline"]["frac"] > 0 and line["roofline"]["peak"] > 0
    assert set(line["err_vs_oracle"]) == {"vortex64", "tube40x20", "member"}
    text = json.dumps(line, separators=(",", ":"))
    assert len(text) < 1450, len(text)
    assert json.loads(text) == line
