"""The benchmark's algorithmic flop counts (paper_2606_17772_gb300/flops.py):
the kernel arithmetic instantiated on the host with an operation-counting
scalar.  Host logic only: the counting build compiles, every kernel class has
a positive count in its own precision (FP64 path: all FP64; mixed path on the
vortex: all FP32, the time coefficients there being in their FP32 range), and
the second stage of a point or a node does less than the first (no F and
W~ values, no nodal F and G)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2606_17772_gb300 import flops, inputs  # noqa: E402


def test_step_counts_fp64_and_mixed():
    case = inputs.vortex(32)
    S = case.initial_state()
    for prec, own, other in ((0, "fp64", "fp32"), (1, "fp32", "fp64")):
        c = flops.step_counts(case, S, 0.05, precision=prec, nsample=400)
        for k in ("point_stage1", "point_stage2", "node", "node_stage2", "update_stage1", "update_stage2"):
            assert c[k][own] > 0 and c[k][other] == 0, (prec, k, c[k])
        assert c["point_stage2"][own] < c["point_stage1"][own]
        assert c["node_stage2"][own] < c["node"][own]
        assert 5e3 < c["per_node_update_total"][own] < 5e4
