"""Serving with continuous batching: results in the mix equal results alone.

Requests from the seeded serving stream (n in [10, 60], 200-5000 Clifford
gates, 0-14 T/RZ) are submitted together; the server's slots propagate them
concurrently on their own streams.  Every result must equal qx_propagate of
the same circuit alone: the same strings and, in FP64, bit-identical weights
(every sum in the kernels has a fixed order, only the term order may differ).
Every served result is also compared with the oracle's plan mode: exact
string sets, FP64 weights within 1e-12 |w| + 1e-15, FP32 weights within
1e-5 |w| + 1e-7.
"""
import os

import pytest

from gpu_util import compare_gen
from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def _alone(n, instrs, precision=64):
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan, precision=precision)
    return [res.export_dict(g) for g in range(n)]


def test_mix_equals_alone_fp64():
    reqs = W.serving_stream(11, count=48)
    srv = qx.Server(slots=6)
    tickets = [(srv.submit(n, instrs), n, instrs) for _, n, instrs in reqs]
    for t, n, instrs in tickets:
        res, lat = srv.wait(t)
        assert lat > 0
        want = _alone(n, instrs)
        ref = O.propagate(n, instrs, mode="plan", threads=os.cpu_count() or 1)
        for g in range(n):
            got = res.export_dict(g)
            assert got == want[g], (t, g)
            compare_gen(got, O.as_dict(ref[g]), f"request {t} generator {g}")
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_budget_admission_reruns_exclusive():
    """A budget so small that heavy requests exceed their per-slot share: they
    are run again alone with the whole budget, with unchanged results."""
    heavy = W.fan_in_heavy(3, n=20, n_s=10, total=700, tail=100)  # 10 x 1024 terms
    light = [W.random_layers(s) for s in range(6)]
    srv = qx.Server(slots=4, hbm_budget=4 * 200_000)  # 200 KB per slot; heavy needs ~290 KB
    tickets = [(srv.submit(*heavy), heavy)] + [(srv.submit(*c), c) for c in light]
    for t, (n, instrs) in tickets:
        res, _ = srv.wait(t)
        want = _alone(n, instrs)
        ref = O.propagate(n, instrs, mode="plan", threads=os.cpu_count() or 1)
        for g in range(n):
            got = res.export_dict(g)
            assert got == want[g]
            compare_gen(got, O.as_dict(ref[g]), f"generator {g}")
    assert srv.stats()["retried_exclusive"] >= 1
    srv.close()


def test_fp32_serving_matches_fp64_alone():
    reqs = W.serving_stream(12, count=16)
    srv = qx.Server(slots=4, precision=32)
    tickets = [(srv.submit(n, instrs), n, instrs) for _, n, instrs in reqs]
    worst = 0.0
    for t, n, instrs in tickets:
        res, _ = srv.wait(t)
        want = _alone(n, instrs, precision=64)
        ref = O.propagate(n, instrs, mode="plan", threads=os.cpu_count() or 1)
        for g in range(n):
            got = res.export_dict(g)
            assert got.keys() == want[g].keys()
            for s, w in want[g].items():
                d = abs(got[s] - w)
                assert d <= 1e-5 * abs(w) + 1e-7
            for s, w in O.as_dict(ref[g]).items():
                d = abs(got[s] - w)
                assert d <= 1e-5 * abs(w) + 1e-7, (t, g, s, got[s], w)
                if abs(w) > 1e-3:
                    worst = max(worst, d / abs(w))
    print(f"FP32 serving vs the FP64 oracle: max relative error {worst:.2e}")
    srv.close()
