"""Serving with continuous batching: results in the mix equal results alone.

Requests from the seeded serving stream (n in [10, 60], 200-5000 Clifford
gates, 0-14 T/RZ) are submitted together; the server plans each as a
push-through plan and propagates admitted requests in batches that share one
term store.  Every result must equal qx_propagate of the same circuit's
push-through plan alone: the same strings and, in FP64, bit-identical weights
(the batched kernels do the same arithmetic per term; only the term order may
differ).  Every served result is also compared with the oracle's push-through
mode (pinned to dense matrices): exact string sets, FP64 weights within
1e-12 |w| + 1e-15, FP32 weights within 1e-5 |w| + 1e-7.
"""
import os

import pytest

from gpu_util import compare_gen
from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def _alone(n, instrs, precision=64):
    plan = qx.group_ops(qx.load_circuit(n, instrs), pushthrough=True)
    res = qx.propagate(plan, precision=precision)
    return [res.export_dict(g) for g in range(n)]


def _check_fp64(res, n, instrs, label):
    want = _alone(n, instrs)
    ref = O.propagate(n, instrs, mode="push", threads=CORES)
    for g in range(n):
        got = res.export_dict(g)
        assert got == want[g], (label, g)
        compare_gen(got, O.as_dict(ref[g]), f"{label} generator {g}")


def test_mix_equals_alone_fp64():
    reqs = W.serving_stream(11, count=48)
    # two wider circuits (two words per string) in the same stream: batches
    # hold one word count
    wide = [W.random_pairs(5, n=70, n_cliff=600, n_rz=6), W.random_pairs(6, n=100, n_cliff=800, n_rz=5)]
    items = [(n, instrs) for _, n, instrs in reqs[:20]] + wide + [(n, i) for _, n, i in reqs[20:]]
    srv = qx.Server(slots=2)
    tickets = [(srv.submit(n, instrs), n, instrs) for n, instrs in items]
    for t, n, instrs in tickets:
        res, lat = srv.wait(t)
        assert lat > 0
        _check_fp64(res, n, instrs, f"request {t}")
    st = srv.stats()
    assert st["completed"] == len(items) and st["failed"] == 0
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_requests_that_wait_share_a_batch():
    """A request whose bound exceeds the budget runs by itself first (its
    exact size fits); the light requests submitted behind it wait for it and
    then run as shared batches.  Each result equals its circuit alone."""
    heavy = W.fan_in_heavy(2, n=60, n_s=17, total=1500, tail=200)  # 43 x 2^17 terms
    light = [(n, instrs) for _, n, instrs in W.serving_stream(14, count=40)]
    srv = qx.Server(slots=1, hbm_budget=8 << 30)
    first = srv.submit(*heavy)
    tickets = [(srv.submit(n, instrs), n, instrs) for n, instrs in light]
    res, _ = srv.wait(first)
    assert res.nterms >= 43 * 2 ** 17
    for g in (0, 20, 59):
        assert abs(res.info(g)["sumsq"] - 1.0) < 1e-10
    res.free()
    for t, n, instrs in tickets:
        res, _ = srv.wait(t)
        _check_fp64(res, n, instrs, f"request {t}")
    st = srv.stats()
    assert st["alone"] == 1 and st["failed"] == 0
    assert st["batches"] < 1 + len(light) and st["mean_batch"] > 1.0
    srv.close()


def test_ledger_admission_and_requests_over_the_budget():
    """A budget that holds a few requests' reservations at a time: batches
    stay within it, a request whose bound alone exceeds it runs by itself
    (its exact size fits), and one that really needs more fails with
    QX_EBUDGET while the others complete unchanged."""
    light = [W.random_layers(s) for s in range(8)]  # n = 8, 10 T: bound 8 x 1024 terms
    big = W.fan_in_heavy(3, n=20, n_s=10, total=700, tail=100)  # 20 rotations: bound 20 x 2^20
    too_big = W.fan_in_heavy(4, n=30, n_s=14, total=900, tail=60)  # 16 x 2^14 x 2 terms exactly
    budget = 6 << 20
    srv = qx.Server(slots=2, hbm_budget=budget)
    tickets = [(srv.submit(*big), big)] + [(srv.submit(*c), c) for c in light]
    bad = srv.submit(*too_big)
    tickets += [(srv.submit(*c), c) for c in light[:3]]
    for t, (n, instrs) in tickets:
        res, _ = srv.wait(t)
        _check_fp64(res, n, instrs, f"request {t}")
    with pytest.raises(qx.QxError) as e:
        srv.wait(bad)
    assert e.value.name == "QX_EBUDGET"
    st = srv.stats()
    assert st["alone"] >= 2 and st["failed"] == 1
    assert st["peak_reserved"] <= budget
    srv.close()


def test_fp32_serving_matches_the_oracle():
    reqs = W.serving_stream(12, count=16)
    srv = qx.Server(slots=2, precision=32)
    tickets = [(srv.submit(n, instrs), n, instrs) for _, n, instrs in reqs]
    worst = 0.0
    for t, n, instrs in tickets:
        res, _ = srv.wait(t)
        want = _alone(n, instrs, precision=32)
        ref = O.propagate(n, instrs, mode="push", threads=CORES)
        for g in range(n):
            got = res.export_dict(g)
            assert got == want[g], (t, g)
            for s, w in O.as_dict(ref[g]).items():
                d = abs(got[s] - w)
                assert d <= 1e-5 * abs(w) + 1e-7, (t, g, s, got[s], w)
                if abs(w) > 1e-3:
                    worst = max(worst, d / abs(w))
    print(f"FP32 serving vs the FP64 oracle: max relative error {worst:.2e}")
    srv.close()


def test_pruning_in_batches():
    reqs = W.serving_stream(13, count=12, rot_range=(8, 14))
    eps = 1e-3
    srv = qx.Server(slots=1, eps=eps)
    tickets = [(srv.submit(n, instrs), n, instrs) for _, n, instrs in reqs]
    for t, n, instrs in tickets:
        res, _ = srv.wait(t)
        plan = qx.group_ops(qx.load_circuit(n, instrs), pushthrough=True)
        alone = qx.propagate(plan, eps=eps)
        for g in range(n):
            assert res.export_dict(g) == alone.export_dict(g)
            assert abs(res.info(g)["pruned_sumsq"] - alone.info(g)["pruned_sumsq"]) <= 1e-12
    srv.close()
