"""CPU checks that the seeded workloads have the shapes their recipes state
(the bench's configurations are quoted on them)."""
import math

import numpy as np

from paper_2505_03307_gb300 import workloads as W

CLIFFORD = {"H", "S", "CX"}


def test_fan_in_deep_n100_recipe():
    """n = 100, 100,000 gates: H on all, the CX fan-in onto the 20 fan-out
    qubits, 20 RZ (one per fan-out qubit, in order) between Clifford blocks
    on the other 80 qubits."""
    n, instrs = W.fan_in_deep(1)
    assert n == 100 and len(instrs) == 100_000
    assert instrs[:100] == [("H", q, -1, 0.0) for q in range(100)]
    fan = instrs[100:100 + 80 * 20]
    assert all(g[0] == "CX" and g[1] >= 20 and g[2] < 20 for g in fan)
    assert len({(g[1], g[2]) for g in fan}) == 1600
    rest = instrs[1700:]
    rz = [g for g in rest if g[0] == "RZ"]
    assert [g[1] for g in rz] == list(range(20))
    assert all(0.0 <= g[3] < 2 * math.pi for g in rz)
    for g in rest:
        if g[0] != "RZ":
            assert g[0] in CLIFFORD and g[1] >= 20 and (g[2] < 0 or g[2] >= 20)


def test_random_pairs_n100_recipe():
    n, instrs = W.random_pairs(1)
    assert n == 100 and len(instrs) == 100_020
    rz = [g for g in instrs if g[0] == "RZ"]
    assert len(rz) == 20
    cl = [g for g in instrs if g[0] != "RZ"]
    assert all(g[0] in CLIFFORD for g in cl)
    assert all(g[1] != g[2] for g in cl if g[0] == "CX")
    kinds = np.array([("H", "S", "CX").index(g[0]) for g in cl])
    assert np.all(np.abs(np.bincount(kinds) / len(cl) - 1 / 3) < 0.01)


def test_serving_stream_recipe():
    """n ~ U{10..60}, 200..5000 Clifford gates, 0..14 T / RZ, Poisson
    arrivals at the stated rate."""
    reqs = W.serving_stream(7, count=600, rate_hz=2000.0)
    ts = np.array([t for t, _, _ in reqs])
    assert np.all(np.diff(ts) > 0)
    gaps = np.diff(np.concatenate([[0.0], ts]))
    assert abs(gaps.mean() * 2000.0 - 1.0) < 0.08          # mean gap 1 / rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.08      # exponential: cv = 1
    ns, ms, ks = [], [], []
    for _, n, instrs in reqs:
        rot = [g for g in instrs if g[0] in ("T", "RZ")]
        cl = [g for g in instrs if g[0] not in ("T", "RZ")]
        assert all(g[0] in CLIFFORD for g in cl)
        assert all(0 <= g[1] < n and (g[2] < 0 or 0 <= g[2] < n) for g in instrs)
        ns.append(n)
        ms.append(len(cl))
        ks.append(len(rot))
    assert min(ns) == 10 and max(ns) == 60
    assert 200 <= min(ms) and max(ms) <= 5000
    assert min(ks) == 0 and max(ks) == 14
    assert abs(np.mean(ms) - 2600) < 100


def test_workloads_are_seeded():
    assert W.fan_in_heavy(3) == W.fan_in_heavy(3)
    assert W.fan_in_heavy(3) != W.fan_in_heavy(4)
    a = W.serving_stream(5, count=50)
    b = W.serving_stream(5, count=50)
    assert a == b
