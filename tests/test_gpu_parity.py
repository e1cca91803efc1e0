"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

String sets must be identical; weights agree within the FP64 tolerance of
``gpu_util``.  Sizes span several tiles and ragged tails of the kernels
(256-thread tiles, 1024-child expansion tiles, 2048-element scan tiles).
"""
import math

import numpy as np
import pytest

from gpu_util import base4_order, close, compare_gen, compare_result, rounding_floor
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


def run(n, instrs, **kw):
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    return plan, qx.propagate(plan, **kw)


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_random_layers_n8(seed):
    n, instrs = W.random_layers(seed)
    _, res = run(n, instrs)
    compare_result(res, O.propagate(n, instrs, mode="plan"))


@pytest.mark.parametrize("seed", range(30))
def test_random_small_all_gates(seed):
    n = 1 + seed % 7
    _, instrs = W.random_small(seed, n, 12 + 4 * n, angles="quarter" if seed % 3 == 0 else "uniform")
    _, res = run(n, instrs)
    compare_result(res, O.propagate(n, instrs, mode="plan"))


@pytest.mark.parametrize("n,layers,seed", [(8, 4, 1), (10, 3, 2), (6, 6, 3)])
def test_hea_merge_heavy(n, layers, seed):
    n, instrs = W.hea(seed, n=n, layers=layers)
    _, res = run(n, instrs)
    ref = O.propagate(n, instrs, mode="plan", threads=8)
    compare_result(res, ref)
    for g in range(n):
        assert abs(res.info(g)["sumsq"] - 1.0) < 1e-11


@pytest.mark.parametrize("n,layers,repeats,seed", [(6, 3, 100, 1), (8, 3, 10, 2), (10, 2, 1000, 3)])
def test_xyz_chain(n, layers, repeats, seed):
    """Reconstructed XYZ + chain circuit: every layer's repeated rotation
    blocks compose into one table per wire (Algorithm 1), so the device sees
    one fan-out step per layer whatever the repeat count."""
    _, instrs = W.xyz_chain(seed, n=n, layers=layers, repeats=repeats)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    assert plan.info() == (layers, layers)
    res = qx.propagate(plan)
    ref = O.propagate(n, instrs, mode="plan", threads=8)
    compare_result(res, ref)


def _dag_cases():
    for seed in range(1, 4):
        yield f"layers{seed}", W.random_layers(seed)
    for seed in range(12):
        yield f"small{seed}", W.random_small(seed, 1 + seed % 7, 60,
                                             angles="uniform" if seed % 2 else "quarter")
    yield "hea10", W.hea(2, n=10, layers=3)
    yield "brickwork50", W.brickwork(1)
    yield "xyz8", W.xyz_chain(4, n=8, layers=3, repeats=5)
    yield "pairs100", W.random_pairs(2, n_cliff=20000, n_rz=12)


@pytest.mark.parametrize("case", [c for c, _ in _dag_cases()])
def test_dag_grouping_matches_oracle(case):
    """Qubit-wise grouping (qx_group_ops_dag) against the oracle's own
    qubit-wise plan mode: exact string sets, weights within tolerance; and
    against list-order grouping up to strings of weight 0."""
    n, instrs = dict(_dag_cases())[case]
    plan = qx.group_ops(qx.load_circuit(n, instrs), dag=True)
    res = qx.propagate(plan)
    ref = O.propagate(n, instrs, mode="dag", threads=8)
    compare_result(res, ref)
    lst = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)))
    for g in range(0, n, max(1, n // 8)):
        a = {s: w for s, w in res.export_dict(g).items() if abs(w) > 1e-13}
        b = {s: w for s, w in lst.export_dict(g).items() if abs(w) > 1e-13}
        assert a.keys() == b.keys(), g
        # the two groupings round in different orders: the bound counts the
        # circuit's rounding steps
        for s, w in a.items():
            assert close(b[s], w, rounding_floor(instrs))


def test_fan_in_reduced_full_compare():
    """fan_in_heavy at n=20 with 8 fan-out qubits: 12 generators x 256 terms,
    one-shot expansion then 8 merge passes and a Clifford tail."""
    n, instrs = W.fan_in_heavy(5, n=20, n_s=8, total=600, tail=150)
    _, res = run(n, instrs)
    ref = O.propagate(n, instrs, mode="plan", threads=8)
    compare_result(res, ref)
    assert res.info(10)["nterms"] == 256
    st = res.stats()
    assert st["merge_passes"] == 8 and st["fan_steps"] == 2


def test_brickwork_n50():
    n, instrs = W.brickwork(1)
    _, res = run(n, instrs)
    compare_result(res, O.propagate(n, instrs, mode="plan", threads=8))


@pytest.mark.parametrize("n", [63, 64, 65, 100, 127, 128])
def test_word_boundaries(n):
    """W = 1 / 2 boundaries: random Clifford with rotations on the top qubits."""
    _, instrs = W.random_clifford(n, n, 6 * n)
    rng = np.random.default_rng(n)
    for q in (n - 1, n - 2, 63 % n, 0):
        instrs.insert(int(rng.integers(0, len(instrs))), ("RY", q, -1, 0.7))
        instrs.insert(int(rng.integers(0, len(instrs))), ("T", q, -1, 0.0))
    _, res = run(n, instrs)
    compare_result(res, O.propagate(n, instrs, mode="plan", threads=8))


def test_generator_range_and_export_order():
    n, instrs = W.random_layers(7)
    _, res = run(n, instrs, gens=(3, 6))
    assert res.ngen == 3
    compare_result(res, O.propagate(n, instrs, mode="plan", gens=(3, 6)))
    for g in range(3):
        strings, _ = res.export_strings(g)
        assert base4_order(strings)


def test_pruning_eps():
    """eps > 0: drop |w| < eps after every U_k; kept + pruned mass = 1.
    Strings whose |w| is within 1e-12 eps of eps are excluded (rounding ties)."""
    n, instrs = W.hea(4, n=8, layers=3)
    eps = 1e-3
    _, res = run(n, instrs, eps=eps)
    ref = O.propagate(n, instrs, mode="plan", eps=eps)
    for g, r in enumerate(ref):
        got = res.export_dict(g)
        want = O.as_dict(r)
        near = lambda d: {s for s, w in d.items() if abs(abs(w) - eps) <= 1e-12 * eps}
        tie = near(got) | near(want)
        compare_gen({s: w for s, w in got.items() if s not in tie},
                    {s: w for s, w in want.items() if s not in tie}, f"gen {g}")
        info = res.info(g)
        assert abs(info["sumsq"] + info["pruned_sumsq"] - 1.0) < 1e-11
        assert all(abs(w) >= eps for w in got.values())


def test_clifford_only_single_terms():
    n, instrs = W.random_clifford(3, 100, 5000)
    _, res = run(n, instrs)
    ref = O.propagate(n, instrs, mode="plan")
    compare_result(res, ref)
    for g in range(n):
        assert res.info(g)["nterms"] == 1


def test_empty_and_identity_circuits():
    _, res = run(5, [])
    for g in range(5):
        assert res.export_dict(g) == {"".join("Z" if q == g else "I" for q in range(5)): 1.0}
    _, res = run(3, [("H", 0, -1, 0.0), ("H", 0, -1, 0.0), ("RZ", 1, -1, 0.0)])
    assert res.export_dict(1) == {"IZI": 1.0}


def test_propagate_from_custom_generators():
    n, instrs = W.random_small(8, 5, 40)
    starts = W.random_paulis(3, n, 7)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate_from(plan, starts, weights=[0.5 + i for i in range(7)])
    ref = O.propagate(n, instrs, mode="plan", init=[(s, 0.5 + i) for i, s in enumerate(starts)])
    compare_result(res, ref)


def test_coeff_lookup():
    n, instrs = W.hea(6, n=6, layers=2)
    _, res = run(n, instrs)
    ref = O.propagate(n, instrs, mode="plan")
    for g in (0, 3, 5):
        d = O.as_dict(ref[g])
        present = list(d)[:: max(1, len(d) // 20)]
        absent = [s for s in W.random_paulis(g, n, 50) if s not in d][:10]
        vals = res.coeff_batch([g] * (len(present) + len(absent)), present + absent)
        for s, v in zip(present, vals):
            assert close(v, d[s])
        assert np.all(vals[len(present):] == 0.0)
        assert res.coeff(g, present[0]) == pytest.approx(d[present[0]], rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("seed", range(4))
def test_expval_matches_oracle(seed):
    n, instrs = W.random_small(200 + seed, 6, 50)
    obs = W.random_paulis(seed, n, 5)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    got = qx.expval(plan, obs)
    for q, v in zip(obs, got):
        assert abs(v - O.expval(n, instrs, q)) < 1e-12


def test_budget_and_cap_errors():
    n, instrs = W.fan_in_heavy(5, n=20, n_s=8, total=600, tail=0)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    with pytest.raises(qx.QxError) as e:
        qx.propagate(plan, max_terms=1000)
    assert e.value.name == "QX_ECAP"
    with pytest.raises(qx.QxError) as e:
        qx.propagate(plan, hbm_budget=10_000)
    assert e.value.name == "QX_EBUDGET"
    # the plan stays usable after an error
    res = qx.propagate(plan)
    assert res.info(12)["nterms"] == 256


def test_reserve_device_memory():
    """Growing the memory pool up front: a size the device holds succeeds, one
    it cannot hold fails with QX_ENOMEM and reserves nothing, and results do
    not change either way."""
    import torch
    qx.reserve_device_memory(1 << 30)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(qx.QxError) as e:
        qx.reserve_device_memory(1 << 50)
    assert e.value.name == "QX_ENOMEM"
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    n, instrs = W.random_layers(4)
    compare_result(qx.propagate(qx.group_ops(qx.load_circuit(n, instrs))),
                   O.propagate(n, instrs, mode="plan"))


def test_fan_in_heavy_full_size_sampled():
    """The n=50 heavy workload at full size (2,228,256 terms), in the bench's
    launch configuration: counts and norms of every generator, and the full
    string set of sampled generators against the oracle (gate mode equals plan
    mode here: every one-qubit table of the circuit comes from a single gate)."""
    n, instrs = W.fan_in_heavy(1)
    plan, res = run(n, instrs)
    assert res.nterms == 34 * 65536 + 16 * 2
    for g in range(n):
        info = res.info(g)
        assert info["nterms"] == (65536 if g >= 16 else 2)
        assert abs(info["sumsq"] - 1.0) < 1e-12
    for g in (3, 16, 49):
        ref = O.propagate(n, instrs, mode="gate", gens=(g, g + 1))
        compare_gen(res.export_dict(g), O.as_dict(ref[0]), f"gen {g}")
