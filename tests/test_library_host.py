"""CPU checks of libqx: exported symbols, validation, and the host planner.

The host planner's tables must be bit-equal to the oracle's (their zero
pattern decides which strings exist), and the fused Clifford passes must map
Pauli strings exactly as the oracle's gate-by-gate propagation does.
"""
import math
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

HEADER = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "include", "qx.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_exports_every_declared_symbol():
    text = open(HEADER).read()
    declared = set(re.findall(r"\b(qx_[a-z0-9_]+)\s*\(", text))
    assert declared == set(qx.EXPORTED)
    lib = qx.load_library()
    for name in declared:
        assert hasattr(lib, name), name


def test_validation():
    with pytest.raises(qx.QxError) as e:
        qx.load_circuit(4, [("H", 4, -1, 0.0)])
    assert e.value.name == "QX_EINVAL"
    with pytest.raises(qx.QxError) as e:
        qx.load_circuit(4, [("CX", 1, 1, 0.0)])
    assert e.value.name == "QX_EINVAL"
    with pytest.raises(qx.QxError) as e:
        qx.load_circuit(129, [])
    assert e.value.name == "QX_EUNSUPPORTED"
    with pytest.raises(qx.QxError) as e:
        qx.load_circuit(2, [("RZ", 0, -1, float("nan"))])
    assert e.value.name == "QX_EINVAL"
    qx.load_circuit(3, [])  # empty circuit is valid


@pytest.mark.parametrize("bad,msg", [(("H", 40, -1, 0.0), "wire out of range"),
                                     (("CX", 7, 7, 0.0), "bad second wire"),
                                     (("CZ", 3, -2, 0.0), "bad second wire"),
                                     (("RZ", 1, -1, float("inf")), "theta not finite")])
def test_validation_names_the_first_bad_instruction(bad, msg):
    """In a long valid circuit with two faults, the error names the first."""
    n, instrs = W.random_clifford(5, 20, 3000)
    instrs = list(instrs)
    instrs[1234] = bad
    instrs[2500] = ("H", 99, -1, 0.0)
    with pytest.raises(qx.QxError) as e:
        qx.load_circuit(n, instrs)
    assert e.value.name == "QX_EINVAL"
    assert f"instruction 1234: {msg}" in str(e.value)


def _circuits():
    yield W.random_layers(1)
    yield W.hea(2, n=8, layers=2)
    yield W.fan_in_heavy(1, n=12, n_s=4, total=200, tail=40)
    for seed in range(12):
        yield W.random_small(seed, 1 + seed % 6, 40, angles="quarter" if seed % 2 else "uniform")
    yield W.random_small(99, 70, 300, angles="quarter")


@pytest.mark.parametrize("idx", range(16))
def test_plan_matches_oracle_bit_for_bit(idx):
    n, instrs = list(_circuits())[idx]
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    ref = O.plan(n, instrs)
    assert plan.ops() == [k for k, _ in ref]
    K, Kp = plan.info()
    assert K == sum(k == "U" for k, _ in ref) and Kp == sum(k == "V" for k, _ in ref)
    assert abs(K - Kp) <= 1
    for op, (kind, lut) in enumerate(ref):
        if kind == "U":
            assert np.array_equal(plan.lut(op), lut), op


@pytest.mark.parametrize("idx", range(16))
def test_dag_plan_matches_oracle_bit_for_bit(idx):
    """Qubit-wise grouping: the library orders gates by dependency level, the
    oracle builds the same operators by rounds over per-wire queues; the
    operator kinds and every table must agree bit for bit."""
    n, instrs = list(_circuits())[idx]
    plan = qx.group_ops(qx.load_circuit(n, instrs), dag=True)
    ref = O.plan(n, instrs, dag=True)
    assert plan.ops() == [k for k, _ in ref]
    for op, (kind, lut) in enumerate(ref):
        if kind == "U":
            assert np.array_equal(plan.lut(op), lut), op
    K, Kp = plan.info()
    K0, Kp0 = qx.group_ops(qx.load_circuit(n, instrs)).info()
    assert K + Kp <= K0 + Kp0
    # the plan's order is a permutation that moves gates only past gates on
    # other wires: per wire, the sequence of gates touching it is unchanged
    order = plan.order()
    assert sorted(order.tolist()) == list(range(len(instrs)))
    for w in range(n):
        want = [i for i, g in enumerate(instrs) if w in (g[1], g[2])]
        got = [int(i) for i in order if w in (instrs[i][1], instrs[i][2])]
        assert got == want, w


def _check_passes(n, instrs, seed):
    """A Clifford-only circuit gives one fused pass equal to the whole circuit."""
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    assert plan.clifford_passes() == 1
    starts = W.random_paulis(seed, n, 6) + ["".join("Z" if q == j else "I" for q in range(n))
                                            for j in (0, n - 1)]
    ref = O.propagate(n, instrs, mode="gate", init=[(s, 1.0) for s in starts])
    for s, r in zip(starts, ref):
        (want_s, want_w), = O.as_dict(r).items()
        assert plan.clifford_apply(0, s) == (want_s, int(want_w))


@pytest.mark.parametrize("n,seed", [(6, 1), (40, 2), (70, 3), (100, 4)])
def test_pushthrough_plan_ends_with_the_clifford_part(n, seed):
    """A push-through plan has no operator chain and one Clifford pass: the
    circuit's Clifford gates, SWAP as three CX, in order."""
    _, instrs = W.random_small_2q(seed, n, 4 * n, angles="uniform")
    plan = qx.group_ops(qx.load_circuit(n, instrs), pushthrough=True)
    assert plan.info() == (0, 0)
    assert plan.clifford_passes() == 1
    cliff = [g for g in instrs if g[0] in ("H", "S", "SDG", "X", "Y", "Z", "SX", "SXDG", "CX", "CZ",
                                          "SWAP")]
    starts = W.random_paulis(seed, n, 6)
    ref = O.propagate(n, cliff, mode="gate", init=[(s, 1.0) for s in starts])
    for st, r in zip(starts, ref):
        (want_s, want_w), = O.as_dict(r).items()
        assert plan.clifford_apply(0, st) == (want_s, int(want_w))


@pytest.mark.parametrize("n,m", [(5, 3), (5, 400), (40, 10), (64, 900), (65, 30), (100, 3000),
                                 (128, 2000)])
def test_clifford_pass_matches_oracle(n, m):
    _, instrs = W.random_clifford(n * 7 + m, n, m)
    _check_passes(n, instrs, n + m)


def test_clifford_pass_forms():
    """Short passes use the gate list, long passes the chunk tables; both exact."""
    _check_passes(*W.ghz(60), 3)
    _check_passes(*W.graph_state(4, 90, 0.2), 4)


def test_propagate_without_gpu_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    plan = qx.group_ops(qx.load_circuit(2, [("H", 0, -1, 0.0)]))
    with pytest.raises(qx.QxError) as e:
        qx.propagate(plan)
    assert e.value.name in ("QX_EUNSUPPORTED", "QX_ECUDA")


def test_records_and_tuples_give_the_same_plan():
    """qx_instr records built from column arrays and the tuple list describe
    the same circuit: the same operators, tables and Clifford passes."""
    n, instrs = W.fan_in_heavy(1, n=20, n_s=8, total=500, tail=80)
    cols = list(zip(*instrs))
    rec = qx.instr_records(list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]))
    a = qx.group_ops(qx.load_circuit(n, instrs))
    b = qx.group_ops(qx.load_circuit_records(n, rec))
    assert a.info() == b.info() and a.ops() == b.ops()
    for op, kind in enumerate(a.ops()):
        if kind == "U":
            assert np.array_equal(a.lut(op), b.lut(op))


def test_pass_tables_of_a_many_pass_plan():
    """A plan with tens of thousands of Clifford operations over several
    passes (its pass tables are built on several threads): every pass maps
    strings as the oracle does through that pass's gates.  In list-order
    grouping, pass k holds the Clifford gates up to the end of the one-qubit
    run that holds the k-th RZ (the run's other wires commute with it)."""
    n, instrs = W.fan_in_deep(4, n=70, n_s=6, total=50_000)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    two = {"CX", "CZ", "SWAP", "RXX", "RYY", "RZZ", "CRX", "CRY", "CRZ", "CP"}
    bounds, i = [0], 0
    while i < len(instrs):  # maximal runs of one-qubit / two-qubit gates
        e = i
        while e < len(instrs) and (instrs[e][0] in two) == (instrs[i][0] in two):
            e += 1
        if any(g[0] == "RZ" for g in instrs[i:e]):
            bounds.append(e)
        i = e
    bounds.append(len(instrs))
    passes = [[g for g in instrs[b:e] if g[0] != "RZ"] for b, e in zip(bounds, bounds[1:])]
    assert plan.clifford_passes() == len(passes) == 7
    assert sum(len(p) for p in passes) > 40_000
    for k, gates in enumerate(passes):
        starts = W.random_paulis(100 + k, n, 3)
        ref = O.propagate(n, gates, mode="gate", init=[(s, 1.0) for s in starts])
        for s, r in zip(starts, ref):
            (want_s, want_w), = O.as_dict(r).items()
            assert plan.clifford_apply(k, s) == (want_s, int(want_w))


@pytest.mark.parametrize("dag", [False, True])
def test_plan_tables_outlive_the_circuit(dag):
    """A plan keeps its own instructions: after the circuit is freed, its
    operator tables (recomputed on request) still equal the oracle's."""
    import gc
    n, instrs = W.random_small(21, 6, 120, angles="uniform")
    c = qx.load_circuit(n, instrs)
    plan = qx.group_ops(c, dag=dag)
    del c
    gc.collect()
    ref = O.plan(n, instrs, dag=dag)
    assert plan.ops() == [k for k, _ in ref]
    for op, (kind, lut) in enumerate(ref):
        if kind == "U":
            assert np.array_equal(plan.lut(op), lut), op
