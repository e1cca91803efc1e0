"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: the paper's printed example or
rule list, the textbook definition c_j(P) = Tr(P U Z_j U^dagger) / 2^n built
from dense matrices, the Aaronson-Gottesman tableau rules, closed forms, or
invariants of the mathematics (Parseval, commutation, unitarity).
"""
import math

import numpy as np
import pytest

import refs
from oracle import oracle as O
from paper_2505_03307_gb300 import workloads as W

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")

ONE_Q = ["H", "S", "SDG", "X", "Y", "Z", "SX", "SXDG", "T", "TDG", "RX", "RY", "RZ"]


def base4_index(s):
    v = 0
    for ch in s:
        v = 4 * v + "IXYZ".index(ch)
    return v


# --- gate tables and the CX rule list ---------------------------------------

@pytest.mark.parametrize("name", ONE_Q)
@pytest.mark.parametrize("theta", [0.0, 0.3, 1.0, math.pi / 2, 2.5, -0.7])
def test_gate_table_matches_conjugation(name, theta):
    """Sec. II.C: g P g^dagger; table rows must equal Tr(c g p g^dagger)/2."""
    got = O.gate_table(name, theta)
    want = refs.conj_table(name, theta)
    assert np.allclose(got, want, atol=1e-15, rtol=0)


@pytest.mark.parametrize("name", ONE_Q)
def test_gate_table_orthogonal(name):
    """Conjugation by a unitary is a rotation of (X, Y, Z): R R^T = I."""
    r = O.gate_table(name, 1.234)
    assert np.allclose(r @ r.T, np.eye(3), atol=1e-15)


def test_cx_rules_match_paper_list():
    """Sec. III.C rule list (golden file) for all 16 letter pairs."""
    rows = [ln.split() for ln in open(f"{GOLDEN}/cx_rules.txt") if ln.strip() and ln[0] != "#"]
    assert len(rows) == 16
    assert sorted(r[0] for r in rows) == sorted(a + b for a in "IXYZ" for b in "IXYZ")
    for frm, to, sign in rows:
        assert O.cx(frm[0], frm[1]) == (to, int(sign))


def test_cx_rules_match_dense_conjugation():
    """The same 16 images from the 4x4 CX matrix (control = qubit 0)."""
    U = refs.dense_unitary(2, [("CX", 0, 1, 0.0)])
    for a in "IXYZ":
        for b in "IXYZ":
            M = U @ refs.pauli_matrix(a + b) @ U.conj().T
            pair, sign = O.cx(a, b)
            assert abs(refs.coeff(M, pair) - sign) < 1e-14


def test_t_powers_and_products():
    """T^2 = S and T^8 = 1 and H^2 = 1 as composed plan tables (Algorithm 1)."""
    lut = O.plan(1, [("T", 0, -1, 0.0)] * 2)[0][1][0]
    assert np.array_equal(lut, O.gate_table("S"))
    lut8 = O.plan(1, [("T", 0, -1, 0.0)] * 8)[0][1][0]
    assert np.array_equal(lut8, np.eye(3))
    lut_h = O.plan(1, [("H", 0, -1, 0.0)] * 2)[0][1][0]
    assert np.array_equal(lut_h, np.eye(3))
    lut_rz = O.plan(1, [("RZ", 0, -1, math.pi / 2)])[0][1][0]
    assert np.array_equal(lut_rz, O.gate_table("S"))


# --- Example 1: flatten and the base-4 encoding ------------------------------

def test_example1_flatten():
    parents, terms = [], []
    for ln in open(f"{GOLDEN}/example1_flatten.txt"):
        f = ln.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "parent":
            v = [float(t) for t in f[1:]]
            parents.append((v[0], [v[1:5], v[5:9]]))
        elif f[0] == "term":
            terms.append((f[1], float(f[2]), int(f[3])))
    res = O.flatten([p[0] for p in parents], [p[1] for p in parents])
    got = O.as_dict(res)
    assert got == {s: w for s, w, _ in terms}
    for s, _, idx in terms:
        assert base4_index(s) == idx
    # the oracle's output order is the base-4 index order
    assert [base4_index(s) for s in res["strings"]] == sorted(base4_index(s) for s in res["strings"])


# --- dense brute force -------------------------------------------------------

def _check_dense(n, instrs, mode, tol=1e-12):
    U = refs.dense_unitary(n, instrs)
    res = O.propagate(n, instrs, mode=mode)
    for j, gen in enumerate(res):
        assert np.all(gen["im"] == 0.0)
        M = refs.generator_matrix(U, n, j)
        total = 0.0
        for s, w in zip(gen["strings"], gen["re"]):
            c = refs.coeff(M, s)
            assert abs(c.imag) < 1e-12
            assert abs(w - c.real) <= tol * max(1.0, abs(c.real)), (j, s, w, c)
            total += c.real ** 2
        # Parseval: sum over all 4^n strings of c^2 is Tr(M^2)/2^n = 1, so the
        # produced strings carry all of it and every absent string is 0.
        assert abs(total - 1.0) < 1e-11
    return res


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("mode", ["gate", "plan"])
def test_dense_random_small(seed, mode):
    n = 1 + seed % 5
    _, instrs = W.random_small(seed, n, 6 + 2 * n, angles="uniform" if seed % 2 else "quarter")
    _check_dense(n, instrs, mode)


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("mode", ["gate", "plan"])
def test_dense_random_layers_n8(seed, mode):
    n, instrs = W.random_layers(seed)
    _check_dense(n, instrs, mode)


def test_dense_hea_small():
    n, instrs = W.hea(3, n=6, layers=2)
    _check_dense(n, instrs, "plan")


@pytest.mark.parametrize("mode", ["gate", "plan"])
def test_dense_xyz_chain_small(mode):
    """The reconstructed XYZ + chain circuit: 2 layers of 5 repeated RX RY RZ
    blocks and a CX chain on 5 qubits (each layer's 75 rotations are one U_k
    in plan mode)."""
    n, instrs = W.xyz_chain(2, n=5, layers=2, repeats=5)
    res = _check_dense(n, instrs, mode)
    assert max(len(g["strings"]) for g in res) > 100


@pytest.mark.parametrize("seed", range(12))
def test_dense_dag_grouping(seed):
    """Plan mode with qubit-wise grouping against dense brute force."""
    n = 2 + seed % 5
    _, instrs = W.random_small(seed, n, 10 + 3 * n, angles="uniform" if seed % 2 else "quarter")
    _check_dense(n, instrs, "dag")


def test_dag_grouping_composes_across_other_wires():
    """T on wire 0, a CNOT on wires 1-2, T on wire 0: list-order grouping
    makes two fan-outs (a zero-weight X stays behind), the qubit-wise one
    composes T T = S (no fan-out at all)."""
    ins = [("H", 0, -1, 0.0), ("T", 0, -1, 0.0), ("CX", 1, 2, 0.0), ("T", 0, -1, 0.0)]
    kinds = [k for k, _ in O.plan(3, ins, dag=True)]
    assert kinds == ["U", "V"]
    lut = O.plan(3, ins, dag=True)[0][1]
    assert np.array_equal(lut[0], O.plan(1, [("H", 0, -1, 0.0), ("S", 0, -1, 0.0)])[0][1][0])
    d = O.as_dict(O.propagate(3, ins, mode="dag", gens=(0, 1))[0])
    p = O.as_dict(O.propagate(3, ins, mode="plan", gens=(0, 1))[0])
    assert d == {"YII": 1.0}
    assert p.keys() == {"XII", "YII"} and abs(p["XII"]) < 1e-15


@pytest.mark.parametrize("seed", range(16))
@pytest.mark.parametrize("mode", ["gate", "plan", "dag", "push"])
def test_dense_two_qubit_rotations_and_push(seed, mode):
    """SWAP and the two-qubit rotations (16 x 16 tables from 4 x 4 unitaries
    in the oracle; Kronecker products of textbook matrices here) in every
    oracle mode, including push-through."""
    n = 2 + seed % 5
    _, instrs = W.random_small_2q(seed, n, 12 + 3 * n,
                                  angles="quarter" if seed % 3 == 0 else "uniform")
    assert any(g[0] not in ("CX", "CZ") and g[2] >= 0 for g in instrs) or n < 2
    _check_dense(n, instrs, mode)


def test_dense_qaoa_small():
    n, instrs = W.qaoa(1, n=6, layers=2)
    for mode in ("gate", "plan", "push"):
        _check_dense(n, instrs, mode)


def test_gate_and_plan_agree_semantically():
    """Gate and plan mode may differ only in keys of weight ~0 (T;T = S)."""
    for seed in range(10):
        n, instrs = W.random_small(seed, 4, 30, angles="quarter")
        a = O.propagate(n, instrs, mode="gate")
        b = O.propagate(n, instrs, mode="plan")
        for ga, gb in zip(a, b):
            da = {s: w for s, w in O.as_dict(ga).items() if abs(w) > 1e-13}
            db = {s: w for s, w in O.as_dict(gb).items() if abs(w) > 1e-13}
            assert da.keys() == db.keys()
            for s in da:
                assert abs(da[s] - db[s]) < 1e-12


def test_plan_grouping_and_luts():
    """Sec. III.A: maximal runs, |K - K'| <= 1, first instruction decides the order."""
    instrs = [("H", 0, -1, 0.0), ("T", 0, -1, 0.0), ("RZ", 1, -1, 0.4), ("CX", 0, 1, 0.0),
              ("CZ", 1, 2, 0.0), ("S", 2, -1, 0.0), ("CX", 2, 0, 0.0)]
    p = O.plan(3, instrs)
    assert [k for k, _ in p] == ["U", "V", "U", "V"]
    lut0 = p[0][1]
    # U_{0,0} = H then T, composed in list order (Algorithm 1)
    want = O.gate_table("H") @ O.gate_table("T")
    assert np.allclose(lut0[0], want, atol=1e-15)
    assert np.allclose(lut0[1], O.gate_table("RZ", 0.4), atol=0)
    assert np.array_equal(lut0[2], np.eye(3))
    p2 = O.plan(2, [("CX", 0, 1, 0.0), ("H", 0, -1, 0.0)])
    assert [k for k, _ in p2] == ["V", "U"]


# --- CHP: Clifford circuits keep single +-1 strings ---------------------------

def _check_chp(n, instrs, gens=None):
    res = O.propagate(n, instrs, mode="plan", gens=gens)
    lo = 0 if gens is None else gens[0]
    for k, gen in enumerate(res):
        j = lo + k
        row = refs.chp_row(n, j)
        for g, a, b, _ in instrs:
            refs.chp_apply(row, g, a, b)
        s, sign = refs.chp_string(row)
        assert gen["strings"] == [s]
        assert gen["re"][0] == sign


def test_chp_ghz_and_graph():
    _check_chp(*W.ghz(40))
    _check_chp(*W.graph_state(5, 30))


@pytest.mark.parametrize("seed", range(4))
def test_chp_random_clifford(seed):
    n, instrs = W.random_clifford(seed, 24, 400)
    _check_chp(n, instrs)


def test_chp_random_clifford_n100():
    n, instrs = W.random_clifford(9, 100, 2000)
    _check_chp(n, instrs, gens=(0, 100))


def test_chp_cross_checks_dense():
    """The CHP helper itself against dense matrices (n = 4)."""
    n, instrs = W.random_clifford(3, 4, 60)
    U = refs.dense_unitary(n, instrs)
    for j in range(n):
        row = refs.chp_row(n, j)
        for g, a, b, _ in instrs:
            refs.chp_apply(row, g, a, b)
        s, sign = refs.chp_string(row)
        assert abs(refs.coeff(refs.generator_matrix(U, n, j), s) - sign) < 1e-12


# --- invariants --------------------------------------------------------------

def test_invariants_sumsq_and_commutation():
    n, instrs = W.random_small(11, 6, 60)
    res = O.propagate(n, instrs, mode="plan")
    sums = []
    for gen in res:
        d = O.as_dict(gen)
        sums.append(d)
        assert abs(sum(w * w for w in d.values()) - 1.0) < 1e-12
    # generators of one state commute pairwise: check via dense products
    mats = [sum(w * refs.pauli_matrix(s) for s, w in d.items()) for d in sums]
    for a in range(n):
        for b in range(a + 1, n):
            assert np.allclose(mats[a] @ mats[b], mats[b] @ mats[a], atol=1e-10)


def test_round_trip_identity():
    """U followed by U^dagger returns Z_j with weight 1, everything else ~0."""
    n, instrs = W.random_small(5, 5, 40)
    inv = []
    swap = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T", "SX": "SXDG", "SXDG": "SX"}
    for g, a, b, th in reversed(instrs):
        inv.append((swap.get(g, g), a, b, -th))
    res = O.propagate(n, instrs + inv, mode="plan")
    for j, gen in enumerate(res):
        d = O.as_dict(gen)
        z = "".join("Z" if q == j else "I" for q in range(n))
        assert abs(d[z] - 1.0) < 1e-12
        assert all(abs(w) < 1e-12 for s, w in d.items() if s != z)


def test_pruning_bookkeeping():
    """eps > 0: kept mass plus pruned mass stays 1 (the operators are orthogonal)."""
    n, instrs = W.random_small(21, 5, 80)
    for eps in (1e-3, 1e-2, 0.1):
        res = O.propagate(n, instrs, mode="plan", eps=eps)
        for gen in res:
            kept = float(np.sum(gen["re"] ** 2))
            assert abs(kept + gen["pruned_sumsq"] - 1.0) < 1e-12
            assert np.all(np.abs(gen["re"]) >= eps)


def test_rank_bound():
    """n' <= 4^n - 1 non-identity strings (Sec. II.C)."""
    n, instrs = W.hea(2, n=3, layers=3)
    for gen in O.propagate(n, instrs, mode="plan"):
        assert len(gen["strings"]) <= 4 ** n - 1


# --- expectation values ---------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_expval_matches_state_vector(seed):
    n = 2 + seed % 4
    _, instrs = W.random_small(seed + 100, n, 25)
    for q in W.random_paulis(seed, n, 4):
        assert abs(O.expval(n, instrs, q) - refs.dense_expval(n, instrs, q)) < 1e-12


# --- closed forms of the fan-in workloads --------------------------------------

def _fan_in_closed_form(n, instrs, S):
    """Per generator outside S: sign * N_i on the rest, times per-qubit factors on S.

    Valid while no gate after the CX fan-in touches S except the one-qubit
    rotations on S; the rest of the string comes from the Clifford-only run.
    """
    cliff = [g for g in instrs if not (g[0] in ("T", "RZ") and g[1] in S)]
    base = O.propagate(n, cliff, mode="gate")
    # per-qubit image of X under the rotations on S in order
    fac = {}
    for q in S:
        v = np.array([1.0, 0.0])  # (X, Y) weights
        for g, a, _, th in instrs:
            if a == q and g in ("T", "RZ"):
                c, s = (math.sqrt(0.5), math.sqrt(0.5)) if g == "T" else (math.cos(th), math.sin(th))
                v = np.array([c * v[0] - s * v[1], s * v[0] + c * v[1]])
        fac[q] = v
    return base, fac


def test_fan_in_closed_form_small():
    """fan_in_heavy with 4 fan-out qubits and no tail: 2^4 terms per generator
    whose weights are products of per-qubit (c - s)/sqrt2, (s + c)/sqrt2 factors."""
    n, instrs = W.fan_in_heavy(3, n=10, n_s=4, total=120, tail=0)
    S = list(range(4))
    res = O.propagate(n, instrs, mode="plan")
    base, fac = _fan_in_closed_form(n, instrs, S)
    for i in range(4, n):
        d = O.as_dict(res[i])
        assert len(d) == 16
        (b_s, b_w), = O.as_dict(base[i]).items()
        for s, w in d.items():
            assert s[4:] == b_s[4:]
            want = b_w
            for q in S:
                assert s[q] in "XY"
                want *= fac[q][0 if s[q] == "X" else 1]
            assert abs(w - want) < 1e-12
    # one generator inside S: two terms
    assert len(res[0]["strings"]) == 2


# --- general two-qubit unitaries (U4) ----------------------------------------

@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("mode", ["gate", "plan", "push"])
def test_dense_general_two_qubit_unitaries(seed, mode):
    """U4 gates (Haar-random and named 4 x 4 matrices) in every oracle mode
    against the dense brute force (Kronecker-indexed 4 x 4 blocks applied to
    the state's rows in refs)."""
    n = 2 + seed % 4
    _, instrs = W.random_small_u4(seed, n, 8 + 3 * n)
    assert any(g[0] == "U4" for g in instrs)
    _check_dense(n, instrs, mode)


def test_u4_of_named_gates_equals_the_gate():
    """A U4 holding the matrix of CX (or of RZZ) gives the same generators
    as the gate itself."""
    import cmath
    n = 3
    cx = W.special_u4()["cx"]
    th = 0.37
    rzz = np.diag([cmath.exp(-0.5j * th), cmath.exp(0.5j * th), cmath.exp(0.5j * th),
                   cmath.exp(-0.5j * th)])
    base = [("H", 0, -1, 0.0), ("RY", 1, -1, 0.4), ("T", 2, -1, 0.0)]
    for named, u in ((("CX", 0, 2, 0.0), cx), (("RZZ", 1, 2, th), rzz)):
        a = O.propagate(n, base + [named], mode="gate")
        b = O.propagate(n, base + [("U4", named[1], named[2], u)], mode="gate")
        for ga, gb in zip(a, b):
            da = {s: w for s, w in O.as_dict(ga).items() if abs(w) > 1e-14}
            db = {s: w for s, w in O.as_dict(gb).items() if abs(w) > 1e-14}
            assert da.keys() == db.keys()
            for s, w in da.items():
                assert abs(db[s] - w) < 1e-13


def test_fan_in_deep_final_mix_is_a_clifford_suffix():
    """fan_in_deep(final_mix=k) is the plain circuit followed by k H/S/CX
    gates on all qubits, so each generator keeps its number of terms and the
    multiset of |weights| (a Clifford block maps strings one to one and can
    only flip signs), and every fan-out wire is touched by the suffix."""
    base_n, base = W.fan_in_deep(5, n=12, n_s=4, total=200)
    n, mixed = W.fan_in_deep(5, n=12, n_s=4, total=200, final_mix=60)
    assert n == base_n and mixed[:len(base)] == base and len(mixed) == len(base) + 60
    tail = mixed[len(base):]
    assert all(g[0] in ("H", "S", "CX") for g in tail)
    assert any(g[1] < 4 or (g[0] == "CX" and g[2] < 4) for g in tail)
    a = O.propagate(n, base, mode="plan")
    b = O.propagate(n, mixed, mode="plan")
    for ga, gb in zip(a, b):
        wa = sorted(abs(w) for w in O.as_dict(ga).values())
        wb = sorted(abs(w) for w in O.as_dict(gb).values())
        assert len(wa) == len(wb)
        assert np.allclose(wa, wb, rtol=0, atol=1e-13)
