"""Gradients of output weights on the GPU (qx_tape_*, qx_adjoint_dot) against
the oracle's parameter-shift gradient.

Functional: L = sum_k a_k c_{g_k}(P_k) over queried strings (mostly strings of
the output, a few absent ones), a ~ N(0, 1).  Workloads: the n = 8 random
layers with RX / RY / RZ in place of the T gates, and two layers of the n = 16
hardware-efficient ansatz.  Tolerance: every gradient entry
is a sum of products of weights of magnitude <= 1 taken in a different order
on the two sides; FP64 rounding then stays far below
1e-10 * max(1, sum |a_k|), the bound written in the tests (FP32: 1e-4 relative
to the largest entry plus 1e-5).
"""
import math

import numpy as np
import pytest

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


def _queries(n, instrs, gens, per_gen, seed, absent=2):
    ref = [O.as_dict(r) for r in O.propagate(n, instrs, mode="plan", gens=(gens[0], gens[-1] + 1),
                                             threads=4)]
    rng = np.random.default_rng(seed)
    qs = []
    for g in gens:
        d = ref[g - gens[0]]
        keys = sorted(d, key=lambda s: (-abs(d[s]), s))[: 4 * per_gen]
        for k in rng.choice(len(keys), size=min(per_gen, len(keys)), replace=False):
            qs.append((g, keys[int(k)]))
        for _ in range(absent):
            s = "".join("IXYZ"[int(v)] for v in rng.integers(0, 4, n))
            if s not in d:
                qs.append((g, s))
    return qs, rng.normal(size=len(qs))


def _tape(n, instrs, queries, gens, **kw):
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    lo = gens[0]
    return qx.Tape(plan, [g - lo for g, _ in queries], [p for _, p in queries],
                   gens=(gens[0], gens[-1] + 1), **kw)


def _tol(a):
    return 1e-10 * max(1.0, float(np.sum(np.abs(a))))


def test_from_terms_round_trip():
    n = 70
    rng = np.random.default_rng(4)
    strings = ["".join("IXYZ"[int(v)] for v in rng.integers(0, 4, n)) for _ in range(300)]
    gens = rng.integers(0, 3, 300)
    w = rng.normal(size=300)
    # repeats are summed
    strings += strings[:40]
    gens = np.concatenate([gens, gens[:40]])
    w = np.concatenate([w, w[:40]])
    r = qx.result_from_terms(n, 3, gens, strings, w)
    want = [{} for _ in range(3)]
    for g, s, v in zip(gens, strings, w):
        want[g][s] = want[g].get(s, 0.0) + v
    for g in range(3):
        got = r.export_dict(g)
        assert got.keys() == want[g].keys()
        for s, v in want[g].items():
            assert abs(got[s] - v) <= 1e-15 * abs(v)


@pytest.mark.parametrize("seed", [1, 2])
def test_propagate_result_equals_whole_circuit(seed):
    n, ins = W.rotation_layers(seed)
    cut = len(ins) // 2
    p1 = qx.group_ops(qx.load_circuit(n, ins[:cut]))
    p2 = qx.group_ops(qx.load_circuit(n, ins[cut:]))
    whole = qx.propagate(qx.group_ops(qx.load_circuit(n, ins)))
    mid = qx.propagate(p1)
    two = qx.propagate_result(p2, mid)
    for g in range(n):
        a, b = whole.export_dict(g), two.export_dict(g)
        assert a.keys() == b.keys()
        for s, v in a.items():
            assert abs(b[s] - v) <= 1e-12 * abs(v) + 1e-13
    # the start state is unchanged and can be propagated again
    again = qx.propagate_result(p2, mid)
    assert again.export_dict(3) == two.export_dict(3)


@pytest.mark.parametrize("n", [20, 100])
def test_adjoint_dot_matches_host_sum(n):
    rng = np.random.default_rng(n)

    def rand_state(G, N, seed):
        r = np.random.default_rng(seed)
        base = ["".join("IXYZ"[int(v)] for v in r.integers(0, 4, n)) for _ in range(N // 4)]
        strs, gs = [], []
        for _ in range(N):  # neighbours of a few base strings, so lookups hit
            s = list(base[int(r.integers(0, len(base)))])
            for _ in range(2):
                s[int(r.integers(0, n))] = "IXYZ"[int(r.integers(0, 4))]
            strs.append("".join(s))
            gs.append(int(r.integers(0, G)))
        return gs, strs, r.normal(size=N)

    gm, sm, wm = rand_state(3, 4000, 1)
    gl, sl, wl = rand_state(2, 3000, 1)  # same base strings: overlapping supports
    M = qx.result_from_terms(n, 3, gm, sm, wm)
    L = qx.result_from_terms(n, 2, gl, sl, wl)
    lam_gen = [1, -1, 0]
    nrot = 37
    qubits = rng.integers(0, n, nrot)
    dm = rng.normal(size=(nrot, 3, 3))
    dm[:, 0, 2] = 0.0  # some zero entries, as in real derivative tables
    got = qx.adjoint_dot(M, L, lam_gen, qubits, dm)
    mdicts = [M.export_dict(g) for g in range(3)]
    ldicts = [L.export_dict(g) for g in range(2)]
    want = np.zeros(nrot)
    scale = np.zeros(nrot)
    for g in range(3):
        h = lam_gen[g]
        if h < 0:
            continue
        for s, w in mdicts[g].items():
            for r in range(nrot):
                q = int(qubits[r])
                p = "XYZ".find(s[q])
                if p < 0:
                    continue
                for l in range(3):
                    v = ldicts[h].get(s[:q] + "XYZ"[l] + s[q + 1:], 0.0)
                    want[r] += w * dm[r, p, l] * v
                    scale[r] += abs(w * dm[r, p, l] * v)
    assert np.max(np.abs(want)) > 0.1  # lookups hit
    assert np.all(np.abs(got - want) <= 1e-12 * scale + 1e-15)
    # both iteration orders (M smaller / lam smaller) agree
    got2 = qx.adjoint_dot(L, M, [2, 0], qubits, np.transpose(dm, (0, 2, 1)))
    assert np.allclose(got2, got, rtol=0, atol=1e-12 * (1 + np.max(scale)))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tape_rotation_layers_n8_matches_oracle(seed):
    n, ins = W.rotation_layers(seed)
    gens = [0, 1, 2, 3]
    queries, a = _queries(n, ins, gens, 6, seed)
    tape = _tape(n, ins, queries, gens)
    want_vals = O.coeffs(n, ins, queries)
    assert np.allclose(tape.values, want_vals, atol=1e-13)
    grad = tape.backward(a)
    pos = O.rotation_positions(ins)
    want = O.grad_shift(n, ins, queries, a, workers=8)
    assert np.all(np.abs(grad[pos] - want) <= _tol(a)), np.max(np.abs(grad[pos] - want))
    others = np.setdiff1d(np.arange(len(ins)), pos)
    assert np.all(grad[others] == 0.0)
    assert np.max(np.abs(want)) > 1e-3


def test_tape_hea16_two_layers_matches_oracle():
    n, ins = W.hea(1, n=16, layers=2)
    gens = [0, 1]
    queries, a = _queries(n, ins, gens, 16, 7)
    tape = _tape(n, ins, queries, gens)
    info = tape.info()
    assert info["rotations"] == 64 and info["ops"] == 2 and info["held"] == 2
    grad = tape.backward(a)
    pos = O.rotation_positions(ins)
    rng = np.random.default_rng(3)
    sample = sorted(int(i) for i in rng.choice(pos, size=8, replace=False))
    want = O.grad_shift(n, ins, queries, a, positions=sample, workers=8)
    assert np.all(np.abs(grad[sample] - want) <= _tol(a))
    # every rotation: parameter shift with GPU forward runs
    plan_q = [g for g, _ in queries]
    strings = [p for _, p in queries]

    def L(instrs):
        r = qx.propagate(qx.group_ops(qx.load_circuit(n, instrs)), gens=(0, 2))
        return float(np.dot(a, r.coeff_batch(plan_q, strings)))

    for i in pos:
        g, q0, q1, th = ins[i]
        plus, minus = list(ins), list(ins)
        plus[i] = (g, q0, q1, th + math.pi / 2)
        minus[i] = (g, q0, q1, th - math.pi / 2)
        shift = (L(plus) - L(minus)) / 2
        assert abs(grad[i] - shift) <= _tol(a), (i, grad[i], shift)


def test_tape_hea_n8_four_layers_matches_oracle():
    """The four-layer ansatz at n = 8 (the n = 16 one exceeds the device);
    generators Z_0..Z_3 with output strings of each queried."""
    n, ins = W.hea(1, n=8, layers=4)
    gens = [0, 1, 2, 3]
    queries, a = _queries(n, ins, gens, 4, 21)
    tape = _tape(n, ins, queries, gens, ckpt_stride=0)
    assert tape.info()["ops"] == 4
    grad = tape.backward(a)
    pos = O.rotation_positions(ins)
    rng = np.random.default_rng(5)
    sample = sorted(int(i) for i in rng.choice(pos, size=16, replace=False))
    want = O.grad_shift(n, ins, queries, a, positions=sample, workers=8)
    assert np.all(np.abs(grad[sample] - want) <= _tol(a))
    assert np.max(np.abs(want)) > 1e-3


def test_tape_on_dag_plan_reports_circuit_order():
    """A tape on a qubit-wise plan (gates reordered) returns gradients in the
    circuit's own instruction order, equal to those of list-order grouping."""
    n, ins = W.rotation_layers(8, n_rot=12)
    gens = [0, 2]
    queries, a = _queries(n, ins, gens, 6, 8)
    qg = [g for g, _ in queries]
    qp = [p for _, p in queries]
    lst = qx.Tape(qx.group_ops(qx.load_circuit(n, ins)), qg, qp, gens=(0, 3)).backward(a)
    dplan = qx.group_ops(qx.load_circuit(n, ins), dag=True)
    assert not np.array_equal(dplan.order(), np.arange(len(ins)))
    dag = qx.Tape(dplan, qg, qp, gens=(0, 3)).backward(a)
    assert np.all(np.abs(dag - lst) <= _tol(a))
    pos = O.rotation_positions(ins)
    assert np.max(np.abs(dag[pos])) > 1e-3


def test_tape_qaoa_rzz_matches_oracle():
    """RZZ on graph edges and RX mixers: every angle, against the shift rule
    (exact for single Pauli rotations)."""
    n, ins = W.qaoa(3, n=10, layers=2)
    gens = [0, 1, 2, 3]
    queries, a = _queries(n, ins, gens, 6, 31)
    tape = _tape(n, ins, queries, gens)
    grad = tape.backward(a)
    pos = O.angle_positions(ins)
    assert any(ins[i][0] == "RZZ" for i in pos)
    want = O.grad_shift(n, ins, queries, a, positions=pos, workers=8)
    assert np.all(np.abs(grad[pos] - want) <= _tol(a)), np.max(np.abs(grad[pos] - want))
    assert np.max(np.abs(want)) > 1e-3


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_tape_two_qubit_rotations_match_oracle(seed):
    """RXX ... CP mixed with one-qubit rotations: single Pauli rotations by
    the shift rule, controlled rotations and CP by central differences of
    the oracle (h = 1e-5: error ~1e-10 relative)."""
    n = 5
    _, ins = W.random_small_2q(seed, n, 30, p2=0.5)
    gens = list(range(n))
    queries, a = _queries(n, ins, gens, 4, 40 + seed)
    grad = _tape(n, ins, queries, gens).backward(a)
    single = [i for i, g in enumerate(ins) if g[0] in O.ROTATIONS + O.PAULI_ROTATIONS_2Q]
    split = [i for i, g in enumerate(ins) if g[0] in O.SPLIT_ROTATIONS_2Q]
    if single:
        want = O.grad_shift(n, ins, queries, a, positions=single, workers=8)
        assert np.all(np.abs(grad[single] - want) <= _tol(a))
    if split:
        want = O.grad_fd(n, ins, queries, a, split, workers=8)
        assert np.all(np.abs(grad[split] - want) <= 1e3 * _tol(a))
    others = np.setdiff1d(np.arange(len(ins)), O.angle_positions(ins))
    assert np.all(grad[others] == 0.0)


@pytest.mark.parametrize("case", ["layers", "hea"])
def test_checkpoint_stride_gives_identical_gradients(case):
    if case == "layers":
        n, ins = W.rotation_layers(5, n_rot=14)
        gens = [0, 1, 2]
    else:
        n, ins = W.hea(2, n=12, layers=3)
        gens = [4]
    queries, a = _queries(n, ins, gens, 8, 11)
    ref = None
    for stride in (1, 2, 3, 0):
        tape = _tape(n, ins, queries, gens, ckpt_stride=stride)
        info = tape.info()
        s = stride or math.ceil(math.sqrt(info["ops"]))
        assert info["held"] == math.ceil(info["ops"] / s)
        g = tape.backward(a)
        if ref is None:
            ref = g
        # same states; only the storage order of recomputed terms (and so the
        # order of the sums) may differ
        assert np.allclose(g, ref, rtol=0, atol=1e-3 * _tol(a)), stride
        # recomputed states are released: the same number is held afterwards
        assert tape.info()["held"] == info["held"]


def test_backward_is_linear_and_repeatable():
    n, ins = W.rotation_layers(4)
    gens = [0, 5]
    queries, a1 = _queries(n, ins, gens, 8, 2)
    a2 = np.random.default_rng(8).normal(size=len(queries))
    tape = _tape(n, ins, queries, gens)
    g1 = tape.backward(a1)
    g2 = tape.backward(a2)
    g12 = tape.backward(a1 + a2)
    assert np.allclose(g12, g1 + g2, atol=_tol(a1) + _tol(a2))
    assert np.allclose(tape.backward(a1), g1, rtol=0, atol=1e-3 * _tol(a1))


def test_tape_without_rotations_or_queries():
    n, ins = W.random_layers(1)  # T gates only: no free angles
    tape = _tape(n, ins, [(0, "Z" + "I" * 7)], [0])
    assert np.all(tape.backward([1.0]) == 0.0)
    n, ins = W.rotation_layers(1)
    plan = qx.group_ops(qx.load_circuit(n, ins))
    empty = qx.Tape(plan, [], [])
    assert empty.values.size == 0
    assert np.all(empty.backward([]) == 0.0)


def test_fp32_tape_close_to_fp64():
    n, ins = W.rotation_layers(6, n_rot=12)
    gens = [0, 1, 2, 3]
    queries, a = _queries(n, ins, gens, 8, 6)
    g64 = _tape(n, ins, queries, gens).backward(a)
    g32 = _tape(n, ins, queries, gens, precision=32).backward(a)
    assert np.all(np.abs(g32 - g64) <= 1e-4 * np.max(np.abs(g64)) + 1e-5)


def test_autograd_function_matches_oracle():
    torch = pytest.importorskip("torch")
    from paper_2505_03307_gb300.autograd import RotationCircuit
    n, ins = W.rotation_layers(7)
    circ = RotationCircuit(n, ins)
    gens = [1, 2]
    queries, w = _queries(n, ins, gens, 5, 4)
    theta = circ.angles().cuda().requires_grad_(True)
    vals = circ.coeffs(theta, [g for g, _ in queries], [p for _, p in queries])
    wt = torch.tensor(w, dtype=torch.float64, device=vals.device)
    loss = (vals * wt).sum() + (vals ** 2).sum()
    loss.backward()
    v = vals.detach().cpu().numpy()
    a = w + 2 * v  # dloss / dvalues
    want = O.grad_shift(n, ins, queries, a, workers=8)
    got = theta.grad.cpu().numpy()
    assert np.all(np.abs(got - want) <= _tol(a))


def test_autograd_gradcheck_small():
    torch = pytest.importorskip("torch")
    from paper_2505_03307_gb300.autograd import RotationCircuit
    ins = [("RY", 0, -1, 0.3), ("CX", 0, 1, 0.0), ("RX", 1, -1, 1.1), ("H", 2, -1, 0.0),
           ("RZ", 2, -1, -0.7), ("CX", 1, 2, 0.0), ("RY", 2, -1, 2.0), ("RZ", 0, -1, 0.4)]
    circ = RotationCircuit(3, ins)
    theta = circ.angles().requires_grad_(True)
    f = lambda t: circ.coeffs(t, [0, 0, 1, 2], ["ZII", "XZI", "IZX", "ZZY"])  # noqa: E731
    assert torch.autograd.gradcheck(f, (theta,), eps=1e-6, atol=1e-6, nondet_tol=1e-12)
