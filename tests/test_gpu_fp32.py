"""FP32 weights with compensated arithmetic against the FP64 oracle and the FP64 path.

Strings, signs and phases are integers in both precisions, so string sets
must be identical (eps = 0).  Weights: |w32 - w64| <= 1e-5 |w64| + 1e-7, the
bound stated for the FP32 form.  Each child or merged weight carries about
one float rounding (2^-24) per operator, and rounding errors add in norm over
the unit-norm generator, so s operators give about s * 6e-8; the cases below
have at most ~150 operators acting on a term.  The largest error seen per
generator is printed.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W

pytestmark = pytest.mark.gpu
REL, ABS = 1e-5, 1e-7


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")


def _check(got, want, label):
    assert got.keys() == want.keys(), label
    worst = 0.0
    for s, w in want.items():
        d = abs(got[s] - w)
        assert d <= REL * abs(w) + ABS, (label, s, got[s], w)
        if abs(w) > 1e-3:
            worst = max(worst, d / abs(w))
    return worst


@pytest.mark.parametrize("case", ["layers_n8", "hea_8x4", "fan_in_n20", "small"])
def test_fp32_against_oracle(case):
    if case == "layers_n8":
        n, instrs = W.random_layers(2)
    elif case == "hea_8x4":
        n, instrs = W.hea(1, n=8, layers=4)
    elif case == "fan_in_n20":
        n, instrs = W.fan_in_heavy(5, n=20, n_s=8, total=600, tail=150)
    else:
        n, instrs = W.random_small(9, 6, 60)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan, precision=32)
    ref = O.propagate(n, instrs, mode="plan", threads=8)
    worst = [_check(res.export_dict(g), O.as_dict(r), f"{case} gen {g}") for g, r in enumerate(ref)]
    print(f"{case}: max relative FP32 error per generator {max(worst):.2e}")


def test_fp32_word_boundary_w2():
    n = 100
    _, instrs = W.random_clifford(7, n, 600)
    rng = np.random.default_rng(3)
    for q in (99, 70, 64, 63, 5):
        instrs.insert(int(rng.integers(0, len(instrs))), ("RX", q, -1, 0.37))
        instrs.insert(int(rng.integers(0, len(instrs))), ("T", q, -1, 0.0))
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    res = qx.propagate(plan, precision=32)
    ref = O.propagate(n, instrs, mode="plan", threads=8)
    for g, r in enumerate(ref):
        _check(res.export_dict(g), O.as_dict(r), f"gen {g}")


def test_fp32_vs_fp64_on_gpu_full_size():
    """The heavy n=50 workload in both precisions on the same GPU: identical
    string sets, FP32 weights within 1e-5 relative of the FP64 ones."""
    n, instrs = W.fan_in_heavy(1)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    r64 = qx.propagate(plan)
    r32 = qx.propagate(plan, precision=32)
    assert r32.nterms == r64.nterms == 2228256
    worst = 0.0
    for g in (0, 16, 33, 49):
        worst = max(worst, _check(r32.export_dict(g), r64.export_dict(g), f"gen {g}"))
    for g in range(n):
        assert abs(r32.info(g)["sumsq"] - 1.0) < 1e-5
    print(f"full size: max relative FP32 vs FP64 error {worst:.2e}")


def test_fp32_expval_and_coeff():
    n, instrs = W.random_small(210, 6, 50)
    plan = qx.group_ops(qx.load_circuit(n, instrs))
    obs = W.random_paulis(4, n, 5)
    got = qx.expval(plan, obs, precision=32)
    for q, v in zip(obs, got):
        assert abs(v - O.expval(n, instrs, q)) < 1e-5
    res = qx.propagate(plan, precision=32)
    d = O.as_dict(O.propagate(n, instrs, mode="plan")[2])
    keys = list(d)[:10]
    vals = res.coeff_batch([2] * len(keys), keys)
    for s, v in zip(keys, vals):
        assert abs(v - d[s]) <= REL * abs(d[s]) + ABS
