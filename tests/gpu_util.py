"""Shared helpers of the GPU tests: comparison of a libqx result with the oracle.

Tolerance (FP64 weights): |w_gpu - w_oracle| <= 1e-12 |w_oracle| + 1e-13.
Every one-qubit operator and every fused Clifford pass is an orthogonal map
of a generator's coefficient vector, which has unit norm (sum of w^2 = 1),
so rounding errors add in norm: after s rounding steps the error of any
weight is below s * 3 * 2^-53 ~ s * 3.3e-16.  The 1e-13 floor covers the
~300 merge and expansion steps of the largest parity cases; weights that are
not the result of cancellation also meet the 1e-12 relative bound.
String sets are compared exactly.
"""
import numpy as np

from oracle import oracle as O

REL = 1e-12
ABS = 1e-13


def compare_gen(got: dict, want: dict, label=""):
    assert got.keys() == want.keys(), (
        f"{label}: string sets differ: only gpu {sorted(set(got) - set(want))[:5]}, "
        f"only oracle {sorted(set(want) - set(got))[:5]}")
    worst = 0.0
    for s, w in want.items():
        d = abs(got[s] - w)
        assert d <= REL * abs(w) + ABS, (label, s, got[s], w)
        worst = max(worst, d)
    return worst


def compare_result(res, ref, offset=0, gens=None):
    worst = 0.0
    for k, r in enumerate(ref):
        g = offset + k if gens is None else gens[k]
        worst = max(worst, compare_gen(res.export_dict(g), O.as_dict(r), label=f"gen {g}"))
    return worst


def base4_order(strings):
    key = [tuple("IXYZ".index(c) for c in s) for s in strings]
    return key == sorted(key)
