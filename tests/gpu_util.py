"""Shared helpers of the GPU tests: comparison of a libqx result with the oracle.

Tolerance (FP64 weights): |w_gpu - w_oracle| <= 1e-12 |w_oracle| + 1e-15,
with exactly equal string sets.  The absolute floor of 1e-15 is the floor of
the stated FP64 tolerance; weights are at most 1 in magnitude because every
generator has unit norm (sum of w^2 = 1).

Every compared weight feeds a per-test record of the worst absolute error and
the worst relative error over |w| > 1e-9; ``tests/conftest.py`` prints the
records at the end of the run, so the log shows how far inside the tolerance
each parity test is.

``rounding_floor(instrs)`` gives the one looser bound a test may ask for, per
weight, for weights that come out of cancellation: every one-qubit operator
and fused Clifford pass is an orthogonal map of the generator's unit-norm
coefficient vector, so the rounding errors of the two sides add in norm.  A
Clifford pass rounds nothing (it permutes strings and flips signs); each
application of a non-Clifford table or Pauli rotation rounds every weight it
writes once per product and once per term of its group sum (at most 3 terms of
magnitude <= 1 per group), which bounds that step's error vector by 6 u in
norm (u = 2^-53).  s such steps on both sides give at most 12 s u per weight.
"""
import os

from oracle import oracle as O

REL = 1e-12
ABS = 1e-15
U53 = 2.0 ** -53

#: per-test worst errors: nodeid -> [max |dw|, max |dw|/|w| over |w| > 1e-9, weights compared]
WORST = {}

_NON_CLIFFORD = {"T": 1, "TDG": 1, "RX": 1, "RY": 1, "RZ": 1, "RXX": 1, "RYY": 1, "RZZ": 1,
                 "CRX": 2, "CRY": 2, "CRZ": 2, "CP": 3, "U4": 15}


def rounding_floor(instrs):
    """Absolute per-weight error bound 12 s u from the number s of rounding
    steps of the circuit (non-Clifford one-qubit gates count one, the
    two-qubit rotations count their Pauli rotations), never below ABS."""
    s = sum(_NON_CLIFFORD.get(g[0], 0) for g in instrs)
    return max(ABS, 12.0 * s * U53)


def _record(d, w):
    key = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    rec = WORST.setdefault(key, [0.0, 0.0, 0])
    rec[0] = max(rec[0], d)
    if abs(w) > 1e-9:
        rec[1] = max(rec[1], d / abs(w))
    rec[2] += 1


def compare_gen(got: dict, want: dict, label="", floor=ABS):
    """Exact string sets, weights within REL |w| + floor; returns the worst |dw|."""
    assert got.keys() == want.keys(), (
        f"{label}: string sets differ: only gpu {sorted(set(got) - set(want))[:5]}, "
        f"only oracle {sorted(set(want) - set(got))[:5]}")
    worst = 0.0
    for s, w in want.items():
        d = abs(got[s] - w)
        _record(d, w)
        assert d <= REL * abs(w) + floor, (label, s, got[s], w, d)
        worst = max(worst, d)
    return worst


def compare_result(res, ref, offset=0, gens=None, floor=ABS):
    worst = 0.0
    for k, r in enumerate(ref):
        g = offset + k if gens is None else gens[k]
        worst = max(worst, compare_gen(res.export_dict(g), O.as_dict(r), label=f"gen {g}",
                                       floor=floor))
    return worst


def base4_order(strings):
    key = [tuple("IXYZ".index(c) for c in s) for s in strings]
    return key == sorted(key)


def close(got_w, want_w, floor=ABS):
    """One weight against its expected value (recorded like compare_gen)."""
    d = abs(got_w - want_w)
    _record(d, want_w)
    return d <= REL * abs(want_w) + floor
