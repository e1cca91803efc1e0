"""CPU checks of the Python binding's marshalling (the only Python on the
path): Pauli strings to and from the x / z words of the C interface, and the
two ways of building qx_instr records."""
import ctypes

import numpy as np
import pytest

from paper_2505_03307_gb300 import qx
from paper_2505_03307_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 100, 127, 128])
def test_pauli_words_round_trip(n):
    rng = np.random.default_rng(n)
    for _ in range(20):
        p = "".join(rng.choice(list("IXYZ"), size=n))
        xw, zw = qx.pauli_to_words(p, n)
        assert xw.dtype == np.uint64 and xw.shape == (qx.words(n),) == zw.shape
        assert qx.words_to_pauli(xw, zw, n) == p


def test_pauli_words_letters_and_positions():
    """Letter q sits at bit q % 64 of word q // 64: X sets x, Z sets z, Y both."""
    n = 70
    p = ["I"] * n
    p[0], p[63], p[64], p[69] = "X", "Y", "Z", "Y"
    xw, zw = qx.pauli_to_words("".join(p), n)
    assert [int(v) for v in xw] == [1 | (1 << 63), 1 << 5]
    assert [int(v) for v in zw] == [1 << 63, 1 | (1 << 5)]
    # (x, z) integers give the same words
    x = (1 << 0) | (1 << 63) | (1 << 69)
    z = (1 << 63) | (1 << 64) | (1 << 69)
    xi, zi = qx.pauli_to_words((x, z), n)
    assert np.array_equal(xi, xw) and np.array_equal(zi, zw)
    with pytest.raises(ValueError):
        qx.pauli_to_words("XYZ", 4)


def test_paulis_to_arrays():
    x, z = qx.paulis_to_arrays(["XI" * 40, "IZ" * 40], 80)
    assert x.shape == (2, 2) and z.shape == (2, 2)
    assert qx.words_to_pauli(x[0], z[0], 80) == "XI" * 40
    assert qx.words_to_pauli(x[1], z[1], 80) == "IZ" * 40
    x, z = qx.paulis_to_arrays([], 10)  # at least one row for the C interface
    assert x.shape == (1, 1) and not x.any() and not z.any()


def test_instr_records_match_the_ctypes_array():
    """The column builder and the per-instruction ctypes array give the same
    24-byte records, gate codes included."""
    _, instrs = W.random_small(3, 6, 300)
    instrs = instrs + [("CP", 1, 4, 0.3), ("SWAP", 0, 5, 0.0), ("RZZ", 2, 3, -1.1)]
    cols = list(zip(*instrs))
    rec = qx.instr_records(list(cols[0]), list(cols[1]), list(cols[2]), list(cols[3]))
    arr = qx.instr_array(instrs)
    assert ctypes.sizeof(arr) == rec.nbytes == 24 * len(instrs)
    assert bytes(arr) == rec.tobytes()
    for (name, a, b, th), r in zip(instrs, rec):
        assert r["gate"] == qx.GATE_CODES[name]
        assert (r["q0"], r["q1"], r["theta"]) == (a, b, th)


def test_u4_array_layout():
    u = np.arange(16).reshape(4, 4) + 1j * (100 + np.arange(16).reshape(4, 4))
    a = qx.u4_array(u)
    assert a.shape == (32,)
    for r in range(4):
        for c in range(4):
            assert a[2 * (4 * r + c)] == u[r, c].real
            assert a[2 * (4 * r + c) + 1] == u[r, c].imag
