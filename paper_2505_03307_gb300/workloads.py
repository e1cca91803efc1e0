"""Seeded synthetic circuits: the inputs shared by the oracle, the tests and the bench.

This module only draws gate lists.  It holds none of the propagation
arithmetic (no gate images, no tables, no Pauli algebra), so the CPU oracle
and the CUDA library can both consume its output without sharing any code
that computes a result.

A circuit is ``(n, instrs)`` where ``instrs`` is a list of
``(gate, q0, q1, theta)`` tuples: the instruction tuple ``{g, w, theta}`` of
Section III.A of the Qimax paper (gate name, wire(s), parameter; theta = 0
when the gate has none, q1 = -1 for single-qubit gates).

Gate names: H S SDG X Y Z SX SXDG T TDG RX RY RZ (one qubit), CX CZ (two).
"""
from __future__ import annotations

import math

import numpy as np

ONE_QUBIT = ("H", "S", "SDG", "X", "Y", "Z", "SX", "SXDG", "T", "TDG", "RX", "RY", "RZ")
TWO_QUBIT = ("CX", "CZ")
ROTATIONS = ("RX", "RY", "RZ")
ALL_GATES = ONE_QUBIT + TWO_QUBIT


def _g1(name, q, theta=0.0):
    return (name, int(q), -1, float(theta))


def _g2(name, c, t):
    return (name, int(c), int(t), 0.0)


def _insert_at_random(rng, instrs, extra):
    """Insert each gate of ``extra`` at a uniform position of the growing list."""
    out = list(instrs)
    for g in extra:
        pos = int(rng.integers(0, len(out) + 1))
        out.insert(pos, g)
    return out


def random_layers(seed: int, n: int = 8, layers: int = 20, n_t: int = 10):
    """n-qubit random Clifford layers plus T gates (the n=8, 20-layer, 10-T workload).

    Per layer the qubits are visited in a random order; each visited qubit
    draws H, S or CNOT uniformly; a CNOT takes the visited qubit as control and
    the next unvisited qubit as target (H when none is left).  Then ``n_t`` T
    gates are inserted at uniform positions on uniform qubits.
    """
    rng = np.random.default_rng(seed)
    instrs = []
    for _ in range(layers):
        order = list(rng.permutation(n))
        while order:
            q = order.pop(0)
            kind = int(rng.integers(0, 3))
            if kind == 0:
                instrs.append(_g1("H", q))
            elif kind == 1:
                instrs.append(_g1("S", q))
            elif order:
                t = order.pop(0)
                instrs.append(_g2("CX", q, t))
            else:
                instrs.append(_g1("H", q))
    ts = [_g1("T", int(rng.integers(0, n))) for _ in range(n_t)]
    return n, _insert_at_random(rng, instrs, ts)


def rotation_layers(seed: int, n: int = 8, layers: int = 20, n_rot: int = 10):
    """The random Clifford layers of ``random_layers`` with ``n_rot`` parametric
    rotations in place of the T gates: RX, RY or RZ (uniform) with angle
    U[0, 2 pi) on a uniform qubit, at uniform positions."""
    rng = np.random.default_rng(seed + 7919)
    _, base = random_layers(seed, n=n, layers=layers, n_t=0)
    rots = [_g1(("RX", "RY", "RZ")[int(rng.integers(0, 3))], int(rng.integers(0, n)),
                float(rng.uniform(0.0, 2.0 * math.pi))) for _ in range(n_rot)]
    return n, _insert_at_random(rng, base, rots)


def xyz_chain(seed: int, n: int = 12, layers: int = 2, repeats: int = 100):
    """The |XYZ + chain> benchmark circuit, reconstructed (its topology figure
    is not available): ``layers`` layers, each the XYZ block RX RY RZ (angles
    U[0, 2 pi)) on every qubit repeated ``repeats`` times, then a CX chain
    CX(q, q+1) for q = 0..n-2.  The gate count grows linearly with ``repeats``
    and n; with the paper's grouping each layer's rotations form one U_k."""
    rng = np.random.default_rng(seed)
    instrs = []
    for _ in range(layers):
        th = rng.uniform(0.0, 2.0 * math.pi, size=(repeats, n, 3))
        for r in range(repeats):
            for q in range(n):
                instrs.append(_g1("RX", q, float(th[r, q, 0])))
                instrs.append(_g1("RY", q, float(th[r, q, 1])))
                instrs.append(_g1("RZ", q, float(th[r, q, 2])))
        for q in range(n - 1):
            instrs.append(_g2("CX", q, q + 1))
    return n, instrs


def xyz_chain_columns(seed: int, n: int = 12, layers: int = 2, repeats: int = 100):
    """``xyz_chain`` as column arrays (names, q0, q1, theta), built without a
    Python loop per gate; the same gates in the same order."""
    rng = np.random.default_rng(seed)
    names, q0, q1, theta = [], [], [], []
    rot = np.array(["RX", "RY", "RZ"])
    for _ in range(layers):
        th = rng.uniform(0.0, 2.0 * math.pi, size=(repeats, n, 3))
        names.append(np.tile(rot, repeats * n))
        q0.append(np.tile(np.repeat(np.arange(n, dtype=np.int32), 3), repeats))
        q1.append(np.full(repeats * n * 3, -1, np.int32))
        theta.append(th.reshape(-1))
        names.append(np.full(n - 1, "CX"))
        q0.append(np.arange(n - 1, dtype=np.int32))
        q1.append(np.arange(1, n, dtype=np.int32))
        theta.append(np.zeros(n - 1))
    return n, (np.concatenate(names), np.concatenate(q0), np.concatenate(q1),
               np.concatenate(theta))


def brickwork(seed: int, n: int = 50, n_gates: int = 2000, n_t: int = 16, qubits=None):
    """Random Clifford brickwork plus T gates (the n=50, 2000-gate, 16-T workload).

    Layer L pairs (q, q+1) starting at offset L mod 2; each brick draws H, S or
    CNOT uniformly; a CNOT gets a random orientation, a one-qubit gate a random
    member of the pair.  Stops after ``n_gates`` Clifford gates, then inserts
    ``n_t`` T gates at uniform positions on uniform qubits.
    """
    rng = np.random.default_rng(seed)
    instrs = _brick_gates(rng, list(range(n)) if qubits is None else list(qubits), n_gates)
    ts = [_g1("T", int(rng.integers(0, n))) for _ in range(n_t)]
    return n, _insert_at_random(rng, instrs, ts)


def _brick_gates(rng, wires, count):
    """``count`` random H/S/CNOT bricks over the ordered wire list ``wires``."""
    out = []
    layer = 0
    while len(out) < count:
        for i in range(layer % 2, len(wires) - 1, 2):
            if len(out) >= count:
                break
            a, b = wires[i], wires[i + 1]
            kind = int(rng.integers(0, 3))
            if kind == 2:
                if rng.integers(0, 2):
                    a, b = b, a
                out.append(_g2("CX", a, b))
            else:
                q = a if rng.integers(0, 2) else b
                out.append(_g1("H" if kind == 0 else "S", q))
        layer += 1
    return out


def _random_pair_gates(rng, wires, count):
    """``count`` random H/S/CX gates, CX on a uniform ordered pair of distinct wires."""
    wires = list(wires)
    out = []
    for _ in range(count):
        kind = int(rng.integers(0, 3))
        if kind == 2:
            a, b = rng.choice(len(wires), size=2, replace=False)
            out.append(_g2("CX", wires[int(a)], wires[int(b)]))
        else:
            q = wires[int(rng.integers(0, len(wires)))]
            out.append(_g1("H" if kind == 0 else "S", q))
    return out


def fan_in_heavy(seed: int, n: int = 50, n_s: int = 16, total: int = 2000, tail: int = 600):
    """Heavy n=50 Clifford+T workload: 34 generators of 65,536 terms each.

    Built so that the literal brickwork workload's quoted size (up to ~65k terms
    per generator, millions in total) is actually reached:

    * H on every qubit, then CX(i -> q) for every i outside S = {0..n_s-1} and
      q in S: generator i becomes X on S plus a Pauli on i.
    * A random Clifford prefix on the qubits outside S (keeps X on all of S).
    * T on every q in S: each generator outside S fans out to 2^n_s terms.
    * CX(n-2 -> n-1): a two-qubit operator that closes the one-qubit operator.
    * RZ(theta_q) on every q in S, theta_q ~ U[0, 2 pi): every child now has two
      parents per qubit, so the index-based accumulation is exercised.
    * A random brickwork Clifford tail on all qubits (``tail`` gates).

    The prefix length makes the gate count ``total``.
    """
    rng = np.random.default_rng(seed)
    S = list(range(n_s))
    rest = list(range(n_s, n))
    head = [_g1("H", q) for q in range(n)]
    head += [_g2("CX", i, q) for i in rest for q in S]
    n_prefix = total - len(head) - 2 * n_s - 1 - tail
    if n_prefix < 0:
        raise ValueError("total too small for the fixed part of the workload")
    prefix = _brick_gates(rng, rest, n_prefix)
    ts = [_g1("T", q) for q in S]
    sep = [_g2("CX", n - 2, n - 1)]
    thetas = rng.uniform(0.0, 2.0 * math.pi, size=n_s)
    rz = [_g1("RZ", q, thetas[q]) for q in S]
    tail_g = _brick_gates(rng, list(range(n)), tail)
    return n, head + prefix + ts + sep + rz + tail_g


def hea(seed: int, n: int = 16, layers: int = 4):
    """Hardware-efficient ansatz: per layer RY(t) RZ(t) on each qubit, then a CX ring.

    theta = k pi / 4 with k ~ U{0..7} with probability 0.7, else U[0, 2 pi).
    """
    rng = np.random.default_rng(seed)
    instrs = []

    def draw():
        if rng.random() < 0.7:
            return int(rng.integers(0, 8)) * math.pi / 4.0
        return float(rng.uniform(0.0, 2.0 * math.pi))

    for _ in range(layers):
        for q in range(n):
            instrs.append(_g1("RY", q, draw()))
            instrs.append(_g1("RZ", q, draw()))
        for q in range(n):
            instrs.append(_g2("CX", q, (q + 1) % n))
    return n, instrs


def random_pairs(seed: int, n: int = 100, n_cliff: int = 100_000, n_rz: int = 20):
    """n=100 random-pair Clifford circuit with ``n_rz`` RZ(U[0,2pi)) at uniform positions."""
    rng = np.random.default_rng(seed)
    instrs = _random_pair_gates(rng, range(n), n_cliff)
    rz = [_g1("RZ", int(rng.integers(0, n)), float(rng.uniform(0.0, 2.0 * math.pi)))
          for _ in range(n_rz)]
    return n, _insert_at_random(rng, instrs, rz)


def fan_in_deep(seed: int, n: int = 100, n_s: int = 20, total: int = 100_000,
                final_mix: int = 0):
    """Heavy n=100 workload: 80 generators of 2^20 terms (about 84M terms in all).

    H on every qubit, CX(i -> q) for i outside S = {0..n_s-1} and q in S, then
    n_s rounds of [random Clifford block on the qubits outside S; RZ(theta_r)
    on qubit r], and a last Clifford block outside S.  The blocks never touch
    S, so every coefficient is a product of per-qubit cos/sin factors.
    ``final_mix`` > 0 appends that many random H/S/CX gates on all n qubits
    (drawn after everything else, so the circuit before them is unchanged):
    a last Clifford pass over every term that no expansion can absorb.
    """
    rng = np.random.default_rng(seed)
    S = list(range(n_s))
    rest = list(range(n_s, n))
    instrs = [_g1("H", q) for q in range(n)]
    instrs += [_g2("CX", i, q) for i in rest for q in S]
    n_cliff = total - len(instrs) - n_s
    per = n_cliff // (n_s + 1)
    sizes = [per] * (n_s + 1)
    sizes[-1] += n_cliff - per * (n_s + 1)
    thetas = rng.uniform(0.0, 2.0 * math.pi, size=n_s)
    for r in range(n_s):
        instrs += _random_pair_gates(rng, rest, sizes[r])
        instrs.append(_g1("RZ", r, thetas[r]))
    instrs += _random_pair_gates(rng, rest, sizes[-1])
    if final_mix:
        instrs += _random_pair_gates(rng, range(n), final_mix)
    return n, instrs


def ghz(n: int):
    """GHZ preparation: H(0) then a CX chain."""
    return n, [_g1("H", 0)] + [_g2("CX", q, q + 1) for q in range(n - 1)]


def graph_state(seed: int, n: int, p: float = 0.3):
    """Graph state on a seeded Erdos-Renyi graph: H on all, CZ on each edge."""
    rng = np.random.default_rng(seed)
    instrs = [_g1("H", q) for q in range(n)]
    for a in range(n):
        for b in range(a + 1, n):
            if rng.random() < p:
                instrs.append(_g2("CZ", a, b))
    return n, instrs


def random_clifford(seed: int, n: int, m: int):
    """Random circuit over every Clifford gate name of the gate set."""
    rng = np.random.default_rng(seed)
    names1 = ("H", "S", "SDG", "X", "Y", "Z", "SX", "SXDG")
    out = []
    for _ in range(m):
        if n >= 2 and rng.random() < 0.4:
            a, b = rng.choice(n, size=2, replace=False)
            out.append(_g2(TWO_QUBIT[int(rng.integers(0, 2))], a, b))
        else:
            out.append(_g1(names1[int(rng.integers(0, len(names1)))], int(rng.integers(0, n))))
    return n, out


def random_small(seed: int, n: int, m: int, p2: float = 0.3, angles: str = "uniform"):
    """Random circuit over the whole gate set, for brute-force checks at small n.

    ``angles``: "uniform" draws rotation angles from U[0, 2 pi); "quarter" draws
    multiples of pi/4 (exercises the exact-Clifford rounding of the tables).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(m):
        if n >= 2 and rng.random() < p2:
            a, b = rng.choice(n, size=2, replace=False)
            out.append(_g2(TWO_QUBIT[int(rng.integers(0, 2))], a, b))
        else:
            g = ONE_QUBIT[int(rng.integers(0, len(ONE_QUBIT)))]
            th = 0.0
            if g in ROTATIONS:
                if angles == "quarter":
                    th = int(rng.integers(0, 8)) * math.pi / 4.0
                else:
                    th = float(rng.uniform(0.0, 2.0 * math.pi))
            out.append(_g1(g, int(rng.integers(0, n)), th))
    return n, out


TWO_QUBIT_ROT = ("RXX", "RYY", "RZZ", "CRX", "CRY", "CRZ", "CP")


def random_small_2q(seed: int, n: int, m: int, p2: float = 0.35, angles: str = "uniform"):
    """``random_small`` with the two-qubit gates beyond CX / CZ mixed in: half
    of the two-qubit draws are SWAP or a two-qubit rotation (RXX ... CP)."""
    rng = np.random.default_rng(seed + 104729)
    _, base = random_small(seed, n, m, p2=p2, angles=angles)
    out = []
    for g in base:
        if g[0] in TWO_QUBIT and rng.random() < 0.5:
            name = ("SWAP",) + TWO_QUBIT_ROT
            k = int(rng.integers(0, len(name)))
            if angles == "quarter":
                th = int(rng.integers(0, 8)) * math.pi / 4.0
            else:
                th = float(rng.uniform(0.0, 2.0 * math.pi))
            out.append((name[k], g[1], g[2], th if k > 0 else 0.0))
        else:
            out.append(g)
    # at least one of the new gates whenever there is a two-qubit gate
    if not any(g[0] in ("SWAP",) + TWO_QUBIT_ROT for g in out):
        for i, g in enumerate(out):
            if g[0] in TWO_QUBIT:
                out[i] = ("RZZ", g[1], g[2], float(rng.uniform(0.0, 2.0 * math.pi)))
                break
    return n, out


def qaoa(seed: int, n: int = 16, layers: int = 2, degree: int = 3):
    """QAOA-style circuit on a random ``degree``-regular graph: H on every
    qubit, then per layer RZZ(gamma) on every edge and RX(beta) on every
    qubit (gamma, beta ~ U[0, pi))."""
    rng = np.random.default_rng(seed)
    # random regular graph by repeated perfect matchings on a shuffled ring
    edges = set()
    while len(edges) < n * degree // 2:
        perm = rng.permutation(n)
        for k in range(0, n - 1, 2):
            a, b = int(perm[k]), int(perm[k + 1])
            if a != b and len(edges) < n * degree // 2:
                edges.add((min(a, b), max(a, b)))
    edges = sorted(edges)
    instrs = [_g1("H", q) for q in range(n)]
    for _ in range(layers):
        gamma, beta = float(rng.uniform(0, math.pi)), float(rng.uniform(0, math.pi))
        for a, b in edges:
            instrs.append(("RZZ", a, b, gamma))
        for q in range(n):
            instrs.append(_g1("RX", q, beta))
    return n, instrs


def haar_u4(rng):
    """A Haar-random 4 x 4 unitary (QR of a complex Gaussian matrix with the
    phases of R's diagonal moved into Q)."""
    z = (rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))


def special_u4():
    """Named two-qubit unitaries whose KAK coordinates are degenerate (local
    gates, CX, CZ, SWAP, iSWAP, sqrt(SWAP), controlled phases) as 4 x 4
    matrices (basis index 2 b(q0) + b(q1))."""
    h = np.array([[1, 1], [1, -1]]) / math.sqrt(2.0)
    s = np.diag([1, 1j])
    out = {
        "identity": np.eye(4, dtype=complex),
        "local": np.kron(h, s @ h),
        "cx": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex),
        "cz": np.diag([1, 1, 1, -1]).astype(complex),
        "swap": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex),
        "iswap": np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=complex),
        "cp": np.diag([1, 1, 1, np.exp(0.7j)]),
    }
    a = (1 + 1j) / 2
    out["sqrt_swap"] = np.array([[1, 0, 0, 0], [0, a, a.conjugate(), 0],
                                 [0, a.conjugate(), a, 0], [0, 0, 0, 1]], dtype=complex)
    out["phase"] = np.exp(0.3j) * out["iswap"] @ np.kron(s, h)
    return out


def random_small_u4(seed: int, n: int, m: int, p_u4: float = 0.25, p_cx: float = 0.15):
    """Random circuit of one-qubit gates, CX and general two-qubit unitaries
    ("U4", q0, q1, matrix): Haar matrices, and at times a named one."""
    rng = np.random.default_rng(seed)
    names1 = ("H", "S", "SX", "T", "RX", "RY", "RZ")
    spec = list(special_u4().values())
    out = []
    for _ in range(m):
        r = rng.random()
        if n >= 2 and r < p_u4:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            u = spec[int(rng.integers(0, len(spec)))] if rng.random() < 0.2 else haar_u4(rng)
            out.append(("U4", a, b, u))
        elif n >= 2 and r < p_u4 + p_cx:
            a, b = (int(v) for v in rng.choice(n, size=2, replace=False))
            out.append(_g2("CX", a, b))
        else:
            g = names1[int(rng.integers(0, len(names1)))]
            th = float(rng.uniform(0, 2 * math.pi)) if g.startswith("R") else 0.0
            out.append(_g1(g, int(rng.integers(0, n)), th))
    return n, out


def random_paulis(seed: int, n: int, k: int, min_weight: int = 1):
    """``k`` seeded random Pauli strings ("IXYZ" letters, character i = qubit i)."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < k:
        s = "".join("IXYZ"[int(v)] for v in rng.integers(0, 4, size=n))
        if sum(c != "I" for c in s) >= min_weight:
            out.append(s)
    return out


def serving_stream(seed: int, count: int = 10_000, n_range=(10, 60), gate_range=(200, 5000),
                   rot_range=(0, 14), rate_hz: float = 2000.0):
    """Seeded request stream: (arrival time s, n, instrs) with Poisson arrivals.

    n ~ U{10..60}, Clifford gate count ~ U{200..5000} (random pairs), T/RZ count
    ~ U{0..14} at uniform positions (T or RZ(U[0,2pi)) with equal probability).
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        m = int(rng.integers(gate_range[0], gate_range[1] + 1))
        k = int(rng.integers(rot_range[0], rot_range[1] + 1))
        instrs = _random_pair_gates(rng, range(n), m)
        rots = []
        for _ in range(k):
            q = int(rng.integers(0, n))
            if rng.integers(0, 2):
                rots.append(_g1("T", q))
            else:
                rots.append(_g1("RZ", q, float(rng.uniform(0.0, 2.0 * math.pi))))
        out.append((t, n, _insert_at_random(rng, instrs, rots)))
    return out


#: Named workloads used by the tests and the bench.
WORKLOADS = {
    "random_layers_n8": lambda seed=1: random_layers(seed),
    "brickwork_n50": lambda seed=1: brickwork(seed),
    "fan_in_heavy_n50": lambda seed=1: fan_in_heavy(seed),
    "hea_n16": lambda seed=1: hea(seed),
    "random_pairs_n100": lambda seed=1: random_pairs(seed),
    "fan_in_deep_n100": lambda seed=1: fan_in_deep(seed),
}
