"""Seeded synthetic circuit generators (inputs only).

This module produces gate lists and success-criterion descriptions for the
circuit families evaluated in the paper (Sec. V: arithmetic, Grover, QFT, QV)
and for the families used by the throughput workloads (brickwork, QAOA). It
holds none of the method's arithmetic: no state vectors, no gate matrices
except random unitaries that are themselves drawn inputs, no error sampling.
Both the FP64 oracle and the CUDA library consume these gate lists; each side
builds its own gate matrices from ``(name, qubits, params)``.

Conventions
-----------
* Qubit ``q`` is bit ``q`` of the amplitude index (little-endian).
* A gate is ``Gate(name, qubits, params, matrix)``. ``matrix`` is only set for
  ``U`` (2x2) and ``U2`` (4x4) gates and holds complex128 entries, row-major;
  for ``U2`` the local basis index is ``bit(q0) + 2*bit(q1)``.
* Two-qubit controlled gates list the control first: ``CX(c, t)``.
* Gate names: ID H X Y Z S SDG T TDG RX RY RZ P U (one qubit);
  CX CZ CP SWAP U2 (two qubits).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

ONE_QUBIT = ("ID", "H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U")
TWO_QUBIT = ("CX", "CZ", "CP", "SWAP", "U2")
GATE_NAMES = ONE_QUBIT + TWO_QUBIT


@dataclass(frozen=True)
class Gate:
    name: str
    qubits: tuple
    params: tuple = ()
    matrix: Optional[np.ndarray] = None

    @property
    def arity(self) -> int:
        return len(self.qubits)


@dataclass(frozen=True)
class Criterion:
    """Success criterion (Sec. II: fidelity, measurement probability, binning;
    argmax is the "correct result is the most likely outcome" variant).

    kind: "fidelity" | "outcome" | "binning" | "argmax"
    target: basis index for "outcome"/"argmax"
    basis_set: tuple of basis indices for "binning"
    threshold: a trajectory passes when its score >= threshold
    aggregate: "mean" (the paper's averaged P) or "pass" (pass fraction)
    """
    kind: str = "fidelity"
    target: int = 0
    basis_set: tuple = ()
    threshold: float = 0.5
    aggregate: str = "mean"


@dataclass
class Circuit:
    n: int
    gates: list
    family: str = ""
    criterion: Criterion = field(default_factory=Criterion)
    meta: dict = field(default_factory=dict)

    @property
    def G(self) -> int:
        return len(self.gates)

    @property
    def k(self) -> int:
        return sum(1 for g in self.gates if g.arity == 1)

    @property
    def m(self) -> int:
        return sum(1 for g in self.gates if g.arity == 2)

    @property
    def L(self) -> int:
        return self.k + 2 * self.m


def _g(name, *qubits, params=(), matrix=None):
    return Gate(name, tuple(int(q) for q in qubits), tuple(float(p) for p in params), matrix)


# --------------------------------------------------------------------------
# building blocks
# --------------------------------------------------------------------------

def toffoli_clifford_t(a: int, b: int, c: int) -> list:
    """Toffoli (controls a, b; target c) as the standard 15-gate Clifford+T
    network: 2 H, 6 CX, 7 T/TDG."""
    return [
        _g("H", c), _g("CX", b, c), _g("TDG", c), _g("CX", a, c), _g("T", c),
        _g("CX", b, c), _g("TDG", c), _g("CX", a, c), _g("T", b), _g("T", c),
        _g("H", c), _g("CX", a, b), _g("T", a), _g("TDG", b), _g("CX", a, b),
    ]


def _mcx_vchain_dirty(ctrl: Sequence[int], tgt: int, anc: Sequence[int]) -> list:
    """C^m X with m-2 borrowed (dirty) ancillas as 4(m-2) Toffolis
    (Barenco et al. 1995, Lemma 7.2). Ancillas are returned unchanged."""
    m = len(ctrl)
    assert m >= 3 and len(anc) >= m - 2
    a = list(anc[: m - 2])
    down = [(ctrl[i + 2], a[i], a[i + 1]) for i in range(m - 3 - 1, -1, -1)]
    up = [(ctrl[i + 2], a[i], a[i + 1]) for i in range(0, m - 3)]
    half = down + [(ctrl[0], ctrl[1], a[0])] + up
    seq = [(ctrl[m - 1], a[m - 3], tgt)] + half + [(ctrl[m - 1], a[m - 3], tgt)] + half
    out = []
    for (x, y, z) in seq:
        out += toffoli_clifford_t(x, y, z)
    return out


def mcx(ctrl: Sequence[int], tgt: int, free: Sequence[int]) -> list:
    """Multi-controlled X from {H, CX, T, TDG} using only borrowed qubits
    ``free`` (their state is restored). Barenco et al. 1995, Lemmas 7.2/7.3."""
    ctrl = list(ctrl)
    free = [q for q in free if q not in ctrl and q != tgt]
    m = len(ctrl)
    if m == 0:
        return [_g("X", tgt)]
    if m == 1:
        return [_g("CX", ctrl[0], tgt)]
    if m == 2:
        return toffoli_clifford_t(ctrl[0], ctrl[1], tgt)
    if len(free) >= m - 2:
        return _mcx_vchain_dirty(ctrl, tgt, free)
    if not free:
        raise ValueError("C^mX with m>=3 needs at least one borrowed qubit")
    # Lemma 7.3: split the controls in two halves around one borrowed qubit b.
    b = free[0]
    m1 = (m + 1) // 2
    A, B = ctrl[:m1], ctrl[m1:]
    rest_a = [q for q in free[1:]] + B + [tgt]
    rest_b = [q for q in free[1:]] + A
    p1 = mcx(A, b, rest_a)
    p2 = mcx(B + [b], tgt, rest_b)
    return p1 + p2 + p1 + p2


def mcz(qubits: Sequence[int], free: Sequence[int]) -> list:
    """Multi-controlled Z on ``qubits`` (phase -1 on |1...1>) = H . C^{m-1}X . H."""
    qubits = list(qubits)
    t = qubits[-1]
    if len(qubits) == 1:
        return [_g("Z", t)]
    if len(qubits) == 2:
        return [_g("CZ", qubits[0], qubits[1])]
    return [_g("H", t)] + mcx(qubits[:-1], t, free) + [_g("H", t)]


# --------------------------------------------------------------------------
# families
# --------------------------------------------------------------------------

def qft_gates(n: int, qubits: Optional[Sequence[int]] = None, swaps_as_cx: bool = True) -> list:
    """QFT on ``qubits`` (default 0..n-1) with native controlled-phase gates and
    the final bit-reversal swaps written as three CX each."""
    q = list(range(n)) if qubits is None else list(qubits)
    out = []
    for j in range(n - 1, -1, -1):
        out.append(_g("H", q[j]))
        for k in range(j - 1, -1, -1):
            out.append(_g("CP", q[k], q[j], params=(math.pi / (1 << (j - k)),)))
    for i in range(n // 2):
        a, b = q[i], q[n - 1 - i]
        if swaps_as_cx:
            out += [_g("CX", a, b), _g("CX", b, a), _g("CX", a, b)]
        else:
            out.append(_g("SWAP", a, b))
    return out


def basis_prep(n: int, x: int) -> list:
    return [_g("X", q) for q in range(n) if (x >> q) & 1]


def qft_basis(n: int, x: int, threshold: float = 0.5) -> Circuit:
    """QFT applied to basis state |x> (prepared by X gates counted as gates).
    Scored by fidelity with the ideal output state."""
    gates = basis_prep(n, x) + qft_gates(n)
    return Circuit(n, gates, "qft", Criterion("fidelity", threshold=threshold, aggregate="pass"),
                   {"x": x})


def grover(n_search: int, marked: int, iterations: Optional[int] = None) -> Circuit:
    """Grover search over ``n_search`` qubits plus one borrowed qubit (index
    n_search) that the multi-controlled Z decompositions use; the circuit uses
    only {H, X, CX, T, TDG}. Scored by argmax == marked (ancilla in |0>)."""
    ns = n_search
    n = ns + 1
    anc = ns
    theta = math.asin(2.0 ** (-ns / 2.0))
    k = int(math.floor(math.pi / (4.0 * theta))) if iterations is None else iterations
    search = list(range(ns))
    zmask = [q for q in search if not (marked >> q) & 1]
    gates = [_g("H", q) for q in search]
    for _ in range(k):
        gates += [_g("X", q) for q in zmask]
        gates += mcz(search, [anc])
        gates += [_g("X", q) for q in zmask]
        gates += [_g("H", q) for q in search]
        gates += [_g("X", q) for q in search]
        gates += mcz(search, [anc])
        gates += [_g("X", q) for q in search]
        gates += [_g("H", q) for q in search]
    return Circuit(n, gates, "grover", Criterion("argmax", target=marked, threshold=0.5, aggregate="pass"),
                   {"marked": marked, "iterations": k, "theta": theta})


def grover_seeded(n_total: int, seed: int) -> Circuit:
    rng = np.random.default_rng(seed)
    ns = n_total - 1
    marked = int(rng.integers(0, 1 << ns))
    return grover(ns, marked)


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2): a unit quaternion from four normals."""
    v = rng.standard_normal(4)
    a, b, c, d = v / np.linalg.norm(v)
    return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]], dtype=np.complex128)


def haar_u4(rng: np.random.Generator) -> np.ndarray:
    """Haar-random U(4): QR of a complex Gaussian matrix, with the phases of R's
    diagonal moved into Q (Mezzadri 2007)."""
    z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    qm, r = np.linalg.qr(z)
    return (qm * (np.diag(r) / np.abs(np.diag(r)))).astype(np.complex128)


def quantum_volume(n: int, seed: int) -> Circuit:
    """Quantum-volume model circuit (Cross et al. 2019): n layers; each layer
    pairs the qubits by a random permutation and applies a Haar U(4) to every
    pair (an odd qubit out idles). The criterion is binning on the heavy
    outputs, the basis states whose ideal probability exceeds the median; that
    set depends on the ideal output distribution, so whoever runs the circuit
    fills in ``criterion.basis_set`` from its error-free state."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(n):
        perm = rng.permutation(n)
        for k in range(n // 2):
            gates.append(_g("U2", int(perm[2 * k]), int(perm[2 * k + 1]), matrix=haar_u4(rng)))
    return Circuit(n, gates, "qv", Criterion("binning", threshold=2 / 3, aggregate="mean"), {"seed": seed})


def brickwork(n: int, depth: int, seed: int, threshold: float = 0.9) -> Circuit:
    """Per layer: Haar SU(2) on every qubit, then CZ on (0,1),(2,3),... in even
    layers and (1,2),(3,4),... in odd layers (open chain)."""
    rng = np.random.default_rng(seed)
    gates = []
    for d in range(depth):
        for q in range(n):
            gates.append(_g("U", q, matrix=haar_su2(rng)))
        start = 0 if d % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            gates.append(_g("CZ", a, a + 1))
    return Circuit(n, gates, "brickwork", Criterion("fidelity", threshold=threshold, aggregate="pass"),
                   {"depth": depth, "seed": seed})


def random_3regular(n: int, rng: np.random.Generator) -> list:
    """Random simple 3-regular graph on n (even) vertices: pairing model with
    rejection of loops and multi-edges."""
    assert n % 2 == 0 and n >= 4
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), 3)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for u, v in pairs:
            u, v = int(u), int(v)
            if u == v or (min(u, v), max(u, v)) in edges:
                ok = False
                break
            edges.add((min(u, v), max(u, v)))
        if ok:
            return sorted(edges)
    raise RuntimeError("no simple 3-regular graph found")


def qaoa_maxcut(n: int, seed: int, layers: int = 2, threshold: float = 0.5) -> Circuit:
    rng = np.random.default_rng(seed)
    edges = random_3regular(n, rng)
    gammas = rng.uniform(0.0, math.pi, layers)
    betas = rng.uniform(0.0, math.pi, layers)
    gates = [_g("H", q) for q in range(n)]
    for lay in range(layers):
        for (u, v) in edges:
            gates += [_g("CX", u, v), _g("RZ", v, params=(2.0 * gammas[lay],)), _g("CX", u, v)]
        gates += [_g("RX", q, params=(2.0 * betas[lay],)) for q in range(n)]
    return Circuit(n, gates, "qaoa", Criterion("fidelity", threshold=threshold, aggregate="pass"),
                   {"edges": edges, "gammas": gammas.tolist(), "betas": betas.tolist()})


def bernstein_vazirani(n: int, secret: int) -> Circuit:
    """Bernstein-Vazirani with CX gates (the paper's BV family): n - 1 data
    qubits and the ancilla n - 1 prepared in |->; the oracle is a CX from every
    data qubit whose secret bit is 1 onto the ancilla. Closing H gates leave
    |secret> on the data qubits and |1> on the ancilla: one correct outcome."""
    anc = n - 1
    gates = [_g("X", anc)] + [_g("H", q) for q in range(n)]
    gates += [_g("CX", q, anc) for q in range(n - 1) if (secret >> q) & 1]
    gates += [_g("H", q) for q in range(n)]
    target = (secret & ((1 << (n - 1)) - 1)) | (1 << anc)
    return Circuit(n, gates, "bv", Criterion("outcome", target=target, threshold=0.5, aggregate="mean"),
                   {"secret": secret})


def hidden_linear_function(n: int, seed: int, edge_prob: float = 0.5) -> Circuit:
    """Hidden linear function circuit (Bravyi, Gosset, Koenig 2018): H on every
    qubit, CZ on the edges of a random graph (the symmetric part of the
    quadratic form), S on a random subset (its diagonal), H on every qubit.
    Its outputs are spread uniformly over a subspace, so it is scored by
    fidelity (the paper's choice for circuits without a single correct outcome)."""
    rng = np.random.default_rng(seed)
    gates = [_g("H", q) for q in range(n)]
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < edge_prob:
                gates.append(_g("CZ", u, v))
    gates += [_g("S", q) for q in range(n) if rng.random() < 0.5]
    gates += [_g("H", q) for q in range(n)]
    return Circuit(n, gates, "hlf", Criterion("fidelity", threshold=0.5, aggregate="mean"), {"seed": seed})


def ryrz_ansatz(n: int, depth: int, seed: int) -> Circuit:
    """Hardware-efficient RY-RZ ansatz: a layer of RY and RZ rotations with
    random angles on every qubit, then a CX chain (q, q+1), repeated depth
    times, and a final rotation layer. Scored by fidelity."""
    rng = np.random.default_rng(seed)
    gates = []

    def rot():
        out = []
        for q in range(n):
            out.append(_g("RY", q, params=(rng.uniform(-math.pi, math.pi),)))
            out.append(_g("RZ", q, params=(rng.uniform(-math.pi, math.pi),)))
        return out

    for _ in range(depth):
        gates += rot()
        gates += [_g("CX", q, q + 1) for q in range(n - 1)]
    gates += rot()
    return Circuit(n, gates, "ryrz", Criterion("fidelity", threshold=0.5, aggregate="mean"), {"depth": depth})


def _pauli_exp(string: dict, theta: float) -> list:
    """exp(-i theta/2 P) for a Pauli string {qubit: "X"|"Y"|"Z"}: basis change to
    Z (H for X, RX(pi/2) for Y), a CX ladder that collects the parity on the
    last qubit, RZ(theta), the ladder reversed and the basis change undone."""
    qs = sorted(string)
    pre, post = [], []
    for q in qs:
        if string[q] == "X":
            pre.append(_g("H", q))
            post.append(_g("H", q))
        elif string[q] == "Y":
            pre.append(_g("RX", q, params=(math.pi / 2,)))
            post.append(_g("RX", q, params=(-math.pi / 2,)))
    ladder = [_g("CX", qs[i], qs[i + 1]) for i in range(len(qs) - 1)]
    return pre + ladder + [_g("RZ", qs[-1], params=(theta,))] + ladder[::-1] + post


def uccsd_ansatz(n: int, electrons: int, seed: int, max_doubles: int = 6) -> Circuit:
    """UCCSD-style ansatz in the Jordan-Wigner encoding: X gates load the
    Hartree-Fock state (the first `electrons` orbitals occupied), then every
    single excitation i -> a and up to max_doubles double excitations
    (i, j) -> (a, b) with random amplitudes, each as its Pauli-string
    exponentials (2 strings per single, 8 per double) with Z strings on the
    orbitals in between. Every excitation conserves the number of occupied
    orbitals. Scored by fidelity."""
    rng = np.random.default_rng(seed)
    occ, vir = list(range(electrons)), list(range(electrons, n))
    gates = [_g("X", q) for q in occ]

    def strings(ops):
        # ops: sorted list of (qubit, X|Y); the Jordan-Wigner Z string fills the gaps
        lo, hi = ops[0][0], ops[-1][0]
        st = {q: "Z" for q in range(lo, hi + 1)}
        for q, p in ops:
            st[q] = p
        return st

    for i in occ:
        for a in vir:
            t = rng.uniform(-0.5, 0.5)
            gates += _pauli_exp(strings([(i, "X"), (a, "Y")]), t)
            gates += _pauli_exp(strings([(i, "Y"), (a, "X")]), -t)
    doubles = [(i, j, a, b) for i in occ for j in occ if j > i for a in vir for b in vir if b > a]
    rng.shuffle(doubles)
    for (i, j, a, b) in doubles[:max_doubles]:
        t = rng.uniform(-0.5, 0.5)
        for k, combo in enumerate(("XXXY", "XXYX", "XYYY", "YXYY", "XYXX", "YXXX", "YYXY", "YYYX")):
            sign = 1.0 if k < 4 else -1.0
            ops = sorted(zip((i, j, a, b), combo))
            gates += _pauli_exp(strings(ops), sign * t / 4)
    return Circuit(n, gates, "uccsd", Criterion("fidelity", threshold=0.5, aggregate="mean"),
                   {"electrons": electrons})


def cuccaro_adder(bits: int, a: int, b: int) -> Circuit:
    """Ripple-carry adder (Cuccaro, Draper, Kutin, Moulton 2004) on 2*bits+2
    qubits: [c0, b0, a0, b1, a1, ..., z]. Operands are loaded by X gates;
    Toffolis are in Clifford+T. Scored by the probability of the outcome that
    holds b <- a+b (low bits), z <- carry, a unchanged."""
    if a >> bits or b >> bits:
        raise ValueError(f"operands must fit in {bits} bits")
    n = 2 * bits + 2
    c0 = 0
    bq = [1 + 2 * i for i in range(bits)]
    aq = [2 + 2 * i for i in range(bits)]
    z = n - 1
    gates = []
    gates += [_g("X", aq[i]) for i in range(bits) if (a >> i) & 1]
    gates += [_g("X", bq[i]) for i in range(bits) if (b >> i) & 1]

    def maj(x, y, w):
        return [_g("CX", w, y), _g("CX", w, x)] + toffoli_clifford_t(x, y, w)

    def uma(x, y, w):
        return toffoli_clifford_t(x, y, w) + [_g("CX", w, x), _g("CX", x, y)]

    gates += maj(c0, bq[0], aq[0])
    for i in range(1, bits):
        gates += maj(aq[i - 1], bq[i], aq[i])
    gates.append(_g("CX", aq[bits - 1], z))
    for i in range(bits - 1, 0, -1):
        gates += uma(aq[i - 1], bq[i], aq[i])
    gates += uma(c0, bq[0], aq[0])
    s = a + b
    out = 0
    for i in range(bits):
        if (a >> i) & 1:
            out |= 1 << aq[i]
        if (s >> i) & 1:
            out |= 1 << bq[i]
    if (s >> bits) & 1:
        out |= 1 << z
    return Circuit(n, gates, "adder", Criterion("outcome", target=out, threshold=0.5, aggregate="pass"),
                   {"a": a, "b": b, "bits": bits})


def ghz(n: int) -> Circuit:
    gates = [_g("H", 0)] + [_g("CX", q, q + 1) for q in range(n - 1)]
    return Circuit(n, gates, "ghz", Criterion("fidelity", threshold=0.5, aggregate="mean"))


def identity_chain(G: int) -> Circuit:
    """G identity gates on one qubit: under the uniform Pauli channel the
    fidelity with |0> is (1 + (1 - 4p/3)^G) / 2."""
    return Circuit(1, [_g("ID", 0) for _ in range(G)], "idchain",
                   Criterion("fidelity", threshold=0.5, aggregate="mean"))


def random_circuit(n: int, G: int, seed: int, two_qubit_frac: float = 0.4) -> Circuit:
    """Random mix of every gate kind, used by parity tests."""
    rng = np.random.default_rng(seed)
    one = ["ID", "H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P", "U"]
    two = ["CX", "CZ", "CP", "SWAP", "U2"]
    gates = []
    for _ in range(G):
        if n >= 2 and rng.random() < two_qubit_frac:
            name = two[int(rng.integers(len(two)))]
            a, b = rng.choice(n, 2, replace=False)
            if name == "CP":
                gates.append(_g(name, a, b, params=(rng.uniform(-math.pi, math.pi),)))
            elif name == "U2":
                gates.append(_g(name, a, b, matrix=haar_u4(rng)))
            else:
                gates.append(_g(name, a, b))
        else:
            name = one[int(rng.integers(len(one)))]
            q = int(rng.integers(n))
            if name in ("RX", "RY", "RZ", "P"):
                gates.append(_g(name, q, params=(rng.uniform(-math.pi, math.pi),)))
            elif name == "U":
                gates.append(_g(name, q, matrix=haar_su2(rng)))
            else:
                gates.append(_g(name, q))
    return Circuit(n, gates, "random", Criterion("fidelity", threshold=0.5, aggregate="mean"))


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------

def qft4_0101() -> Circuit:
    """4-qubit QFT on |0101> (X on qubits 0 and 2), CP native, swaps as 3 CX:
    G = 18 (k = 6, m = 12), L = 30. Fidelity >= 0.5."""
    return qft_basis(4, 0b0101)


def grover12(seed: int = 0) -> Circuit:
    """11 search qubits + 1 borrowed qubit, marked item from the seed."""
    return grover_seeded(12, seed)


def brickwork24(seed: int = 0) -> Circuit:
    return brickwork(24, 40, seed)


def mix_family(seed: int, count: int = 256, n_lo: int = 8, n_hi: int = 22,
               grover_max_n: int = 12) -> list:
    """Uneven batch: ``count`` circuits of n in [n_lo, n_hi] drawn from the
    seed, family uniform over {QFT on a random basis state, Grover, QAOA p=2 on
    a random 3-regular graph, ripple-carry adder}. Grover circuits are drawn
    with n <= grover_max_n (the optimal iteration count grows as 2^(n/2)),
    QAOA with even n, adders with n = 2*bits + 2."""
    rng = np.random.default_rng(seed)
    fams = ["qft", "grover", "qaoa", "adder"]
    out = []
    for i in range(count):
        fam = fams[int(rng.integers(4))]
        sub = int(rng.integers(1 << 31))
        if fam == "qft":
            n = int(rng.integers(n_lo, n_hi + 1))
            out.append(qft_basis(n, int(rng.integers(0, 1 << n))))
        elif fam == "grover":
            n = int(rng.integers(n_lo, min(n_hi, grover_max_n) + 1))
            out.append(grover_seeded(n, sub))
        elif fam == "qaoa":
            n = 2 * int(rng.integers((n_lo + 1) // 2, n_hi // 2 + 1))
            out.append(qaoa_maxcut(n, sub))
        else:
            bits = int(rng.integers(max(1, (n_lo - 2 + 1) // 2), (n_hi - 2) // 2 + 1))
            a = int(rng.integers(0, 1 << bits))
            b = int(rng.integers(0, 1 << bits))
            out.append(cuccaro_adder(bits, a, b))
    return out
