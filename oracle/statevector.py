"""Plain state-vector simulation in complex128 (Sec. II; Sec. IV-B).

An n-qubit state is the vector of its 2^n complex amplitudes; qubit q is bit q
of the amplitude index. A gate updates the amplitudes by the textbook pair
(one-qubit) or quad (two-qubit) rule. A Pauli error is an "error gate"
appended right after the gate it follows (Sec. IV-B), acting on the amplitudes
as written in Eq. (2).
"""
from functools import lru_cache

import numpy as np

from .gates import matrix_of


def zero_state(n):
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def _base_indices(n, mask):
    """All indices i in [0, 2^n) whose bits in ``mask`` are zero."""
    if n >= 18:
        return _base_indices_uncached(n, mask)
    return _base_indices_cached(n, mask)


def _base_indices_uncached(n, mask):
    i = np.arange(1 << n, dtype=np.int64)
    return i[(i & mask) == 0]


_base_indices_cached = lru_cache(maxsize=512)(_base_indices_uncached)


def apply_1q(psi, n, q, U):
    """For every i with bit q = 0: (psi_i, psi_{i|2^q}) <- U (psi_i, psi_{i|2^q})."""
    i0 = _base_indices(n, 1 << q)
    i1 = i0 | (1 << q)
    a0 = psi[i0].copy()
    a1 = psi[i1].copy()
    psi[i0] = U[0, 0] * a0 + U[0, 1] * a1
    psi[i1] = U[1, 0] * a0 + U[1, 1] * a1


def apply_2q(psi, n, q0, q1, U):
    """4x4 analogue on (i, i|2^q0, i|2^q1, i|2^q0|2^q1); local index
    k = bit(q0) + 2*bit(q1)."""
    base = _base_indices(n, (1 << q0) | (1 << q1))
    idx = [base, base | (1 << q0), base | (1 << q1), base | (1 << q0) | (1 << q1)]
    a = [psi[ix].copy() for ix in idx]
    for k in range(4):
        psi[idx[k]] = U[k, 0] * a[0] + U[k, 1] * a[1] + U[k, 2] * a[2] + U[k, 3] * a[3]


def apply_gate(psi, n, gate):
    U = matrix_of(gate)
    if gate.arity == 1:
        apply_1q(psi, n, gate.qubits[0], U)
    else:
        apply_2q(psi, n, gate.qubits[0], gate.qubits[1], U)


def apply_pauli(psi, n, q, code):
    """Eq. (2) on qubit q with (a0, a1) = (psi_i, psi_{i|2^q}), bit q of i = 0:
    X: (a1, a0);  Z: (a0, -a1);  Y: (-i*a1, i*a0).
    Codes: 1 = X, 2 = Z, 3 = Y."""
    i0 = _base_indices(n, 1 << q)
    i1 = i0 | (1 << q)
    a0 = psi[i0].copy()
    a1 = psi[i1].copy()
    if code == 1:
        psi[i0], psi[i1] = a1, a0
    elif code == 2:
        psi[i1] = -a1
    elif code == 3:
        psi[i0], psi[i1] = -1j * a1, 1j * a0
    elif code != 0:
        raise ValueError(f"bad Pauli code {code}")


def location_table(circuit):
    """Error locations in circuit order: location l -> (gate index, qubit).
    One location per qubit of each gate, so L = k + 2m (Eq. (3))."""
    table = []
    for g, gate in enumerate(circuit.gates):
        for q in gate.qubits:
            table.append((g, q))
    return table


def simulate(circuit, events=(), psi0=None):
    """Run ``circuit`` from |0...0> (or ``psi0``), appending the Pauli error
    gates ``events`` = [(location, code), ...] after the gates they follow.
    Errors that follow the same gate are applied in location order."""
    n = circuit.n
    psi = zero_state(n) if psi0 is None else np.array(psi0, dtype=np.complex128)
    table = location_table(circuit)
    after = {}
    for (l, code) in events:
        g, q = table[l]
        after.setdefault(g, []).append((l, q, code))
    for g, gate in enumerate(circuit.gates):
        apply_gate(psi, n, gate)
        for (_, q, code) in sorted(after.get(g, ())):
            apply_pauli(psi, n, q, code)
    return psi
