"""Exact density-matrix Pauli channel, n <= 6 (Sec. II: a density matrix holds
2^n x 2^n amplitudes). Used only to pin the Monte Carlo estimator: after each
gate rho <- U rho U^dagger, then at each of the gate's error locations
rho <- (1 - p_tot) rho + p_X X rho X + p_Z Z rho Z + p_Y Y rho Y.
The expected score of a linear criterion is its value on rho.
"""
import numpy as np

from .gates import PAULI, matrix_of


def embed(U, qubits, n):
    """Full 2^n x 2^n matrix of a gate acting on ``qubits`` (local index
    k = sum_j bit(q_j) 2^j); entries are U[k', k] where i and i' agree on all
    other qubits."""
    N = 1 << n
    F = np.zeros((N, N), dtype=np.complex128)
    mask = 0
    for q in qubits:
        mask |= 1 << q
    for i in range(N):
        k = sum(((i >> q) & 1) << j for j, q in enumerate(qubits))
        rest = i & ~mask
        for k2 in range(1 << len(qubits)):
            i2 = rest
            for j, q in enumerate(qubits):
                if (k2 >> j) & 1:
                    i2 |= 1 << q
            F[i2, i] = U[k2, k]
    return F


def evolve(circuit, p_x, p_z, p_y):
    n = circuit.n
    assert n <= 6, "density-matrix oracle is for n <= 6"
    N = 1 << n
    rho = np.zeros((N, N), dtype=np.complex128)
    rho[0, 0] = 1.0
    P = {q: {c: embed(PAULI[c], (q,), n) for c in (1, 2, 3)} for q in range(n)}
    p = {1: p_x, 2: p_z, 3: p_y}
    for gate in circuit.gates:
        U = embed(matrix_of(gate), gate.qubits, n)
        rho = U @ rho @ U.conj().T
        for q in gate.qubits:
            new = (1.0 - p_x - p_z - p_y) * rho
            for c in (1, 2, 3):
                new = new + p[c] * (P[q][c] @ rho @ P[q][c].conj().T)
            rho = new
    return rho


def expected_score(circuit, rho, psi_ref):
    crit = circuit.criterion
    if crit.kind == "fidelity":
        return float(np.real(np.vdot(psi_ref, rho @ psi_ref)))
    if crit.kind == "outcome":
        return float(np.real(rho[crit.target, crit.target]))
    if crit.kind == "binning":
        return float(sum(np.real(rho[k, k]) for k in crit.basis_set))
    raise ValueError("density-matrix expectation is defined for linear criteria only")
