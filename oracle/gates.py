"""Gate matrices from their textbook definitions (complex128).

Two-qubit matrices act on the local index k = bit(q0) + 2*bit(q1) where
(q0, q1) are the gate's qubits in the order written; CX/CP list the control
first, so CX maps |c=1,t=0> (k=1) <-> |c=1,t=1> (k=3).
"""
import cmath
import math

import numpy as np

_S2 = 1.0 / math.sqrt(2.0)


def one_qubit(name, params=(), matrix=None):
    if name == "ID":
        return np.eye(2, dtype=np.complex128)
    if name == "H":
        return np.array([[_S2, _S2], [_S2, -_S2]], dtype=np.complex128)
    if name == "X":
        return np.array([[0, 1], [1, 0]], dtype=np.complex128)
    if name == "Y":
        return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
    if name == "Z":
        return np.array([[1, 0], [0, -1]], dtype=np.complex128)
    if name == "S":
        return np.array([[1, 0], [0, 1j]], dtype=np.complex128)
    if name == "SDG":
        return np.array([[1, 0], [0, -1j]], dtype=np.complex128)
    if name == "T":
        return np.array([[1, 0], [0, cmath.exp(1j * math.pi / 4)]], dtype=np.complex128)
    if name == "TDG":
        return np.array([[1, 0], [0, cmath.exp(-1j * math.pi / 4)]], dtype=np.complex128)
    if name == "RX":
        t = params[0] / 2
        return np.array([[math.cos(t), -1j * math.sin(t)], [-1j * math.sin(t), math.cos(t)]],
                        dtype=np.complex128)
    if name == "RY":
        t = params[0] / 2
        return np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]], dtype=np.complex128)
    if name == "RZ":
        t = params[0] / 2
        return np.array([[cmath.exp(-1j * t), 0], [0, cmath.exp(1j * t)]], dtype=np.complex128)
    if name == "P":
        return np.array([[1, 0], [0, cmath.exp(1j * params[0])]], dtype=np.complex128)
    if name == "U":
        return np.asarray(matrix, dtype=np.complex128).reshape(2, 2)
    raise ValueError(f"unknown one-qubit gate {name}")


def two_qubit(name, params=(), matrix=None):
    if name == "CX":
        m = np.eye(4, dtype=np.complex128)
        m[[1, 3]] = m[[3, 1]]
        return m
    if name == "CZ":
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if name == "CP":
        return np.diag([1, 1, 1, cmath.exp(1j * params[0])]).astype(np.complex128)
    if name == "SWAP":
        m = np.eye(4, dtype=np.complex128)
        m[[1, 2]] = m[[2, 1]]
        return m
    if name == "U2":
        return np.asarray(matrix, dtype=np.complex128).reshape(4, 4)
    raise ValueError(f"unknown two-qubit gate {name}")


def matrix_of(gate):
    if gate.arity == 1:
        return one_qubit(gate.name, gate.params, gate.matrix)
    return two_qubit(gate.name, gate.params, gate.matrix)


# Pauli matrices in the order used by the error codes: 1 = X, 2 = Z, 3 = Y.
PAULI = {
    1: np.array([[0, 1], [1, 0]], dtype=np.complex128),
    2: np.array([[1, 0], [0, -1]], dtype=np.complex128),
    3: np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
}
