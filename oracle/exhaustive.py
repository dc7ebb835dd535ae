"""Exhaustive single-error simulation and the closed forms built on it.

Sec. IV-B.1 / Eq. (3): the reference state psi_R (no error), then every single
X, Z and Y error at every error location, k + 2m locations for a circuit with
k one-qubit and m two-qubit gates, giving 3(k+2m) erroneous states.

Sec. IV-C / Eq. (4): with P_psi_e the criterion averaged over the states of
error type e and E(N_e) the expected number of type-e errors,
    P = sum_e P_psi_e E(N_e) + P_psi_R (1 - sum_e E(N_e)).

Sec. IV-D / Eq. (5): for a uniform rate (p_e = p/3),
    p = (P - P_psi_R) / (count * (sum_e P_psi_e / 3 - P_psi_R)).

Reading: ``count`` (the number that multiplies p_e in E(N_e)) is the number of
error locations L = k + 2m, because two-qubit gates draw an error on each of
their qubits (Sec. IV-B.2); with that count Eq. (4) is the exact first-order
expansion of the Monte Carlo model in p. ``count="gates"`` gives the literal
G reading of the text.
"""
import numpy as np

from .criteria import passes, score
from .statevector import location_table, simulate

CODES = {"X": 1, "Z": 2, "Y": 3}


def single_error_states(circuit):
    """Yield (location, code, state) for every element of the Eq. (3) set."""
    L = len(location_table(circuit))
    for name in ("X", "Z", "Y"):
        code = CODES[name]
        for l in range(L):
            yield l, code, simulate(circuit, [(l, code)])


def _value(crit, psi, psi_ref):
    s = score(crit, psi, psi_ref)
    return s if crit.aggregate == "mean" else float(passes(crit, s))


def analyse(circuit):
    """Return P_R, P_e (dict over X, Z, Y), the per-location values and L, G."""
    crit = circuit.criterion
    psi_ref = simulate(circuit)
    P_R = _value(crit, psi_ref, psi_ref)
    L = circuit.L
    per = {"X": np.zeros(L), "Z": np.zeros(L), "Y": np.zeros(L)}
    inv = {v: k for k, v in CODES.items()}
    for l, code, psi in single_error_states(circuit):
        per[inv[code]][l] = _value(crit, psi, psi_ref)
    P_e = {e: float(np.mean(v)) if L else 0.0 for e, v in per.items()}
    return {"P_R": P_R, "P_e": P_e, "per_location": per, "L": L, "G": circuit.G}


def _count(a, count):
    return a["L"] if count == "locations" else a["G"]


def eq4(a, p_x, p_z, p_y, count="locations"):
    c = _count(a, count)
    E = {"X": c * p_x, "Z": c * p_z, "Y": c * p_y}
    return sum(a["P_e"][e] * E[e] for e in E) + a["P_R"] * (1.0 - sum(E.values()))


def one_error_success(a):
    """Success probability subject to one average error: sum_e P_psi_e / 3."""
    return sum(a["P_e"].values()) / 3.0


def eq5(a, P_target, count="locations"):
    c = _count(a, count)
    denom = one_error_success(a) - a["P_R"]
    if denom == 0.0:
        return float("inf")
    return (P_target - a["P_R"]) / (c * denom)
