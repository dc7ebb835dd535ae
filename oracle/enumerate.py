"""Brute-force expectation of the Monte Carlo model: every assignment of
{I, X, Z, Y} to the L error locations (4^L patterns, L <= 8), weighted by
prod over locations of (1 - p_tot) or p_e. Gives the exact expected score
and the exact pass probability, for any criterion.
"""
import itertools

from .criteria import passes, score
from .statevector import simulate


def expectation(circuit, p_x, p_z, p_y):
    L = circuit.L
    assert L <= 8, "brute force is for L <= 8"
    crit = circuit.criterion
    psi_ref = simulate(circuit)
    w = {0: 1.0 - p_x - p_z - p_y, 1: p_x, 2: p_z, 3: p_y}
    e_score = 0.0
    e_pass = 0.0
    for pattern in itertools.product((0, 1, 2, 3), repeat=L):
        weight = 1.0
        for c in pattern:
            weight *= w[c]
        if weight == 0.0:
            continue
        ev = [(l, c) for l, c in enumerate(pattern) if c]
        s = score(crit, simulate(circuit, ev), psi_ref)
        e_score += weight * s
        e_pass += weight * float(passes(crit, s))
    return e_score, e_pass
