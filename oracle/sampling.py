"""Monte Carlo Pauli error sampling (Sec. IV-B.2).

After a one-qubit gate an X, Z or Y error occurs with probabilities
p_X, p_Z, p_Y; after a two-qubit gate each of its qubits draws independently
with the same probabilities. Each (trajectory t, location l) draws from
Philox4x32-10 with

    counter = (l >> 1, t mod 2^32, t >> 32, 0x41525345),  key = (seed mod 2^32, seed >> 32)

and uses output words (w0, w1) when l is even, (w2, w3) when l is odd.
An error occurs iff w_a < thr, thr = min(floor(p_tot * 2^32), 2^32 - 1) with
p_tot = p_X + p_Z + p_Y (FP64). Its type compares w_b with
cut_X = floor(p_X / p_tot * 2^32) and cut_XZ = floor((p_X + p_Z) / p_tot * 2^32):
w_b < cut_X -> X, w_b < cut_XZ -> Z, else Y. Codes: 1 = X, 2 = Z, 3 = Y.

The draw does not depend on p, so the error sets at two rates are nested
(common random numbers across p).
"""
import math

import numpy as np

from .philox import philox4x32

STREAM_ERRORS = 0x41525345


def thresholds(p_x, p_z, p_y):
    p_tot = p_x + p_z + p_y
    if p_tot <= 0.0:
        return 0, 0, 0
    thr = min(math.floor(p_tot * 4294967296.0), 4294967295)
    cut_x = min(math.floor(p_x / p_tot * 4294967296.0), 4294967296)
    cut_xz = min(math.floor((p_x + p_z) / p_tot * 4294967296.0), 4294967296)
    return thr, cut_x, cut_xz


def draws(seed, t, L):
    """(w_a, w_b) for locations 0..L-1 of trajectory t, as uint64 arrays."""
    l = np.arange(L, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32(l >> np.uint64(1), np.uint64(t & 0xFFFFFFFF), np.uint64(t >> 32),
                                np.uint64(STREAM_ERRORS), np.uint64(seed & 0xFFFFFFFF),
                                np.uint64(seed >> 32))
    odd = (l & np.uint64(1)).astype(bool)
    wa = np.where(odd, w2, w0)
    wb = np.where(odd, w3, w1)
    return wa, wb


def sample_trajectory(seed, t, L, p_x, p_z, p_y):
    """Sorted list [(location, code), ...] of the errors of trajectory t."""
    thr, cut_x, cut_xz = thresholds(p_x, p_z, p_y)
    if thr == 0:
        return []
    wa, wb = draws(seed, t, L)
    hit = np.nonzero(wa < np.uint64(thr))[0]
    out = []
    for l in hit:
        b = int(wb[l])
        code = 1 if b < cut_x else (2 if b < cut_xz else 3)
        out.append((int(l), code))
    return out


def sample(seed, traj_begin, n_traj, L, p_x, p_z, p_y):
    return [sample_trajectory(seed, traj_begin + i, L, p_x, p_z, p_y) for i in range(n_traj)]
