"""Monte Carlo success probability (Sec. IV-B.2, Sec. IV-C last paragraph):
simulate N trajectories under sampled Pauli errors and average the criterion
score P_psi over psi_1..psi_N. Also reports the pass fraction and the standard
error of each. Every trajectory is simulated from |0...0> (no prefix reuse).
"""
import math

import numpy as np

from .criteria import passes, score
from .sampling import sample_trajectory
from .statevector import simulate


def reference_state(circuit):
    return simulate(circuit)


def run_trajectories(circuit, seed, traj_begin, n_traj, p_x, p_z, p_y, psi_ref=None):
    """Per-trajectory (scores, pass flags, error lists)."""
    crit = circuit.criterion
    if psi_ref is None:
        psi_ref = reference_state(circuit)
    L = circuit.L
    scores = np.empty(n_traj)
    flags = np.empty(n_traj, dtype=bool)
    errs = []
    for i in range(n_traj):
        ev = sample_trajectory(seed, traj_begin + i, L, p_x, p_z, p_y)
        psi = simulate(circuit, ev) if ev else psi_ref
        s = score(crit, psi, psi_ref)
        scores[i] = s
        flags[i] = passes(crit, s)
        errs.append(ev)
    return scores, flags, errs


def aggregate(scores, flags):
    n = len(scores)
    mean = float(np.mean(scores)) if n else 0.0
    pf = float(np.mean(flags)) if n else 0.0
    sd_s = float(np.std(scores, ddof=1)) if n > 1 else 0.0
    sd_p = float(np.std(flags.astype(float), ddof=1)) if n > 1 else 0.0
    return {"mean": mean, "pass_frac": pf, "stderr_mean": sd_s / math.sqrt(max(n, 1)),
            "stderr_pass": sd_p / math.sqrt(max(n, 1))}


def success_prob_mc(circuit, p, n_traj=1000, seed=0, traj_begin=0):
    """Uniform rate p (p_X = p_Z = p_Y = p/3)."""
    s, f, _ = run_trajectories(circuit, seed, traj_begin, n_traj, p / 3, p / 3, p / 3)
    return aggregate(s, f)
