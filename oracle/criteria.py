"""Success criteria (Sec. II): the score P_psi of one final state.

fidelity  |<psi_R|psi>|^2 with the error-free final state psi_R
outcome   |psi_target|^2, the probability of measuring the correct result
binning   sum over the acceptable set S of |psi_k|^2
argmax    1 if the most likely outcome is the target (lowest index wins a tie), else 0
A trajectory passes when its score >= threshold.
"""
import numpy as np


def score(crit, psi, psi_ref=None):
    if crit.kind == "fidelity":
        return float(abs(np.vdot(psi_ref, psi)) ** 2)
    if crit.kind == "outcome":
        return float(abs(psi[crit.target]) ** 2)
    if crit.kind == "binning":
        idx = np.asarray(crit.basis_set, dtype=np.int64)
        return float(np.sum(np.abs(psi[idx]) ** 2))
    if crit.kind == "argmax":
        probs = np.abs(psi) ** 2
        return 1.0 if int(np.argmax(probs)) == crit.target else 0.0
    raise ValueError(crit.kind)


def passes(crit, s):
    return s >= crit.threshold


def heavy_outputs(psi_ref):
    """Heavy outputs of a quantum-volume circuit (Cross et al. 2019, the
    success measure the paper's QV evaluation uses): the basis states whose
    ideal probability exceeds the median of the ideal output distribution."""
    probs = np.abs(np.asarray(psi_ref)) ** 2
    return np.flatnonzero(probs > np.median(probs)).astype(np.uint64)
