"""Tolerable Pauli error rate (Sec. IV-D, Fig. 3).

1. Exhaustive single-error analysis gives P_psi_R and P_psi_e, hence the
   success probability subject to one average error, sum_e P_psi_e / 3.
2. If the target P is at least that value, at most one error is tolerable and
   Eq. (5) gives p directly.
3. Otherwise Monte Carlo simulations at increasing p are run until the target
   is matched. The paper converges with Powell's method; on this
   one-dimensional problem the oracle bisects in log10 p on estimates that
   share their random numbers across p (common random numbers), and returns
   the log-linear interpolation of the crossing inside the final bracket.
"""
import math

from . import exhaustive
from .montecarlo import aggregate, run_trajectories


def mc_value(circuit, p, n_traj, seed):
    s, f, _ = run_trajectories(circuit, seed, 0, n_traj, p / 3, p / 3, p / 3)
    a = aggregate(s, f)
    return a["mean"] if circuit.criterion.aggregate == "mean" else a["pass_frac"]


def bisect_log(f, target, p_lo, p_hi, rel_tol=0.02, max_probes=64):
    """Find p in [p_lo, p_hi] with f(p) = target, f decreasing. Returns
    (p, lo, hi, probes, converged)."""
    v_lo, v_hi = f(p_lo), f(p_hi)
    probes = 2
    if v_lo < target:
        return p_lo, p_lo, p_lo, probes, False
    if v_hi >= target:
        return p_hi, p_hi, p_hi, probes, False
    lo, hi = p_lo, p_hi
    while hi / lo > 1.0 + rel_tol and probes < max_probes:
        mid = math.sqrt(lo * hi)
        v = f(mid)
        probes += 1
        if v >= target:
            lo, v_lo = mid, v
        else:
            hi, v_hi = mid, v
    if v_lo == v_hi:
        p = math.sqrt(lo * hi)
    else:
        frac = (v_lo - target) / (v_lo - v_hi)
        p = 10 ** (math.log10(lo) + frac * (math.log10(hi) - math.log10(lo)))
    return p, lo, hi, probes, hi / lo <= 1.0 + rel_tol


def tolerable_rate(circuit, P_target, n_traj=1000, seed=0, p_lo=1e-6, p_hi=1e-1,
                   rel_tol=0.02, count="locations", mode="auto"):
    """mode "auto" follows Fig. 3; "mc" skips the Eq. (5) branch."""
    a = exhaustive.analyse(circuit)
    P1 = exhaustive.one_error_success(a)
    if mode == "auto" and P_target >= P1:
        return {"p": exhaustive.eq5(a, P_target, count), "mode": "eq5", "P1": P1, "analysis": a}
    p, lo, hi, probes, ok = bisect_log(lambda q: mc_value(circuit, q, n_traj, seed), P_target,
                                       p_lo, p_hi, rel_tol)
    return {"p": p, "lo": lo, "hi": hi, "probes": probes, "converged": ok, "mode": "mc",
            "P1": P1, "analysis": a}
