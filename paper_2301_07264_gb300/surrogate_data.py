"""Training rows for the surrogate, produced by the trajectory simulator.

A row is (32 circuit features, log10 p) and its label is one trajectory's
pass flag at rate p (uniform p_X = p_Z = p_Y = p/3), so the network learns
P(pass | circuit, p) under the binary cross-entropy. Features, errors,
trajectories and flags all come from the C-ABI library; this module only
arranges the calls and concatenates device buffers.
"""
from __future__ import annotations

import math

import numpy as np

from . import arso


def rows_for_circuit(cc, crit, log10_ps, traj_per_p, seed, traj_begin=0, stream=None):
    """Device tensors (x: n x 33 float32, y: n float32) for one compiled circuit; the
    errors of all rates are sampled in one call and their trajectories run in one
    arso_run_batch call."""
    import torch
    f = torch.from_numpy(arso.circuit_features(cc, crit)).cuda()
    c = arso.make_criterion(crit)
    ps = [10.0 ** float(lp) / 3 for lp in log10_ps]
    errs = arso.sample_errors_batch([cc] * len(ps), ps, ps, ps, seed,
                                    [traj_begin + i * traj_per_p for i in range(len(ps))], traj_per_p, stream)
    scores, flags, xs = [], [], []
    for i, lp in enumerate(log10_ps):
        scores.append(torch.empty(traj_per_p, dtype=torch.float64, device="cuda"))
        flags.append(torch.empty(traj_per_p, dtype=torch.uint8, device="cuda"))
        x = torch.empty((traj_per_p, arso.SURROGATE_INPUTS), dtype=torch.float32, device="cuda")
        x[:, : arso.N_FEATURES] = f
        x[:, arso.N_FEATURES] = float(lp)
        xs.append(x)
    arso.run_batch([cc] * len(errs), errs, [c] * len(errs), scores, flags, stream)
    return torch.cat(xs), torch.cat([fl.to(torch.float32) for fl in flags])


def generate(circuits, n_rows, seed, lp_lo=-5.0, lp_hi=-1.0, p_points=16, stream=None):
    """Rows spread evenly over `circuits` (workload Circuit objects), log10 p
    drawn uniformly in [lp_lo, lp_hi] per point."""
    import torch
    rng = np.random.default_rng(seed)
    per_circuit = max(p_points, n_rows // max(len(circuits), 1))
    traj_per_p = max(1, per_circuit // p_points)
    xs, ys = [], []
    for k, circ in enumerate(circuits):
        cc = arso.compile_circuit(circ.n, circ.gates)
        lps = rng.uniform(lp_lo, lp_hi, size=p_points)
        x, y = rows_for_circuit(cc, circ.criterion, lps, traj_per_p, seed + k, stream=stream)
        xs.append(x)
        ys.append(y)
        del cc
    return torch.cat(xs), torch.cat(ys)


def log10_grid(p_lo, p_hi, k):
    a, b = math.log10(p_lo), math.log10(p_hi)
    return [a + (b - a) * i / (k - 1) for i in range(k)]
