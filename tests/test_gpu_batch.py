"""Batched execution of an uneven circuit mix through arso_run_batch: every
circuit's scores equal its own arso_run_trajectories scores (same error
lists), and a sample of trajectories matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import criteria, sampling, statevector
from workloads import circuits as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batch_matches_per_circuit_runs():
    from paper_2301_07264_gb300 import arso
    mix = [W.qft_basis(10, 77), W.grover(9, 5), W.qaoa_maxcut(12, 3), W.cuccaro_adder(5, 9, 22),
           W.qft_basis(13, 4000), W.qaoa_maxcut(8, 2), W.brickwork(11, 6, 5), W.cuccaro_adder(6, 40, 17),
           W.qaoa_maxcut(14, 8), W.qft_basis(16, 12345)]
    p, T = 5e-3, 300
    ccs, errs, crits, outs, flags, ref = [], [], [], [], [], []
    for k, circ in enumerate(mix):
        cc = arso.compile_circuit(circ.n, circ.gates)
        e = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, 1000 * k, T)
        ccs.append(cc)
        errs.append(e)
        crits.append(circ.criterion)
        outs.append(torch.full((T,), -1.0, dtype=torch.float64, device="cuda"))
        flags.append(torch.zeros(T, dtype=torch.uint8, device="cuda"))
        r = np.zeros(T)
        arso.run_trajectories(cc, e, circ.criterion, r)
        ref.append(r)
    host = [np.zeros(T) for _ in mix]
    arso.run_batch(ccs, errs, crits, outs, flags)
    arso.run_batch(ccs, errs, crits, host)
    for k, circ in enumerate(mix):
        got = outs[k].cpu().numpy()
        assert np.max(np.abs(got - ref[k])) < 1e-9, circ.family
        assert np.array_equal(host[k], got)
        assert np.array_equal(flags[k].cpu().numpy().astype(bool), got >= circ.criterion.threshold)
    # oracle spot checks on the batched (persistent-kernel) circuits
    for k in (0, 2, 6):
        circ = mix[k]
        lists = sampling.sample(0, 1000 * k, 6, circ.L, p / 3, p / 3, p / 3)
        psi_ref = statevector.simulate(circ)
        got = outs[k].cpu().numpy()
        for t in range(6):
            psi = statevector.simulate(circ, lists[t]) if lists[t] else psi_ref
            assert abs(got[t] - criteria.score(circ.criterion, psi, psi_ref)) < 1e-5
