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


def _mix_cases():
    """Every family at every engine size: below 10 qubits (shared-memory items),
    10..13 (register-blocked resident items) and 14+ (streaming tiles)."""
    return [W.qft_basis(8, 201), W.grover(7, 3), W.qaoa_maxcut(8, 11), W.cuccaro_adder(3, 5, 6),
            W.qft_basis(9, 300), W.grover_seeded(9, 17), W.brickwork(9, 12, 4),
            W.qft_basis(10, 77), W.grover(9, 5), W.qaoa_maxcut(12, 3), W.cuccaro_adder(5, 9, 22),
            W.qft_basis(14, 9000), W.qaoa_maxcut(14, 8), W.cuccaro_adder(6, 40, 17), W.brickwork(15, 10, 6),
            W.qft_basis(16, 12345), W.qaoa_maxcut(16, 21), W.cuccaro_adder(7, 101, 77), W.brickwork(18, 8, 7)]


@pytest.mark.parametrize("p", [2e-3, 2e-2])
def test_persistent_batch_matches_separate_launches_and_oracle(p):
    """One persistent launch for the whole mix against the same circuits run on
    their own launches (ARSO_OPT_NO_PERSISTENT) and against the FP64 oracle."""
    from paper_2301_07264_gb300 import arso
    mix = _mix_cases()
    T = 96
    ccs, sep, errs, errs_sep, crits = [], [], [], [], []
    for k, circ in enumerate(mix):
        cc = arso.compile_circuit(circ.n, circ.gates)
        cs = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_PERSISTENT)
        ccs.append(cc)
        sep.append(cs)
        errs.append(arso.sample_errors(cc, p / 3, p / 3, p / 3, 3, 500 * k, T))
        errs_sep.append(arso.sample_errors(cs, p / 3, p / 3, p / 3, 3, 500 * k, T))
        crits.append(circ.criterion)
    got = [torch.full((T,), -1.0, dtype=torch.float64, device="cuda") for _ in mix]
    gotf = [torch.zeros(T, dtype=torch.uint8, device="cuda") for _ in mix]
    ref = [np.full(T, -1.0) for _ in mix]
    arso.run_batch(ccs, errs, crits, got, gotf)  # builds every circuit's prefix cache
    for g in got:
        g.fill_(-1.0)
    arso.profile_reset()
    arso.run_batch(ccs, errs, crits, got, gotf)
    launches, _, _ = arso.profile_counters()
    assert arso.profile_read(arso.K_MIX).launches == 1
    assert launches == 1  # the persistent launch; no other kernel of the library
    arso.run_batch(sep, errs_sep, crits, ref)
    for k, circ in enumerate(mix):
        g = got[k].cpu().numpy()
        assert np.all(g >= 0.0), (circ.family, circ.n)
        assert np.max(np.abs(g - ref[k])) < 1e-12, (circ.family, circ.n)
        assert np.array_equal(gotf[k].cpu().numpy().astype(bool), g >= circ.criterion.threshold)
    # FP64 oracle on trajectories with errors, every family and engine size
    for k, circ in enumerate(mix):
        if circ.n > 16:
            continue
        lists = sampling.sample(3, 500 * k, T, circ.L, p / 3, p / 3, p / 3)
        psi_ref = statevector.simulate(circ)
        g = got[k].cpu().numpy()
        checked = 0
        for t in range(T):
            if not lists[t] and checked:
                continue
            psi = statevector.simulate(circ, lists[t]) if lists[t] else psi_ref
            assert abs(g[t] - criteria.score(circ.criterion, psi, psi_ref)) < 1e-5, (circ.family, circ.n, t)
            checked += 1
            if checked >= 3:
                break


def test_persistent_batch_repeated_circuit_and_empty_lists():
    """The same circuit several times in one call (the Grover rate sweep does this),
    an empty error list and error-free lists."""
    from paper_2301_07264_gb300 import arso
    a, b = W.grover(10, 7), W.qaoa_maxcut(14, 5)
    ca = arso.compile_circuit(a.n, a.gates)
    cb = arso.compile_circuit(b.n, b.gates)
    rates = (0.0, 1e-3, 1e-2)
    ccs, errs, crits, outs = [], [], [], []
    for r in rates:
        for cc, circ in ((ca, a), (cb, b)):
            ccs.append(cc)
            errs.append(arso.sample_errors(cc, r / 3, r / 3, r / 3, 1, 0, 64))
            crits.append(circ.criterion)
            outs.append(np.zeros(64))
    ccs.append(ca)
    errs.append(arso.sample_errors(ca, 1e-3, 1e-3, 1e-3, 1, 0, 0))
    crits.append(a.criterion)
    outs.append(np.zeros(0))
    arso.run_batch(ccs, errs, crits, outs)
    for i in range(len(rates) * 2):
        single = np.zeros(64)
        arso.run_trajectories(ccs[i], errs[i], crits[i], single)
        assert np.max(np.abs(single - outs[i])) < 1e-12
    assert np.ptp(outs[0]) == 0.0 and np.ptp(outs[1]) == 0.0  # p = 0: every trajectory error-free


def test_autotuned_schedule_against_oracle():
    """A circuit compiled with the schedule arso_autotune picks scores its
    trajectories like the FP64 oracle."""
    from paper_2301_07264_gb300 import arso
    circ = W.qaoa_maxcut(16, 9)
    opts, ms = arso.autotune(circ.n, circ.gates, circ.criterion, 4e-3, n_traj=32)
    assert len(ms) > 1 and np.all(ms > 0)
    cc = arso.compile_circuit(circ.n, circ.gates, **opts)
    T, p = 40, 3e-3
    s = np.zeros(T)
    arso.run_trajectories(cc, arso.sample_errors(cc, p / 3, p / 3, p / 3, 2, 0, T), circ.criterion, s)
    lists = sampling.sample(2, 0, T, circ.L, p / 3, p / 3, p / 3)
    psi_ref = statevector.simulate(circ)
    for t in [i for i in range(T) if lists[i]][:4]:
        assert abs(s[t] - criteria.score(circ.criterion, statevector.simulate(circ, lists[t]), psi_ref)) < 1e-5


def test_persistent_batch_wait_that_runs_out_reports_timeout():
    """The failure path of the persistent launch's bounded dependency waits: a
    launch whose waits cannot be met gives up (no hang, no fault), the call
    returns ETIMEOUT, and the next call on the same context gives the scores of
    the circuits' own launches again."""
    import time
    from paper_2301_07264_gb300 import arso
    mix = [W.qaoa_maxcut(12, 3), W.qft_basis(14, 9000), W.brickwork(15, 10, 6), W.grover(7, 3)]
    p, T = 5e-3, 64
    ccs, errs, crits, ref = [], [], [], []
    for k, circ in enumerate(mix):
        cc = arso.compile_circuit(circ.n, circ.gates)
        e = arso.sample_errors(cc, p / 3, p / 3, p / 3, 9, 100 * k, T)
        r = np.zeros(T)
        arso.run_trajectories(cc, e, circ.criterion, r)
        ccs.append(cc)
        errs.append(e)
        crits.append(circ.criterion)
        ref.append(r)
    got = [torch.full((T,), -1.0, dtype=torch.float64, device="cuda") for _ in mix]
    arso.debug_stall_next_batch()
    t0 = time.perf_counter()
    with pytest.raises(arso.ArsoError) as e:
        arso.run_batch(ccs, errs, crits, got)
    assert e.value.status == arso.ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    arso.run_batch(ccs, errs, crits, got)
    for k, circ in enumerate(mix):
        assert np.max(np.abs(got[k].cpu().numpy() - ref[k])) < 1e-9, circ.family
