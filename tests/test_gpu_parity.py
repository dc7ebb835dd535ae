"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars: sampled error events bit-exact; complex64 amplitudes within 1e-5
max-abs of the FP64 oracle (complex128 within 1e-12); per-trajectory scores
within 1e-5; pass flags identical except for trajectories whose oracle score
lies within 1e-5 of the threshold (or, for argmax, whose two largest
probabilities lie within 1e-6).
"""
import math

import numpy as np
import pytest

from oracle import criteria, exhaustive as ox, montecarlo, sampling, search, statevector
from workloads import circuits as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL_C64 = 1e-5
AMP_TOL_C128 = 1e-12
SCORE_TOL = 1e-5


@pytest.fixture(scope="module")
def arso():
    from paper_2301_07264_gb300 import arso as mod
    assert torch.cuda.is_available()
    return mod


def oracle_csr(lists):
    off = np.zeros(len(lists) + 1, dtype=np.uint64)
    ev = []
    for i, l in enumerate(lists):
        off[i + 1] = off[i] + len(l)
        ev += [(loc << 2) | code for loc, code in l]
    return off, np.asarray(ev, dtype=np.uint32)


def gpu_states(arso, circ, cc, errs, first, count, c128=False):
    dt = torch.complex128 if c128 else torch.complex64
    out = torch.empty((count, 1 << circ.n), dtype=dt, device="cuda")
    arso.trajectory_states(cc, errs, first, count, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def flags_comparable(crit, oracle_score, psi=None):
    if crit.kind == "argmax":
        p = np.sort(np.abs(psi) ** 2)
        return p[-1] - p[-2] > 1e-6
    return abs(oracle_score - crit.threshold) > SCORE_TOL


# ------------------------------------------------------------- sampling ---

@pytest.mark.parametrize("case", [
    ("qft4", 1e-3, 1e-3, 1e-3, 0, 0, 1000),
    ("qft4", 0.2, 0.05, 0.01, 7, 2**32 - 3, 300),     # traj ids cross 2^32
    ("rand", 0.3, 0.0, 0.0, 1, 5, 200),               # X only
    ("rand", 0.0, 0.0, 0.4, 2, 0, 100),               # Y only
    ("rand", 1 / 3, 1 / 3, 1 / 3, 3, 0, 20),          # p_tot = 1
    ("rand", 0.0, 0.0, 0.0, 4, 0, 50),                # no errors
    ("grover", 1e-3, 1e-3, 1e-3, 0, 0, 16),
])
def test_sampling_bit_exact(arso, case):
    name, px, pz, py, seed, begin, T = case
    circ = {"qft4": C.qft4_0101, "rand": lambda: C.random_circuit(5, 37, 11),
            "grover": lambda: C.grover12(0)}[name]()
    cc = arso.compile_circuit(circ.n, circ.gates)
    errs = arso.sample_errors(cc, px, pz, py, seed, begin, T)
    off, ev = arso.error_list_copy(errs)
    o_off, o_ev = oracle_csr(sampling.sample(seed, begin, T, circ.L, px, pz, py))
    assert np.array_equal(off, o_off)
    assert np.array_equal(ev, o_ev)


def test_sampling_empty_and_single(arso):
    circ = C.Circuit(1, [C.Gate("H", (0,))])
    cc = arso.compile_circuit(1, circ.gates)
    errs = arso.sample_errors(cc, 0.1, 0.1, 0.1, 0, 0, 0)
    assert errs.info() == (0, 0)
    errs = arso.sample_errors(cc, 0.3, 0.3, 0.3, 9, 0, 500)
    off, ev = arso.error_list_copy(errs)
    o_off, o_ev = oracle_csr(sampling.sample(9, 0, 500, 1, 0.3, 0.3, 0.3))
    assert np.array_equal(off, o_off) and np.array_equal(ev, o_ev)


def test_batched_sampling_bit_exact(arso):
    """arso_sample_errors_batch: every list equals the oracle's sampling and the
    per-list sampler's, including trajectory ids across 2^32, single-type rates,
    p = 0, an empty list and a streaming schedule that reorders gates (whose
    engine-order keys decide the scores)."""
    circs = [C.qft4_0101(), C.random_circuit(5, 37, 11), C.grover(7, 3), C.brickwork(14, 6, 2),
             C.random_circuit(6, 50, 3), C.qaoa_maxcut(12, 5)]
    kws = [{"precision": arso.C128}, {}, {}, {"tile_qubits": 10}, {}, {}]
    par = [(0.2, 0.05, 0.01, 7, 2**32 - 3, 300), (0.3, 0.0, 0.0, 1, 5, 200), (1e-3, 1e-3, 1e-3, 0, 0, 64),
           (4e-3, 4e-3, 4e-3, 2, 100, 48), (0.0, 0.0, 0.0, 4, 0, 50), (0.0, 0.0, 0.4, 2, 0, 0)]
    ccs = [arso.compile_circuit(c.n, c.gates, **kw) for c, kw in zip(circs, kws)]
    lists = arso.sample_errors_batch(ccs, [q[0] for q in par], [q[1] for q in par], [q[2] for q in par],
                                     [q[3] for q in par], [q[4] for q in par], [q[5] for q in par])
    for circ, cc, q, e in zip(circs, ccs, par, lists):
        px, pz, py, seed, begin, T = q
        off, ev = arso.error_list_copy(e)
        o_off, o_ev = oracle_csr(sampling.sample(seed, begin, T, circ.L, px, pz, py))
        assert np.array_equal(off, o_off) and np.array_equal(ev, o_ev), circ.family
        if T:
            single = arso.sample_errors(cc, px, pz, py, seed, begin, T)
            a, b = np.zeros(T), np.zeros(T)
            arso.run_trajectories(cc, e, circ.criterion, a)
            arso.run_trajectories(cc, single, circ.criterion, b)
            assert np.array_equal(a, b), circ.family


# ------------------------------------------------------------ amplitudes --

def _random_error_lists(circ, T, rng, max_err=4):
    lists = []
    for t in range(T):
        k = int(rng.integers(0, max_err + 1))
        locs = sorted(rng.choice(circ.L, size=min(k, circ.L), replace=False).tolist()) if circ.L else []
        lists.append([(int(l), int(rng.integers(1, 4))) for l in locs])
    return lists


@pytest.mark.parametrize("n,G,seed,c128", [
    (1, 30, 1, False), (2, 40, 2, False), (4, 60, 3, True), (7, 120, 4, False),
    (10, 150, 5, False), (12, 200, 6, True), (13, 160, 7, False),
])
def test_resident_amplitudes(arso, n, G, seed, c128):
    circ = C.random_circuit(n, G, seed)
    rng = np.random.default_rng(seed)
    lists = _random_error_lists(circ, 6, rng)
    lists[0] = []                                       # error-free
    lists[1] = [(0, 3)] if circ.L else []               # first location
    lists[2] = [(circ.L - 1, 1)] if circ.L else []      # last location
    cc = arso.compile_circuit(n, circ.gates, precision=arso.C128 if c128 else arso.C64)
    assert cc.info().engine == 0
    errs = arso.error_list_from_host(cc, lists)
    got = gpu_states(arso, circ, cc, errs, 0, len(lists), c128)
    tol = AMP_TOL_C128 if c128 else AMP_TOL_C64
    for t, ev in enumerate(lists):
        assert np.max(np.abs(got[t] - statevector.simulate(circ, ev))) < tol, t


@pytest.mark.parametrize("n,G,tile,low,seed", [
    (14, 200, 8, 3, 1), (15, 300, 10, 4, 2), (16, 260, 13, 4, 3), (14, 120, 6, 1, 4), (17, 150, 14, 5, 5),
    (17, 320, 12, 4, 6), (16, 240, 11, 3, 7),
])
def test_streaming_amplitudes(arso, n, G, tile, low, seed):
    circ = C.random_circuit(n, G, seed)
    rng = np.random.default_rng(seed)
    lists = _random_error_lists(circ, 5, rng, max_err=6)
    lists[0] = []
    # both slots of one two-qubit gate
    g2 = next(i for i, g in enumerate(circ.gates) if g.arity == 2)
    loc = sum(g.arity for g in circ.gates[:g2])
    lists[1] = [(loc, 2), (loc + 1, 3)]
    cc = arso.compile_circuit(n, circ.gates, tile_qubits=tile, low_qubits=low)
    info = cc.info()
    assert info.engine == 1 and info.n_passes > 1
    errs = arso.error_list_from_host(cc, lists)
    got = gpu_states(arso, circ, cc, errs, 0, len(lists))
    for t, ev in enumerate(lists):
        assert np.max(np.abs(got[t] - statevector.simulate(circ, ev))) < AMP_TOL_C64, t


@pytest.mark.parametrize("tile,seed", [(10, 11), (11, 12), (12, 14), (13, 13)])
def test_register_blocked_many_errors(arso, tile, seed):
    """Dense error lists: X/Y errors become index masks that later gates
    (dense, CX, CZ, diagonal, SWAP, U2) must see through."""
    circ = C.random_circuit(15, 250, seed, two_qubit_frac=0.5)
    rng = np.random.default_rng(seed)
    lists = _random_error_lists(circ, 6, rng, max_err=40)
    cc = arso.compile_circuit(15, circ.gates, tile_qubits=tile)
    errs = arso.error_list_from_host(cc, lists)
    got = gpu_states(arso, circ, cc, errs, 0, len(lists))
    for t, ev in enumerate(lists):
        assert np.max(np.abs(got[t] - statevector.simulate(circ, ev))) < AMP_TOL_C64, t


@pytest.mark.parametrize("cache_boundaries", [0, 5])
def test_suffix_reuse_scores_equal_full_runs(arso, cache_boundaries):
    """Fidelity taken right after the last error against the cached error-free
    state equals fidelity of the full run (the error-free suffix is unitary)."""
    circ = C.brickwork(18, 24, seed=4)
    sb = (1 << 18) * 8
    kw = dict(tile_qubits=12, cache_bytes=cache_boundaries * sb)
    on = arso.compile_circuit(circ.n, circ.gates, **kw)
    off = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_SUFFIX_REUSE, **kw)
    T, p = 48, 2e-3
    s_on, s_off = np.zeros(T), np.zeros(T)
    arso.run_trajectories(on, arso.sample_errors(on, p / 3, p / 3, p / 3, 9, 0, T), circ.criterion, s_on)
    arso.run_trajectories(off, arso.sample_errors(off, p / 3, p / 3, p / 3, 9, 0, T), circ.criterion, s_off)
    assert np.max(np.abs(s_on - s_off)) < SCORE_TOL
    lists = sampling.sample(9, 0, T, circ.L, p / 3, p / 3, p / 3)
    psi_ref = statevector.simulate(circ)
    for t in [i for i in range(T) if lists[i]][:3]:
        o = criteria.score(circ.criterion, statevector.simulate(circ, lists[t]), psi_ref)
        assert abs(s_on[t] - o) < SCORE_TOL


def test_streaming_prefix_cache_subset(arso):
    # a cache budget that cannot hold every pass boundary forces restarts from
    # an earlier cached boundary
    circ = C.brickwork(14, 12, seed=3)
    rng = np.random.default_rng(0)
    lists = _random_error_lists(circ, 6, rng, max_err=3)
    sb = (1 << 14) * 8
    cc = arso.compile_circuit(14, circ.gates, tile_qubits=8, low_qubits=3, cache_bytes=6 * sb)
    assert cc.info().n_passes > 6
    errs = arso.error_list_from_host(cc, lists)
    got = gpu_states(arso, circ, cc, errs, 0, len(lists))
    for t, ev in enumerate(lists):
        assert np.max(np.abs(got[t] - statevector.simulate(circ, ev))) < AMP_TOL_C64


def test_reference_state(arso):
    for circ in (C.qft_basis(9, 300), C.brickwork(15, 6, 2), C.ghz(13)):
        cc = arso.compile_circuit(circ.n, circ.gates)
        out = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
        arso.reference_state(cc, out)
        assert np.max(np.abs(out.cpu().numpy() - statevector.simulate(circ))) < AMP_TOL_C64


# ---------------------------------------------------------------- scores --

def _crit_cases(n, psi_ref):
    probs = np.abs(psi_ref) ** 2
    top = int(np.argmax(probs))
    heavy = tuple(int(i) for i in np.nonzero(probs > np.median(probs))[0])
    return [
        C.Criterion("fidelity", threshold=0.9, aggregate="pass"),
        C.Criterion("outcome", target=top, threshold=0.5 * probs[top], aggregate="mean"),
        C.Criterion("binning", basis_set=heavy, threshold=0.5, aggregate="mean"),
        C.Criterion("argmax", target=top, threshold=0.5, aggregate="pass"),
    ]


@pytest.mark.parametrize("n,G,tile", [(6, 80, 0), (12, 150, 0), (15, 120, 9)])
def test_scores_every_criterion(arso, n, G, tile):
    circ = C.random_circuit(n, G, 40 + n)
    psi_ref = statevector.simulate(circ)
    p = 3.0 / circ.L
    cc = arso.compile_circuit(n, circ.gates, tile_qubits=tile)
    T = 24
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 5, 0, T)
    lists = sampling.sample(5, 0, T, circ.L, p / 3, p / 3, p / 3)
    states = [statevector.simulate(circ, ev) if ev else psi_ref for ev in lists]
    for crit in _crit_cases(n, psi_ref):
        score = np.zeros(T)
        flags = np.zeros(T, dtype=np.uint8)
        arso.run_trajectories(cc, errs, crit, score, flags)
        dev = torch.zeros(T, dtype=torch.float64, device="cuda")
        arso.run_trajectories(cc, errs, crit, dev)
        assert np.array_equal(dev.cpu().numpy(), score)
        for t in range(T):
            o = criteria.score(crit, states[t], psi_ref)
            assert abs(score[t] - o) < SCORE_TOL, (crit.kind, t)
            if flags_comparable(crit, o, states[t]):
                assert bool(flags[t]) == criteria.passes(crit, o), (crit.kind, t)


def _unitary4(rng):
    z = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def test_score_state_and_standalone_kernels(arso):
    rng = np.random.default_rng(1)
    for n in (3, 12, 20):
        psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        psi /= np.linalg.norm(psi)
        d = torch.from_numpy(psi.astype(np.complex64)).cuda()
        for gate in [C.Gate("H", (0,)), C.Gate("T", (n - 1,)), C.Gate("X", (n // 2,)),
                     C.Gate("RY", (1 % n,), (0.3,)), C.Gate("U", (n - 1,), (), C.haar_su2(rng))] + (
                [C.Gate("CX", (n - 1, 0)), C.Gate("CZ", (1, n - 1)), C.Gate("CP", (0, 2), (1.1,)),
                 C.Gate("SWAP", (n - 1, 1)), C.Gate("U2", (2, n - 2), (), _unitary4(rng))] if n >= 3 else []):
            arso.apply_gate(n, d, gate)
            statevector.apply_gate(psi, n, gate)
            assert np.max(np.abs(d.cpu().numpy() - psi)) < AMP_TOL_C64, gate.name
        for q, code in ((0, 1), (n - 1, 3), (n // 2, 2)):
            arso.apply_pauli(n, d, q, code)
            statevector.apply_pauli(psi, n, q, code)
            assert np.max(np.abs(d.cpu().numpy() - psi)) < AMP_TOL_C64
        ref = torch.from_numpy(psi.astype(np.complex64)).cuda()
        s = arso.score_state(n, d, ref, C.Criterion("fidelity"))
        assert abs(s - 1.0) < 1e-5
        s = arso.score_state(n, d, None, C.Criterion("binning", basis_set=(0, 1, 5 % (1 << n))))
        assert abs(s - criteria.score(C.Criterion("binning", basis_set=(0, 1, 5 % (1 << n))), psi)) < 1e-6


# ------------------------------------------------- aggregates and search --

def test_qft4_config_full_parity(arso):
    """4-qubit QFT on |0101>, p = 1e-3, 1000 trajectories, seed 0, complex128."""
    circ = C.qft4_0101()
    crit = circ.criterion
    cc = arso.compile_circuit(circ.n, circ.gates, precision=arso.C128)
    errs = arso.sample_errors(cc, 1e-3 / 3, 1e-3 / 3, 1e-3 / 3, 0, 0, 1000)
    score = np.zeros(1000)
    flags = np.zeros(1000, dtype=np.uint8)
    arso.run_trajectories(cc, errs, crit, score, flags)
    o_s, o_f, _ = montecarlo.run_trajectories(circ, 0, 0, 1000, 1e-3 / 3, 1e-3 / 3, 1e-3 / 3)
    assert np.max(np.abs(score - o_s)) < 1e-12
    # some single errors leave the fidelity at exactly 1/2 = threshold; there the
    # flag depends on the last rounding, so only scores away from it are compared
    away = np.abs(o_s - crit.threshold) > 1e-9
    assert away.sum() > 900
    assert np.array_equal(flags.astype(bool)[away], o_f[away])
    r = arso.success_prob(cc, crit, 1e-3, mode="mc", n_traj=1000, seed=0)
    agg = montecarlo.aggregate(o_s, o_f)
    assert abs(r.pass_frac - agg["pass_frac"]) <= (~away).sum() / 1000 + 1e-12
    assert abs(r.mean - agg["mean"]) < 1e-12
    own = montecarlo.aggregate(score, flags.astype(bool))  # the GPU's own flags
    assert abs(r.pass_frac - own["pass_frac"]) < 1e-12
    assert abs(r.stderr_value - own["stderr_pass"]) < 1e-9


def test_exhaustive_and_eq4(arso):
    for circ in (C.ghz(5), C.random_circuit(6, 30, 2), C.qft4_0101()):
        crit = C.Criterion("fidelity", threshold=0.5, aggregate="mean")
        circ.criterion = crit
        cc = arso.compile_circuit(circ.n, circ.gates)
        P, per = arso.exhaustive(cc, crit)
        a = ox.analyse(circ)
        assert abs(P[0] - a["P_R"]) < SCORE_TOL
        for k, e in enumerate(("X", "Z", "Y")):
            assert abs(P[1 + k] - a["P_e"][e]) < SCORE_TOL
            assert np.max(np.abs(per[k * circ.L:(k + 1) * circ.L] - a["per_location"][e])) < SCORE_TOL
        p = 0.2 / circ.L
        r = arso.success_prob(cc, crit, p, mode="auto")
        assert r.mode_used == 2
        assert abs(r.value - ox.eq4(a, p / 3, p / 3, p / 3)) < SCORE_TOL


def test_tolerable_rate_matches_oracle(arso):
    circ = C.ghz(4)
    crit = C.Criterion("fidelity", aggregate="mean")
    circ.criterion = crit
    cc = arso.compile_circuit(circ.n, circ.gates)
    a = ox.analyse(circ)
    P1 = ox.one_error_success(a)
    target = 0.5 * (P1 + a["P_R"])
    r = arso.tolerable_rate(cc, crit, target)
    # complex64 scores agree within 1e-5, so Eq. (5) agrees to ~1e-5 relative
    assert r.mode_used == 0 and abs(r.p - ox.eq5(a, target)) < 1e-4 * ox.eq5(a, target)
    # Monte Carlo branch on common random numbers: identical probes
    r = arso.tolerable_rate(cc, crit, 0.8, n_traj=400, seed=3, mode="mc", rel_tol=0.05)
    o = search.bisect_log(lambda q: search.mc_value(circ, q, 400, 3), 0.8, 1e-6, 1e-1, rel_tol=0.05)
    assert r.converged and o[4]
    assert abs(r.p - o[0]) / o[0] < 1e-3


def test_error_free_and_empty_circuits(arso):
    circ = C.Circuit(3, [])
    cc = arso.compile_circuit(3, [])
    errs = arso.sample_errors(cc, 0.1, 0.1, 0.1, 0, 0, 5)
    s = np.zeros(5)
    arso.run_trajectories(cc, errs, C.Criterion("outcome", target=0), s)
    assert np.allclose(s, 1.0)
    big = C.Circuit(15, [])
    cc = arso.compile_circuit(15, [])
    out = torch.empty(1 << 15, dtype=torch.complex64, device="cuda")
    arso.reference_state(cc, out)
    v = out.cpu().numpy()
    assert v[0] == 1 and np.all(v[1:] == 0)


def test_invalid_arguments_fail_cleanly(arso):
    with pytest.raises(arso.ArsoError) as e:
        arso.compile_circuit(3, [C.Gate("H", (3,))])
    assert e.value.status == arso.EINVAL
    cc = arso.compile_circuit(2, [C.Gate("H", (0,))])
    with pytest.raises(arso.ArsoError):
        arso.sample_errors(cc, 0.5, 0.5, 0.5, 0, 0, 10)
    errs = arso.sample_errors(cc, 0.1, 0.1, 0.1, 0, 0, 10)
    with pytest.raises(arso.ArsoError):
        arso.run_trajectories(cc, errs, C.Criterion("outcome", target=4), np.zeros(10))
    with pytest.raises(arso.ArsoError):
        arso.error_list_from_host(cc, [[(0, 1), (0, 2)]])


# --------------------------------------------------- full-size workloads --

def test_grover12_sampled_trajectories(arso):
    """Grover, 11 search qubits + 1 borrowed, resident engine at full size:
    bit-exact events for 64 trajectories, scores and amplitudes for two."""
    circ = C.grover12(0)
    cc = arso.compile_circuit(circ.n, circ.gates)
    p = 1e-4
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, 0, 64)
    off, ev = arso.error_list_copy(errs)
    lists = sampling.sample(0, 0, 64, circ.L, p / 3, p / 3, p / 3)
    o_off, o_ev = oracle_csr(lists)
    assert np.array_equal(off, o_off) and np.array_equal(ev, o_ev)
    score = np.zeros(64)
    arso.run_trajectories(cc, errs, circ.criterion, score)
    idx = [t for t in range(64) if lists[t]][:2]
    states = gpu_states(arso, circ, cc, errs, idx[0], 1)
    psi = statevector.simulate(circ, lists[idx[0]])
    assert np.max(np.abs(states[0] - psi)) < AMP_TOL_C64
    for t in idx:
        psi = statevector.simulate(circ, lists[t])
        o = criteria.score(circ.criterion, psi)
        if flags_comparable(circ.criterion, o, psi):
            assert score[t] == o


def test_brickwork16_streaming_parity(arso):
    circ = C.brickwork(16, 40, seed=0)
    cc = arso.compile_circuit(circ.n, circ.gates)
    T = 8
    p = 1e-3
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, 0, T)
    lists = sampling.sample(0, 0, T, circ.L, p / 3, p / 3, p / 3)
    score = np.zeros(T)
    arso.run_trajectories(cc, errs, circ.criterion, score)
    psi_ref = statevector.simulate(circ)
    got = gpu_states(arso, circ, cc, errs, 0, T)
    for t in range(T):
        psi = statevector.simulate(circ, lists[t]) if lists[t] else psi_ref
        assert np.max(np.abs(got[t] - psi)) < AMP_TOL_C64
        assert abs(score[t] - criteria.score(circ.criterion, psi, psi_ref)) < SCORE_TOL


def test_brickwork24_full_size_launch(arso):
    """Brickwork at 24 qubits in the benchmark's launch configuration: the
    depth-2 circuit is checked against the oracle amplitude by amplitude; the
    depth-40 circuit through properties that hold at any size."""
    circ = C.brickwork(24, 2, seed=0)
    cc = arso.compile_circuit(24, circ.gates, tile_qubits=14)
    lists = [[], [(3, 1), (40, 3)], [(circ.L - 1, 2)]]
    errs = arso.error_list_from_host(cc, lists)
    out = torch.empty((1, 1 << 24), dtype=torch.complex64, device="cuda")
    for t, ev in enumerate(lists):
        arso.trajectory_states(cc, errs, t, 1, out)
        psi = statevector.simulate(circ, ev)
        assert torch.max(torch.abs(out[0].cpu() - torch.from_numpy(psi))).item() < AMP_TOL_C64
    full = C.brickwork24(0)
    cc = arso.compile_circuit(24, full.gates, tile_qubits=12)  # the benchmark's tile shape
    T = 64
    p = 1e-3
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 0, 0, T)
    off, ev = arso.error_list_copy(errs)
    o_off, o_ev = oracle_csr(sampling.sample(0, 0, T, full.L, p / 3, p / 3, p / 3))
    assert np.array_equal(off, o_off) and np.array_equal(ev, o_ev)
    score = np.zeros(T)
    arso.run_trajectories(cc, errs, full.criterion, score)
    assert np.all(score >= -1e-6) and np.all(score <= 1 + 1e-5)
    err_free = np.diff(off.astype(np.int64)) == 0
    assert np.all(np.abs(score[err_free] - 1.0) < 1e-5)
    states = torch.empty((2, 1 << 24), dtype=torch.complex64, device="cuda")
    arso.trajectory_states(cc, errs, 0, 2, states)
    norms = torch.sum(torch.abs(states.to(torch.complex128)) ** 2, dim=1).cpu().numpy()
    assert np.all(np.abs(norms - 1.0) < 1e-4)


@pytest.fixture(scope="module")
def brickwork24_single_errors():
    """Oracle fidelities of brickwork-24 trajectories whose errors all follow one of
    the first 63 gates. For a Pauli P after gate g the rest of the circuit U is
    unitary and psi_R = U psi_g, so the fidelity is |<psi_g|P|psi_g>|^2; with P1
    after g1 and P2 after g2 it is |<psi_g2|P2 V P1|psi_g1>|^2, V the gates between.
    Locations: X after the SU(2) gate 40, Y after gate 44, Y on the first qubit of
    the CZ gate 60, Z on the second qubit of the CZ gate 62, and X at 40 with Z at 62."""
    full = C.brickwork24(0)
    n = full.n
    table = statevector.location_table(full)
    gates_of = {g: [l for l, (gg, _) in enumerate(table) if gg == g] for g in (40, 44, 60, 62)}
    x40, y44, y60, z62 = ((gates_of[40][0], 1), (gates_of[44][0], 3), (gates_of[60][0], 3), (gates_of[62][1], 2))
    cases = [[x40], [y44], [y60], [z62], [x40, z62]]
    psi = statevector.zero_state(n)
    snap = {}
    for g in range(63):
        statevector.apply_gate(psi, n, full.gates[g])
        if g in gates_of:
            snap[g] = psi.copy()

    def pauli(state, ev):
        out = state.copy()
        statevector.apply_pauli(out, n, table[ev[0]][1], ev[1])
        return out

    def single(ev):
        g = table[ev[0]][0]
        return abs(np.vdot(snap[g], pauli(snap[g], ev))) ** 2

    expected = [single(x40), single(y44), single(y60), single(z62)]
    branch = pauli(snap[40], x40)
    for g in range(41, 63):
        statevector.apply_gate(branch, n, full.gates[g])
    expected.append(abs(np.vdot(snap[62], pauli(branch, z62))) ** 2)
    return full, cases, np.array(expected)


@pytest.mark.parametrize("tile", [12, 13])
@pytest.mark.parametrize("suffix_reuse", [True, False])
def test_brickwork24_full_depth_against_oracle(arso, brickwork24_single_errors, suffix_reuse, tile):
    """Brickwork-24 depth 40 in the benchmark's launch configuration (12-qubit tiles;
    and the library default, 13; prefix cache): the GPU runs these trajectories
    through every pass after the first error (suffix reuse off) or stops after the
    last error's pass and scores against the cached error-free state there (on, as
    in the benchmark)."""
    full, cases, expected = brickwork24_single_errors
    assert np.all((expected[:4] > 0.05) & (expected[:4] < 0.95))  # entangled: neither 0 nor 1
    cc = arso.compile_circuit(full.n, full.gates, tile_qubits=tile,
                              flags=0 if suffix_reuse else arso.OPT_NO_SUFFIX_REUSE)
    errs = arso.error_list_from_host(cc, cases)
    score = np.zeros(len(cases))
    arso.run_trajectories(cc, errs, full.criterion, score)
    assert np.max(np.abs(score - expected)) < SCORE_TOL, (score, expected)


def test_grover12_reference_state_unbiased(arso):
    """60,771 gates, ~37k of them H or T: with a rounded 1/sqrt(2) the norm would
    drift by ~5e-4; the two-float constant keeps complex64 within 1e-5."""
    circ = C.grover12(0)
    cc = arso.compile_circuit(circ.n, circ.gates)
    out = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
    arso.reference_state(cc, out)
    got = out.cpu().numpy()
    psi = statevector.simulate(circ)
    assert np.max(np.abs(got - psi)) < AMP_TOL_C64
    assert abs(np.vdot(got, got).real - 1.0) < 1e-5


def test_graph_replay_equals_direct_launches(arso):
    """Small batches force many replays of captured pass sequences."""
    circ = C.brickwork(16, 16, seed=8)
    kw = dict(tile_qubits=11, max_batch=3)
    g = arso.compile_circuit(circ.n, circ.gates, **kw)
    d = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_GRAPHS, **kw)
    T, p = 40, 3e-3
    sg, sd = np.zeros(T), np.zeros(T)
    st = torch.cuda.Stream()  # the legacy default stream is never captured
    arso.run_trajectories(g, arso.sample_errors(g, p / 3, p / 3, p / 3, 4, 0, T, st), circ.criterion, sg, stream=st)
    arso.run_trajectories(d, arso.sample_errors(d, p / 3, p / 3, p / 3, 4, 0, T, st), circ.criterion, sd, stream=st)
    assert np.array_equal(sg, sd)
    # and the default stream (no capture) gives the same scores
    s0 = np.zeros(T)
    arso.run_trajectories(g, arso.sample_errors(g, p / 3, p / 3, p / 3, 4, 0, T), circ.criterion, s0)
    assert np.array_equal(s0, sd)


def test_autotune_returns_a_measured_candidate(arso):
    circ = C.brickwork(15, 8, seed=2)
    best, ms = arso.autotune(circ.n, circ.gates, circ.criterion, 1e-3, n_traj=16)
    assert len(ms) == 15 and np.all(ms > 0)
    assert 10 <= best["tile_qubits"] <= 14 and 3 <= best["low_qubits"] <= 5
    k = (best["tile_qubits"] - 10) * 3 + (best["low_qubits"] - 3)
    assert ms[k] == ms.min()


@pytest.mark.parametrize("n,depth", [(12, 20), (14, 12)])
def test_search_probe_reuse_is_exact(arso, n, depth):
    # probes of one search share their random numbers, so a trajectory with as
    # many events as at an earlier probe has the same events: reusing its score
    # must give exactly the search that simulates every trajectory (12 qubits:
    # resident engine, 14: streaming engine), with fewer amplitudes swept
    circ = C.brickwork(n, depth, 11)
    crit = C.Criterion("fidelity", threshold=0.9, aggregate="pass")
    cc = arso.compile_circuit(circ.n, circ.gates)
    kw = dict(n_traj=2000, seed=5, mode="mc", rel_tol=0.05, p_lo=1e-5, p_hi=1e-1)
    swept = {}
    res = {}
    for reuse in (False, True):
        arso.profile_reset()
        arso.profile_enable(True)
        res[reuse] = arso.tolerable_rate(cc, crit, 2 / 3, reuse=reuse, **kw)
        arso.profile_enable(False)
        swept[reuse] = sum(arso.profile_read(k).bytes for k in (arso.K_PASS, arso.K_PASS_LAST, arso.K_RESIDENT))
    a, b = res[False], res[True]
    assert a.converged and b.converged
    assert a.probes == b.probes and a.lo == b.lo and a.hi == b.hi
    assert a.value_lo == b.value_lo and a.value_hi == b.value_hi
    assert abs(a.p - b.p) <= 1e-12 * a.p
    assert swept[True] < 0.8 * swept[False]


@pytest.mark.parametrize("case", ["resident_c64", "resident_c128", "streaming_c64"])
def test_fast_exhaustive_matches_single_error_trajectories(arso, case):
    # the error-free sweep of Pauli expectations (fidelity = <psi_g|P|psi_g>^2)
    # against simulating every single-error state as a trajectory
    if case == "resident_c64":
        circ, kw, tol = C.brickwork(12, 10, 3), {}, AMP_TOL_C64
    elif case == "resident_c128":
        circ, kw, tol = C.qft4_0101(), {"precision": arso.C128}, AMP_TOL_C128
    else:
        circ, kw, tol = C.brickwork(14, 8, 4), {"tile_qubits": 10}, AMP_TOL_C64
    crit = C.Criterion("fidelity", threshold=0.9, aggregate="mean")
    fast = arso.compile_circuit(circ.n, circ.gates, **kw)
    slow = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_FAST_EXHAUSTIVE, **kw)
    Pf, per_f = arso.exhaustive(fast, crit)
    Ps, per_s = arso.exhaustive(slow, crit)
    assert per_f.shape == (3 * circ.L,)
    assert np.max(np.abs(per_f - per_s)) < 10 * tol
    assert np.max(np.abs(Pf - Ps)) < 10 * tol


def test_fast_exhaustive_streaming_matches_oracle(arso):
    circ = C.brickwork(14, 4, 5)
    crit = C.Criterion("fidelity", threshold=0.5, aggregate="mean")
    circ.criterion = crit
    cc = arso.compile_circuit(circ.n, circ.gates, tile_qubits=10)
    P, per = arso.exhaustive(cc, crit)
    a = ox.analyse(circ)
    assert abs(P[0] - a["P_R"]) < SCORE_TOL
    for k, e in enumerate(("X", "Z", "Y")):
        assert abs(P[1 + k] - a["P_e"][e]) < SCORE_TOL
        assert np.max(np.abs(per[k * circ.L:(k + 1) * circ.L] - a["per_location"][e])) < SCORE_TOL


def test_fast_exhaustive_streaming_every_gate_kind(arso):
    # every gate class (identity, X, diagonal, dense one-qubit, CX, SWAP, diagonal and
    # dense two-qubit) through the fused gate-and-expectation HBM kernel
    circ = C.random_circuit(14, 60, 9)
    crit = C.Criterion("fidelity", threshold=0.5, aggregate="mean")
    circ.criterion = crit
    names = {g.name for g in circ.gates}
    assert {"ID", "X", "CX", "SWAP", "U2", "CP", "U"} <= names
    cc = arso.compile_circuit(circ.n, circ.gates, tile_qubits=10)
    P, per = arso.exhaustive(cc, crit)
    a = ox.analyse(circ)
    for k, e in enumerate(("X", "Z", "Y")):
        assert np.max(np.abs(per[k * circ.L:(k + 1) * circ.L] - a["per_location"][e])) < SCORE_TOL


@pytest.mark.parametrize("n,kw", [(10, {}), (14, {"tile_qubits": 10})])
def test_quantum_volume_heavy_output_scores(arso, n, kw):
    # QV circuits (Haar U(4) layers, dense two-qubit gates) scored by binning on
    # the heavy outputs of their ideal distribution, per trajectory against the oracle
    circ = C.quantum_volume(n, 7)
    heavy = criteria.heavy_outputs(statevector.simulate(circ, []))
    crit = C.Criterion("binning", basis_set=heavy.tolist(), threshold=2 / 3, aggregate="mean")
    cc = arso.compile_circuit(n, circ.gates, **kw)
    T, p = 6, 3e-2
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 5, 0, T)
    got = np.zeros(T)
    arso.run_trajectories(cc, errs, crit, got)
    lists = sampling.sample(5, 0, T, circ.L, p / 3, p / 3, p / 3)
    for t in range(T):
        want = criteria.score(crit, statevector.simulate(circ, lists[t]))
        assert abs(got[t] - want) < SCORE_TOL


@pytest.mark.parametrize("family", ["bv", "hlf", "ryrz", "uccsd", "ryrz_streaming"])
def test_paper_families_scores(arso, family):
    # the paper's remaining circuit families, per trajectory against the oracle
    kw = {}
    if family == "bv":
        circ = C.bernstein_vazirani(11, 0b1011001101)
    elif family == "hlf":
        circ = C.hidden_linear_function(10, 2)
    elif family == "ryrz":
        circ = C.ryrz_ansatz(10, 3, 4)
    elif family == "uccsd":
        circ = C.uccsd_ansatz(8, 4, 5)
    else:
        circ, kw = C.ryrz_ansatz(14, 2, 6), {"tile_qubits": 10}
    cc = arso.compile_circuit(circ.n, circ.gates, **kw)
    T, p = 5, 1e-2
    errs = arso.sample_errors(cc, p / 3, p / 3, p / 3, 9, 0, T)
    got = np.zeros(T)
    arso.run_trajectories(cc, errs, circ.criterion, got)
    ref = statevector.simulate(circ, [])
    lists = sampling.sample(9, 0, T, circ.L, p / 3, p / 3, p / 3)
    for t in range(T):
        want = criteria.score(circ.criterion, statevector.simulate(circ, lists[t]), ref)
        assert abs(got[t] - want) < SCORE_TOL


@pytest.mark.parametrize("n,kw", [(12, {}), (16, {"tile_qubits": 12})])
def test_split_trajectory_ranges_are_bit_identical(arso, n, kw):
    # the sharding contract on one GPU: error draws depend only on (seed,
    # trajectory id, location), so scoring [0, T) in one call or as two ranks'
    # contiguous ranges gives the same score for every trajectory, bit for bit
    circ = C.brickwork(n, 12, 21)
    crit = C.Criterion("fidelity", threshold=0.9, aggregate="pass")
    cc = arso.compile_circuit(circ.n, circ.gates, **kw)
    T, p, seed = 600, 2e-3, 13
    whole = np.zeros(T)
    arso.run_trajectories(cc, arso.sample_errors(cc, p / 3, p / 3, p / 3, seed, 0, T), crit, whole)
    parts = []
    for begin, count in ((0, 257), (257, T - 257)):
        s = np.zeros(count)
        arso.run_trajectories(cc, arso.sample_errors(cc, p / 3, p / 3, p / 3, seed, begin, count), crit, s)
        parts.append(s)
    assert np.array_equal(np.concatenate(parts), whole)


# ---------------------- outcome probability: backward states (Eq. (3), Eq. (4)) ---

def _outcome_case(arso, case):
    """(circuit with an outcome criterion, compile kwargs, tolerance)."""
    if case == "adder_resident_c64":
        circ, kw, tol = C.cuccaro_adder(4, 11, 6), {}, SCORE_TOL
    elif case == "adder_resident_c128":
        circ, kw, tol = C.cuccaro_adder(2, 3, 2), {"precision": arso.C128}, 1e-12
    elif case == "random_resident_c64":
        circ, kw, tol = C.random_circuit(9, 90, 21), {}, SCORE_TOL
    elif case == "random_resident_c128":
        circ, kw, tol = C.random_circuit(7, 90, 22), {"precision": arso.C128}, 1e-12
    elif case == "bv_streaming":
        circ, kw, tol = C.bernstein_vazirani(15, 0b10110011010101), {"tile_qubits": 10}, SCORE_TOL
    else:  # random_streaming: every gate kind through the HBM backward kernel
        circ, kw, tol = C.random_circuit(14, 40, 9), {"tile_qubits": 10}, SCORE_TOL
    if case.startswith("random"):
        psi = statevector.simulate(circ)
        circ.criterion = C.Criterion("outcome", target=int(np.argmax(np.abs(psi))), threshold=0.5, aggregate="mean")
    else:
        circ.criterion = C.Criterion("outcome", target=circ.criterion.target, threshold=0.5, aggregate="mean")
    return circ, kw, tol


@pytest.mark.parametrize("case", ["adder_resident_c64", "adder_resident_c128", "random_resident_c64",
                                  "random_resident_c128", "bv_streaming", "random_streaming"])
def test_fast_outcome_exhaustive_matches_oracle(arso, case):
    # the backward sweep scores the single-error state with P after gate g as
    # |<phi_g|P|psi_g>|^2 (phi_g = W^dagger |t>); the oracle simulates every such state
    circ, kw, tol = _outcome_case(arso, case)
    crit = circ.criterion
    cc = arso.compile_circuit(circ.n, circ.gates, **kw)
    P, per = arso.exhaustive(cc, crit)
    a = ox.analyse(circ)
    assert abs(P[0] - a["P_R"]) < tol
    for k, e in enumerate(("X", "Z", "Y")):
        assert abs(P[1 + k] - a["P_e"][e]) < tol, e
        assert np.max(np.abs(per[k * circ.L:(k + 1) * circ.L] - a["per_location"][e])) < tol, e


@pytest.mark.parametrize("case", ["adder_resident_c64", "random_streaming"])
def test_fast_outcome_exhaustive_matches_single_error_trajectories(arso, case):
    circ, kw, tol = _outcome_case(arso, case)
    fast = arso.compile_circuit(circ.n, circ.gates, **kw)
    slow = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_FAST_EXHAUSTIVE, **kw)
    Pf, per_f = arso.exhaustive(fast, circ.criterion)
    Ps, per_s = arso.exhaustive(slow, circ.criterion)
    assert np.max(np.abs(per_f - per_s)) < 10 * tol
    assert np.max(np.abs(Pf - Ps)) < 10 * tol


def test_fast_outcome_exhaustive_streaming_adder(arso):
    # a 14-qubit Clifford+T adder on the streaming engine: backward sweep against
    # simulating all 3L single-error states as trajectories
    circ = C.cuccaro_adder(6, 45, 17)
    crit = C.Criterion("outcome", target=circ.criterion.target, threshold=0.5, aggregate="mean")
    fast = arso.compile_circuit(circ.n, circ.gates, tile_qubits=10)
    slow = arso.compile_circuit(circ.n, circ.gates, tile_qubits=10, flags=arso.OPT_NO_FAST_EXHAUSTIVE)
    Pf, per_f = arso.exhaustive(fast, crit)
    Ps, per_s = arso.exhaustive(slow, crit)
    assert np.max(np.abs(per_f - per_s)) < 10 * SCORE_TOL
    assert np.max(np.abs(Pf - Ps)) < 10 * SCORE_TOL
    assert abs(Pf[0] - 1.0) < SCORE_TOL  # the error-free adder reaches its sum with certainty


@pytest.mark.parametrize("cache_boundaries", [0, 4])
def test_outcome_suffix_reuse_scores_equal_full_runs(arso, cache_boundaries):
    """Outcome probability taken right after the last error as the overlap with the
    backward state W^dagger |t> at that boundary equals the full run's |<t|psi>|^2."""
    circ = C.cuccaro_adder(7, 101, 77)  # 16 qubits
    sb = (1 << circ.n) * 8
    kw = dict(tile_qubits=11, cache_bytes=cache_boundaries * sb)
    on = arso.compile_circuit(circ.n, circ.gates, **kw)
    off = arso.compile_circuit(circ.n, circ.gates, flags=arso.OPT_NO_SUFFIX_REUSE, **kw)
    assert on.info().n_passes > 3
    T, p = 64, 3e-3
    s_on, s_off = np.zeros(T), np.zeros(T)
    f_on, f_off = np.zeros(T, np.uint8), np.zeros(T, np.uint8)
    arso.run_trajectories(on, arso.sample_errors(on, p / 3, p / 3, p / 3, 4, 0, T), circ.criterion, s_on, f_on)
    arso.run_trajectories(off, arso.sample_errors(off, p / 3, p / 3, p / 3, 4, 0, T), circ.criterion, s_off, f_off)
    assert np.max(np.abs(s_on - s_off)) < SCORE_TOL
    away = np.abs(s_off - circ.criterion.threshold) > SCORE_TOL
    assert np.array_equal(f_on[away], f_off[away])
    lists = sampling.sample(4, 0, T, circ.L, p / 3, p / 3, p / 3)
    errored = [i for i in range(T) if lists[i]]
    assert len(errored) > 10
    for t in errored[:3]:
        o = criteria.score(circ.criterion, statevector.simulate(circ, lists[t]))
        assert abs(s_on[t] - o) < SCORE_TOL
