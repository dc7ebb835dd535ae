"""Tensor-core phases (ARSO_OPT_TENSOR_PHASES): a phase's gates on its five
register bits fused into one 32 x 32 unitary and applied to the tile as an
FP16-split contraction with FP32 accumulation. Checked against the FP64 oracle
(amplitudes within 1e-5 max-abs, scores within 1e-5) and against the same
circuits run gate by gate, on every tile size the route takes (12-14 qubits),
on circuits whose phases hold every gate class, and with Pauli errors inside,
before and after tensor phases."""
import numpy as np
import pytest

from oracle import criteria, statevector
from workloads import circuits as C

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

AMP_TOL_C64 = 1e-5
SCORE_TOL = 1e-5

CASES = {
    "brickwork16_t13": (lambda: C.brickwork(16, 12, 3), 13),
    "brickwork15_t12": (lambda: C.brickwork(15, 10, 4), 12),
    "brickwork17_t14": (lambda: C.brickwork(17, 8, 5), 14),
    "random16_t13": (lambda: C.random_circuit(16, 300, 6), 13),
    "qaoa16_t13": (lambda: C.qaoa_maxcut(16, 2), 13),
    "qft15_t13": (lambda: C.qft_basis(15, 12345), 13),
}


@pytest.fixture(scope="module")
def arso():
    from paper_2301_07264_gb300 import arso as mod
    assert torch.cuda.is_available()
    return mod


def _compile(arso, circ, tile, tensor):
    cc = arso.compile_circuit(circ.n, circ.gates, tile_qubits=tile,
                              flags=arso.OPT_TENSOR_PHASES if tensor else 0)
    info = cc.info()
    assert info.engine == 1
    if tensor:
        assert info.tensor_phases > 0
    else:
        assert info.tensor_phases == 0
    return cc


def _error_lists(circ, T, seed, max_err=3):
    rng = np.random.default_rng(seed)
    lists = [[]]
    lists.append([(0, 1)])                  # an X error on the first location: the mask is set from the start
    lists.append([(circ.L - 1, 3)])         # a Y error on the last location
    while len(lists) < T:
        k = int(rng.integers(1, max_err + 1))
        locs = sorted(rng.choice(circ.L, size=k, replace=False).tolist())
        lists.append([(int(l), int(rng.integers(1, 4))) for l in locs])
    return lists


def _states(arso, circ, cc, errs, count):
    out = torch.empty((count, 1 << circ.n), dtype=torch.complex64, device="cuda")
    arso.trajectory_states(cc, errs, 0, count, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", sorted(CASES))
def test_tensor_amplitudes_match_oracle(arso, case):
    make, tile = CASES[case]
    circ = make()
    cc = _compile(arso, circ, tile, True)
    lists = _error_lists(circ, 6, 11)
    errs = arso.error_list_from_host(cc, lists)
    got = _states(arso, circ, cc, errs, len(lists))
    for t, ev in enumerate(lists):
        ref = statevector.simulate(circ, ev)
        assert np.max(np.abs(got[t] - ref)) < AMP_TOL_C64, (case, t)
        assert abs(np.vdot(got[t], got[t]).real - 1.0) < 1e-5, (case, t)


@pytest.mark.parametrize("case", sorted(CASES))
def test_tensor_scores_match_gate_by_gate_and_oracle(arso, case):
    """Per-trajectory scores of sampled trajectories: the tensor route against
    the gate-by-gate route on the same error lists, and a sample against the
    oracle."""
    make, tile = CASES[case]
    circ = make()
    ct = _compile(arso, circ, tile, True)
    cf = _compile(arso, circ, tile, False)
    p, T = 2e-3, 400
    et = arso.sample_errors(ct, p / 3, p / 3, p / 3, 21, 0, T)
    ef = arso.sample_errors(cf, p / 3, p / 3, p / 3, 21, 0, T)
    st, sf = np.zeros(T), np.zeros(T)
    arso.run_trajectories(ct, et, circ.criterion, st)
    arso.run_trajectories(cf, ef, circ.criterion, sf)
    assert np.max(np.abs(st - sf)) < SCORE_TOL, case
    from oracle import sampling
    lists = sampling.sample(21, 0, 12, circ.L, p / 3, p / 3, p / 3)
    psi_r = statevector.simulate(circ)
    for t in range(12):
        psi = statevector.simulate(circ, lists[t]) if lists[t] else psi_r
        assert abs(st[t] - criteria.score(circ.criterion, psi, psi_r)) < SCORE_TOL, (case, t)


def test_tensor_brickwork20_error_free_and_suffix_reuse(arso):
    """psi_R of a 20-qubit brickwork circuit (the error-free sweep runs every
    tensor phase) against the oracle, and scores with suffix reuse on and off."""
    circ = C.brickwork(20, 16, 9)
    cc = _compile(arso, circ, 13, True)
    ref = torch.empty(1 << circ.n, dtype=torch.complex64, device="cuda")
    arso.reference_state(cc, ref)
    torch.cuda.synchronize()
    psi = statevector.simulate(circ)
    assert np.max(np.abs(ref.cpu().numpy() - psi)) < AMP_TOL_C64
    cn = arso.compile_circuit(circ.n, circ.gates, tile_qubits=13,
                              flags=arso.OPT_TENSOR_PHASES | arso.OPT_NO_SUFFIX_REUSE)
    p, T = 1e-3, 200
    a, b = np.zeros(T), np.zeros(T)
    arso.run_trajectories(cc, arso.sample_errors(cc, p / 3, p / 3, p / 3, 4, 0, T), circ.criterion, a)
    arso.run_trajectories(cn, arso.sample_errors(cn, p / 3, p / 3, p / 3, 4, 0, T), circ.criterion, b)
    assert np.max(np.abs(a - b)) < SCORE_TOL


def test_tensor_outcome_criterion(arso):
    """Outcome probabilities of a streaming adder through tensor phases against
    the oracle (the scoring pass reads the backward states)."""
    circ = C.cuccaro_adder(7, 101, 77)
    cc = _compile(arso, circ, 13, True)
    lists = _error_lists(circ, 5, 3)
    errs = arso.error_list_from_host(cc, lists)
    s = np.zeros(len(lists))
    arso.run_trajectories(cc, errs, circ.criterion, s)
    psi_r = statevector.simulate(circ)
    for t, ev in enumerate(lists):
        psi = statevector.simulate(circ, ev)
        assert abs(s[t] - criteria.score(circ.criterion, psi, psi_r)) < SCORE_TOL, t
