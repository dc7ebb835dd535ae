"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (Eq. (2) and the XX example, tests/golden/), published
known-answer vectors (Philox), closed forms (QFT of a basis state, Grover's
sin^2((2k+1)theta), the one-qubit depolarising fidelity), invariants (norm,
unitarity, Pauli commutation), two independent exact expectations (density
matrix, brute-force enumeration) and the algebra of Eq. (4)/(5).
"""
import cmath
import math
import os

import numpy as np
import pytest

from oracle import criteria, density, exhaustive, montecarlo, philox, sampling, search, statevector
from oracle.gates import matrix_of
from workloads import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ---

def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(w, 16) for w in line.split()])
    return rows


def test_philox_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = philox.philox4x32(r[0], r[1], r[2], r[3], r[4], r[5])
        assert [int(w) for w in out] == r[6:10]


def test_philox_vectorised_matches_scalar():
    l = np.arange(50, dtype=np.uint64)
    v = philox.philox4x32(l, 7, 0, 3, 11, 13)
    for i in (0, 17, 49):
        s = philox.philox4x32(i, 7, 0, 3, 11, 13)
        assert all(int(a[i]) == int(b) for a, b in zip(v, s))


# ------------------------------------------------------------- Eq. (2) -----

def test_eq2_single_qubit_paulis_match_paper():
    a0, a1 = 0.6 + 0.1j, -0.3 + 0.7j
    expect = {1: (a1, a0), 2: (a0, -a1), 3: (-1j * a1, 1j * a0)}
    for code, (e0, e1) in expect.items():
        psi = np.array([a0, a1])
        statevector.apply_pauli(psi, 1, 0, code)
        assert psi[0] == pytest.approx(e0, abs=0) and psi[1] == pytest.approx(e1, abs=0)


def test_eq2_golden_fixture_and_xx_example():
    rows = {}
    with open(os.path.join(GOLDEN, "eq2_pauli.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = parts[1:]
    coef = {"1": 1, "-1": -1, "i": 1j, "-i": -1j}
    a = np.array([0.1 + 0.2j, 0.3 - 0.1j, -0.5 + 0.4j, 0.2 + 0.6j])
    for name, code in (("X", 1), ("Z", 2), ("Y", 3)):
        psi = a[:2].copy()
        statevector.apply_pauli(psi, 1, 0, code)
        for k, tok in enumerate(rows[name]):
            c, src = tok.split(":")
            assert psi[k] == coef[c] * a[int(src[1])]
    psi = a.copy()
    statevector.apply_pauli(psi, 2, 0, 1)
    statevector.apply_pauli(psi, 2, 1, 1)
    for k, tok in enumerate(rows["XX"]):
        c, src = tok.split(":")
        assert psi[k] == coef[c] * a[int(src[1])]


def test_pauli_codes_agree_with_textbook_matrices():
    rng = np.random.default_rng(3)
    for n in (1, 3):
        for q in range(n):
            psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
            for code, name in ((1, "X"), (2, "Z"), (3, "Y")):
                a = psi.copy()
                statevector.apply_pauli(a, n, q, code)
                b = psi.copy()
                statevector.apply_gate(b, n, C.Gate(name, (q,)))
                assert np.allclose(a, b, atol=0, rtol=0)


# --------------------------------------------------- gates & closed forms --

@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_qft_of_basis_states_closed_form(n):
    for x in range(1 << n):
        psi = statevector.simulate(C.qft_basis(n, x))
        y = np.arange(1 << n)
        expect = np.exp(2j * math.pi * x * y / (1 << n)) / math.sqrt(1 << n)
        assert np.max(np.abs(psi - expect)) < 1e-13


def test_qft4_0101_counts():
    c = C.qft4_0101()
    assert (c.G, c.k, c.m, c.L) == (18, 6, 12, 30)


@pytest.mark.parametrize("n", [2, 3, 6])
def test_ghz_amplitudes(n):
    psi = statevector.simulate(C.ghz(n))
    expect = np.zeros(1 << n, dtype=complex)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - expect)) < 1e-15


def test_norm_preserved_every_gate():
    c = C.random_circuit(5, 200, seed=4)
    psi = statevector.zero_state(5)
    for g in c.gates:
        statevector.apply_gate(psi, 5, g)
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-14


def test_unitarity_u_then_udagger():
    c = C.random_circuit(4, 120, seed=5)
    psi = statevector.simulate(c)
    inv = []
    for g in reversed(c.gates):
        M = matrix_of(g).conj().T
        inv.append(C.Gate("U" if g.arity == 1 else "U2", g.qubits, (), M))
    back = statevector.simulate(C.Circuit(4, inv), psi0=psi)
    assert np.max(np.abs(back - statevector.zero_state(4))) < 1e-13


def test_two_qubit_local_index_convention():
    # CX(control=0, target=1) on |q0=1,q1=0> (index 1) gives |q0=1,q1=1> (index 3)
    c = C.Circuit(2, [C.Gate("X", (0,)), C.Gate("CX", (0, 1))])
    psi = statevector.simulate(c)
    assert abs(psi[3] - 1) < 1e-15
    c = C.Circuit(3, [C.Gate("X", (2,)), C.Gate("CX", (2, 0))])
    assert abs(statevector.simulate(c)[5] - 1) < 1e-15


def test_toffoli_and_borrowed_mcx_are_exact_permutations():
    for x in range(8):
        psi = statevector.simulate(C.Circuit(3, C.basis_prep(3, x) + C.toffoli_clifford_t(0, 1, 2)))
        assert abs(psi[x ^ 4 if (x & 3) == 3 else x] - 1) < 1e-12
    rng = np.random.default_rng(1)
    for m in range(3, 8):
        n = m + 2
        for _ in range(6):
            x = int(rng.integers(1 << n))
            psi = statevector.simulate(C.Circuit(n, C.basis_prep(n, x) + C.mcx(range(m), m, [m + 1])))
            full = (x & ((1 << m) - 1)) == (1 << m) - 1
            assert abs(psi[x ^ (1 << m) if full else x] - 1) < 1e-10


def test_adder_outcome_is_sum():
    for bits in (1, 2, 3):
        for a in range(1 << bits):
            for b in range(1 << bits):
                c = C.cuccaro_adder(bits, a, b)
                assert abs(abs(statevector.simulate(c)[c.criterion.target]) ** 2 - 1) < 1e-10


@pytest.mark.parametrize("ns", [3, 5])
def test_grover_success_closed_form_every_k(ns):
    theta = math.asin(2.0 ** (-ns / 2))
    kstar = int(math.floor(math.pi / (4 * theta)))
    for k in range(kstar + 1):
        c = C.grover(ns, marked=5 % (1 << ns), iterations=k)
        psi = statevector.simulate(c)
        assert abs(abs(psi[c.meta["marked"]]) ** 2 - math.sin((2 * k + 1) * theta) ** 2) < 1e-12


@pytest.mark.slow
def test_grover12_success_closed_form():
    c = C.grover12(0)
    psi = statevector.simulate(c)
    th, k = c.meta["theta"], c.meta["iterations"]
    assert k == 35
    assert abs(abs(psi[c.meta["marked"]]) ** 2 - math.sin((2 * k + 1) * th) ** 2) < 1e-11


# ---------------------------------------------------- Pauli commutation ----

def _with_error(gates, n, l, code):
    return statevector.simulate(C.Circuit(n, gates), [(l, code)])


def test_pauli_commutation_through_gates():
    # Error after the ID equals (before H) vs after H. H X = Z H, H Z = X H, H Y = -Y H.
    g = [C.Gate("ID", (0,)), C.Gate("H", (0,))]
    for before, after, sign in ((1, 2, 1), (2, 1, 1), (3, 3, -1)):
        a = _with_error(g, 1, 0, before)
        b = _with_error(g, 1, 1, after)
        assert np.allclose(a, sign * b, atol=1e-15)
    # CX (X on control) = (X x X) CX ; CX (Z on target) = (Z x Z) CX. Start from a
    # generic state so that no identity holds by accident.
    rng = np.random.default_rng(7)
    v = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    v /= np.linalg.norm(v)
    pre = [C.Gate("U2", (0, 1), (), np.diag(v / np.abs(v))), C.Gate("ID", (0,)), C.Gate("ID", (1,))]
    gates = pre + [C.Gate("CX", (0, 1))]
    # with the two leading H: locations 0,1 -> H; 2,3 -> U2; 4 -> ID q0; 5 -> ID q1;
    # 6 -> CX q0; 7 -> CX q1
    a = statevector.simulate(C.Circuit(2, [C.Gate("H", (0,)), C.Gate("H", (1,))] + gates), [(4, 1)])
    b = statevector.simulate(C.Circuit(2, [C.Gate("H", (0,)), C.Gate("H", (1,))] + gates), [(6, 1), (7, 1)])
    assert np.allclose(a, b, atol=1e-14)
    a = statevector.simulate(C.Circuit(2, [C.Gate("H", (0,)), C.Gate("H", (1,))] + gates), [(5, 2)])
    b = statevector.simulate(C.Circuit(2, [C.Gate("H", (0,)), C.Gate("H", (1,))] + gates), [(6, 2), (7, 2)])
    assert np.allclose(a, b, atol=1e-14)


# ------------------------------------------------------------- sampling ----

def test_sampling_nested_in_p_and_types_fixed():
    L = 500
    e1 = dict(sampling.sample_trajectory(9, 3, L, 1e-2 / 3, 1e-2 / 3, 1e-2 / 3))
    e2 = dict(sampling.sample_trajectory(9, 3, L, 5e-2 / 3, 5e-2 / 3, 5e-2 / 3))
    assert set(e1) <= set(e2)
    assert all(e1[l] == e2[l] for l in e1)


def test_sampling_rates_and_type_split():
    L, T = 2000, 60
    p = 0.03
    counts = np.zeros(4)
    for t in range(T):
        for _, code in sampling.sample_trajectory(1, t, L, p / 3, p / 3, p / 3):
            counts[code] += 1
    n = L * T
    tot = counts.sum()
    assert abs(tot - n * p) < 5 * math.sqrt(n * p * (1 - p))
    for c in (1, 2, 3):
        assert abs(counts[c] - tot / 3) < 5 * math.sqrt(tot * (1 / 3) * (2 / 3))


def test_sampling_thresholds_edge_cases():
    assert sampling.thresholds(0, 0, 0) == (0, 0, 0)
    thr, cx, cxz = sampling.thresholds(1.0, 0.0, 0.0)
    assert thr == 2 ** 32 - 1 and cx == 2 ** 32 and cxz == 2 ** 32
    thr, cx, cxz = sampling.thresholds(0.0, 0.0, 0.5)
    assert thr == 2 ** 31 and cx == 0 and cxz == 0
    assert sampling.sample_trajectory(0, 0, 100, 0, 0, 0) == []
    ev = sampling.sample_trajectory(0, 0, 100, 0.0, 0.0, 1.0)
    assert [l for l, _ in ev] == list(range(100)) and all(c == 3 for _, c in ev)


def test_sampling_uses_both_halves_of_a_philox_block():
    # locations 2j and 2j+1 share the counter (j, t, 0, stream): draws must be
    # the (w0,w1) and (w2,w3) halves of the same block
    wa, wb = sampling.draws(5, 11, 6)
    w = philox.philox4x32(1, 11, 0, sampling.STREAM_ERRORS, 5, 0)
    assert int(wa[2]) == int(w[0]) and int(wb[2]) == int(w[1])
    assert int(wa[3]) == int(w[2]) and int(wb[3]) == int(w[3])


# ---------------------------------------------------- exhaustive / Eq. 3 --

def test_eq3_state_count():
    c = C.random_circuit(3, 25, seed=2)
    states = list(exhaustive.single_error_states(c))
    assert len(states) == 3 * (c.k + 2 * c.m)


def test_ghz_single_error_scores_are_stabiliser_exact():
    c = C.ghz(4)
    a = exhaustive.analyse(c)
    for e, v in a["per_location"].items():
        assert np.all((np.abs(v) < 1e-12) | (np.abs(v - 1) < 1e-12)), e
    # X right after the first H (location 0) on |+>: fidelity 1; Z there: 0.
    assert a["per_location"]["X"][0] == pytest.approx(1, abs=1e-12)
    assert a["per_location"]["Z"][0] == pytest.approx(0, abs=1e-12)


def _small_circuits():
    return [
        C.ghz(3),
        C.Circuit(2, [C.Gate("H", (0,)), C.Gate("CX", (0, 1)), C.Gate("T", (1,)), C.Gate("H", (1,))],
                  criterion=C.Criterion("fidelity")),
        C.Circuit(3, [C.Gate("H", (0,)), C.Gate("RY", (1,), (0.7,)), C.Gate("CZ", (0, 1)),
                      C.Gate("RX", (2,), (1.1,))], criterion=C.Criterion("outcome", target=0)),
        C.Circuit(2, [C.Gate("H", (0,)), C.Gate("H", (1,)), C.Gate("CP", (0, 1), (0.9,)),
                      C.Gate("SDG", (1,))], criterion=C.Criterion("binning", basis_set=(0, 3))),
    ]


def test_density_matrix_equals_bruteforce_enumeration():
    from oracle import enumerate as bf
    for c in _small_circuits():
        assert c.L <= 8
        for (px, pz, py) in ((0.01, 0.02, 0.005), (0.1, 0.1, 0.1)):
            psi_ref = statevector.simulate(c)
            rho = density.evolve(c, px, pz, py)
            d = density.expected_score(c, rho, psi_ref)
            e, _ = bf.expectation(c, px, pz, py)
            assert abs(d - e) < 1e-12


@pytest.mark.parametrize("G", [1, 5, 40])
def test_identity_chain_closed_form(G):
    c = C.identity_chain(G)
    p = 0.03
    exact = (1 + (1 - 4 * p / 3) ** G) / 2
    rho = density.evolve(c, p / 3, p / 3, p / 3)
    assert abs(density.expected_score(c, rho, statevector.simulate(c)) - exact) < 1e-13
    if G <= 5:
        from oracle import enumerate as bf
        assert abs(bf.expectation(c, p / 3, p / 3, p / 3)[0] - exact) < 1e-13


def test_eq4_is_first_order_expansion_of_exact_model():
    for c in _small_circuits():
        a = exhaustive.analyse(c)
        psi_ref = statevector.simulate(c)
        slope_eq4 = (exhaustive.eq4(a, 1 / 3, 1 / 3, 1 / 3) - a["P_R"])
        for p in (1e-5, 1e-6):
            rho = density.evolve(c, p / 3, p / 3, p / 3)
            slope = (density.expected_score(c, rho, psi_ref) - a["P_R"]) / p
            assert abs(slope - slope_eq4) < 5 * c.L * c.L * p + 1e-7


def test_eq4_literal_gate_count_reading_differs_when_two_qubit_gates():
    c = C.ghz(3)
    a = exhaustive.analyse(c)
    assert exhaustive.eq4(a, 1e-3, 1e-3, 1e-3, "locations") != exhaustive.eq4(a, 1e-3, 1e-3, 1e-3, "gates")


def test_eq5_round_trip_and_g_inverse_bound():
    for seed in range(4):
        c = C.random_circuit(3, 12, seed=seed)
        a = exhaustive.analyse(c)
        P1 = exhaustive.one_error_success(a)
        if a["P_R"] - P1 < 1e-6:
            continue
        for P_target in (P1 + 0.3 * (a["P_R"] - P1), P1 + 0.9 * (a["P_R"] - P1)):
            p = exhaustive.eq5(a, P_target)
            assert abs(exhaustive.eq4(a, p / 3, p / 3, p / 3) - P_target) < 1e-12
            assert p < 1.0 / c.L  # Sec. IV-D: p < 1/L whenever P_target > P1


# ------------------------------------------------------- Monte Carlo ------

@pytest.mark.parametrize("idx", [0, 1, 2, 3])
def test_mc_mean_within_4sigma_of_exact(idx):
    c = _small_circuits()[idx]
    p = 0.08
    s, f, _ = montecarlo.run_trajectories(c, 3, 0, 3000, p / 3, p / 3, p / 3)
    agg = montecarlo.aggregate(s, f)
    exact = density.expected_score(c, density.evolve(c, p / 3, p / 3, p / 3), statevector.simulate(c))
    assert abs(agg["mean"] - exact) < 4 * agg["stderr_mean"] + 1e-12


def test_mc_pass_fraction_within_4sigma_of_enumeration():
    from oracle import enumerate as bf
    c = C.Circuit(2, [C.Gate("H", (0,)), C.Gate("CX", (0, 1)), C.Gate("T", (1,))],
                  criterion=C.Criterion("fidelity", threshold=0.9, aggregate="pass"))
    p = 0.1
    s, f, _ = montecarlo.run_trajectories(c, 5, 0, 3000, p / 3, p / 3, p / 3)
    agg = montecarlo.aggregate(s, f)
    _, e_pass = bf.expectation(c, p / 3, p / 3, p / 3)
    assert abs(agg["pass_frac"] - e_pass) < 4 * agg["stderr_pass"] + 1e-12


def test_mc_error_free_trajectories_score_reference():
    c = C.qft4_0101()
    s, f, errs = montecarlo.run_trajectories(c, 0, 0, 200, 1e-3 / 3, 1e-3 / 3, 1e-3 / 3)
    for sc, ev in zip(s, errs):
        if not ev:
            assert sc == pytest.approx(1.0, abs=1e-12)


def test_argmax_tie_lowest_index():
    crit = C.Criterion("argmax", target=1)
    psi = np.array([0.5, 0.5, 0.5, 0.5])
    assert criteria.score(crit, psi) == 0.0
    assert criteria.score(C.Criterion("argmax", target=0), psi) == 1.0


# ------------------------------------------ rotation and phase gates ------
# Textbook definitions (Nielsen & Chuang, Sec. 4.2): R_P(theta) = exp(-i theta P / 2)
# for P in {X, Y, Z}; the phase gate P(phi) = diag(1, e^{i phi}) = exp(i phi |1><1|),
# with S = P(pi/2), SDG = P(-pi/2), T = P(pi/4), TDG = P(-pi/4). scipy's expm is an
# independent route to the same matrices.

_SIGMA = {"X": np.array([[0, 1], [1, 0]], complex), "Y": np.array([[0, -1j], [1j, 0]], complex),
          "Z": np.array([[1, 0], [0, -1]], complex)}
_THETAS = (0.0, 0.3, -1.1, math.pi / 2, math.pi, 2.5, 2 * math.pi - 0.2)


def test_rotations_are_pauli_exponentials():
    from scipy.linalg import expm
    for axis in "XYZ":
        for th in _THETAS:
            got = matrix_of(C.Gate("R" + axis, (0,), (th,)))
            assert np.max(np.abs(got - expm(-0.5j * th * _SIGMA[axis]))) < 1e-14, (axis, th)
    # R_P(pi) = -i P
    for axis in "XYZ":
        assert np.allclose(matrix_of(C.Gate("R" + axis, (0,), (math.pi,))), -1j * _SIGMA[axis], atol=1e-15)


def test_phase_gates_are_projector_exponentials():
    from scipy.linalg import expm
    proj1 = np.array([[0, 0], [0, 1]], complex)
    for phi in _THETAS:
        got = matrix_of(C.Gate("P", (0,), (phi,)))
        assert np.max(np.abs(got - expm(1j * phi * proj1))) < 1e-14
        # RZ(phi) = e^{-i phi / 2} P(phi)
        rz = matrix_of(C.Gate("RZ", (0,), (phi,)))
        assert np.max(np.abs(rz - cmath.exp(-0.5j * phi) * got)) < 1e-14
    for name, phi in (("S", math.pi / 2), ("SDG", -math.pi / 2), ("T", math.pi / 4), ("TDG", -math.pi / 4)):
        assert np.max(np.abs(matrix_of(C.Gate(name, (0,))) - expm(1j * phi * proj1))) < 1e-14, name
    S, SDG, T = (matrix_of(C.Gate(k, (0,))) for k in ("S", "SDG", "T"))
    assert np.allclose(S @ S, _SIGMA["Z"], atol=1e-15)
    assert np.allclose(S @ SDG, np.eye(2), atol=1e-15)
    assert np.allclose(T @ T, S, atol=1e-15)


def test_rotation_gates_on_basis_states_closed_form():
    # through the state-vector update on a multi-qubit register: RX(t)|0> =
    # (cos t/2, -i sin t/2), RY(t)|0> = (cos t/2, sin t/2), RZ(t)|1> = e^{i t/2}|1>,
    # RY(pi/2)|0> = |+>, H RZ(t) H = RX(t)
    n = 3
    for q in range(n):
        for th in _THETAS:
            c, s = math.cos(th / 2), math.sin(th / 2)
            psi = statevector.simulate(C.Circuit(n, [C.Gate("RX", (q,), (th,))]))
            assert abs(psi[0] - c) < 1e-15 and abs(psi[1 << q] - (-1j * s)) < 1e-15
            psi = statevector.simulate(C.Circuit(n, [C.Gate("RY", (q,), (th,))]))
            assert abs(psi[0] - c) < 1e-15 and abs(psi[1 << q] - s) < 1e-15
            psi = statevector.simulate(C.Circuit(n, [C.Gate("X", (q,)), C.Gate("RZ", (q,), (th,))]))
            assert abs(psi[1 << q] - cmath.exp(0.5j * th)) < 1e-15
    psi = statevector.simulate(C.Circuit(1, [C.Gate("RY", (0,), (math.pi / 2,))]))
    assert np.allclose(psi, [1 / math.sqrt(2), 1 / math.sqrt(2)], atol=1e-15)
    rng = np.random.default_rng(11)
    psi0 = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    for th in _THETAS:
        a = statevector.simulate(C.Circuit(3, [C.Gate("H", (1,)), C.Gate("RZ", (1,), (th,)), C.Gate("H", (1,))]),
                                 psi0=psi0.copy())
        b = statevector.simulate(C.Circuit(3, [C.Gate("RX", (1,), (th,))]), psi0=psi0.copy())
        assert np.max(np.abs(a - b)) < 1e-14


def test_qaoa_cost_block_is_zz_exponential():
    # the MaxCut cost block CX(a, b) RZ(2 gamma) on b CX(a, b) equals
    # exp(-i gamma Z_a Z_b): basis state |x> picks up e^{-i gamma z_a z_b}, z = 1 - 2 bit
    n, a, b = 3, 2, 0
    for gamma in (0.4, 1.3, 2.9):
        circ = [C.Gate("CX", (a, b)), C.Gate("RZ", (b,), (2 * gamma,)), C.Gate("CX", (a, b))]
        for x in range(1 << n):
            psi0 = np.zeros(1 << n, complex)
            psi0[x] = 1
            psi = statevector.simulate(C.Circuit(n, circ), psi0=psi0)
            za, zb = 1 - 2 * (x >> a & 1), 1 - 2 * (x >> b & 1)
            expect = np.zeros(1 << n, complex)
            expect[x] = cmath.exp(-1j * gamma * za * zb)
            assert np.max(np.abs(psi - expect)) < 1e-15, (gamma, x)
    # the mixer RX(2 beta) on every qubit: |0..0> -> prod (cos b, -i sin b)
    beta = 0.7
    psi = statevector.simulate(C.Circuit(n, [C.Gate("RX", (q,), (2 * beta,)) for q in range(n)]))
    for x in range(1 << n):
        k = bin(x).count("1")
        assert abs(psi[x] - math.cos(beta) ** (n - k) * (-1j * math.sin(beta)) ** k) < 1e-15


def test_one_and_two_qubit_matrices_act_by_columns():
    # a gate U on a basis state returns U's column: U|j> = sum_i U_ij |i>, with
    # qubit q = bit q of the index and the two-qubit local index bit(q0) + 2 bit(q1)
    rng = np.random.default_rng(12)
    n = 4
    M = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    for q in range(n):
        for j in range(2):
            psi0 = np.zeros(1 << n, complex)
            psi0[j << q] = 1
            psi = statevector.simulate(C.Circuit(n, [C.Gate("U", (q,), (), M)]), psi0=psi0)
            assert abs(psi[0] - M[0, j]) < 1e-15 and abs(psi[1 << q] - M[1, j]) < 1e-15
    M4 = rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4))
    q0, q1 = 3, 1
    for j in range(4):
        psi0 = np.zeros(1 << n, complex)
        psi0[(j & 1) << q0 | (j >> 1) << q1] = 1
        psi = statevector.simulate(C.Circuit(n, [C.Gate("U2", (q0, q1), (), M4)]), psi0=psi0)
        for i in range(4):
            assert abs(psi[(i & 1) << q0 | (i >> 1) << q1] - M4[i, j]) < 1e-15


# --------------------------------------------------- aggregate (stderr) ----

def test_aggregate_standard_error_closed_form():
    # 0/1 scores with k ones among n: the sample variance (n - 1 in the
    # denominator) is k (n - k) / (n (n - 1)), so stderr = sqrt(k (n - k) / (n^2 (n - 1)))
    for n, k in ((10, 3), (400, 17), (2, 1)):
        s = np.array([1.0] * k + [0.0] * (n - k))
        a = montecarlo.aggregate(s, s > 0.5)
        expect = math.sqrt(k * (n - k) / (n * n * (n - 1)))
        assert abs(a["stderr_mean"] - expect) < 1e-15 and abs(a["stderr_pass"] - expect) < 1e-15
        assert a["mean"] == k / n and a["pass_frac"] == k / n
    # the reported stderr matches the spread of batch means of uniform scores
    # (variance 1/12): sd of the mean over 64 scores = sqrt(1 / (12 * 64))
    rng = np.random.default_rng(5)
    errs = [montecarlo.aggregate(x, x > 0.5)["stderr_mean"] for x in rng.random((2000, 64))]
    assert abs(np.mean(errs) / math.sqrt(1 / (12 * 64)) - 1) < 0.02


# ------------------------------------------------------------ search ------

def test_tolerable_rate_closed_form_identity_chain():
    # fidelity target F after G identity gates: p* = 3/4 (1 - (2F - 1)^(1/G))
    G, F = 20, 0.8
    c = C.identity_chain(G)
    c.criterion = C.Criterion("fidelity", aggregate="mean")
    exact = 0.75 * (1 - (2 * F - 1) ** (1 / G))
    r = search.bisect_log(lambda p: (1 + (1 - 4 * p / 3) ** G) / 2, F, 1e-6, 1e-1, rel_tol=1e-3)
    assert abs(r[0] - exact) / exact < 1e-3
    r = search.tolerable_rate(c, F, n_traj=4000, seed=1)
    assert r["mode"] == "eq5"  # one average error already drops F to 1/3 < 0.8
    assert abs(r["p"] - 1.5 * (1 - F) / G) < 1e-12  # Eq. (5): P_R = 1, P_X = P_Y = 0, P_Z = 1
    r = search.tolerable_rate(c, F, n_traj=4000, seed=1, mode="mc")
    assert r["mode"] == "mc"
    assert abs(r["p"] - exact) / exact < 0.1


def test_tolerable_rate_uses_eq5_when_one_error_is_too_many():
    c = C.ghz(3)
    a = exhaustive.analyse(c)
    P1 = exhaustive.one_error_success(a)
    r = search.tolerable_rate(c, 0.5 * (P1 + a["P_R"]))
    assert r["mode"] == "eq5" and 0 < r["p"] < 1 / c.L


# --------------------------------------------- planted mistakes (CPU) -----

def _pin_fails(pin, *args):
    """True when running the pin raises AssertionError (the planted mistake is caught)."""
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


def test_pins_catch_a_wrong_y_sign(monkeypatch):
    # plausible mistake: Y applied with the opposite overall sign
    orig = statevector.apply_pauli

    def wrong(psi, n, q, code):
        orig(psi, n, q, code)
        if code == 3:
            psi *= -1
    monkeypatch.setattr(statevector, "apply_pauli", wrong)
    assert _pin_fails(test_eq2_golden_fixture_and_xx_example)
    assert _pin_fails(test_eq2_single_qubit_paulis_match_paper)


def _patched_one_qubit(monkeypatch, name, fn):
    from oracle import gates
    orig = gates.one_qubit

    def wrong(n, params=(), matrix=None):
        if n == name:
            return fn(orig, params)
        return orig(n, params, matrix)
    monkeypatch.setattr(gates, "one_qubit", wrong)


@pytest.mark.parametrize("mistake", ["rx_sign", "ry_transposed", "rz_full_angle", "s_is_sdg",
                                     "p_conjugated", "sdg_is_s"])
def test_pins_catch_rotation_and_phase_slips(monkeypatch, mistake):
    if mistake == "rx_sign":  # +i sin instead of -i sin
        _patched_one_qubit(monkeypatch, "RX", lambda o, p: o("RX", p).conj())
    elif mistake == "ry_transposed":
        _patched_one_qubit(monkeypatch, "RY", lambda o, p: o("RY", p).T)
    elif mistake == "rz_full_angle":  # exp(-i theta Z) instead of exp(-i theta Z / 2)
        _patched_one_qubit(monkeypatch, "RZ", lambda o, p: o("RZ", (2 * p[0],)))
    elif mistake == "s_is_sdg":
        _patched_one_qubit(monkeypatch, "S", lambda o, p: o("SDG", p))
    elif mistake == "p_conjugated":
        _patched_one_qubit(monkeypatch, "P", lambda o, p: o("P", p).conj())
    elif mistake == "sdg_is_s":
        _patched_one_qubit(monkeypatch, "SDG", lambda o, p: o("S", p))
    caught = [_pin_fails(test_rotations_are_pauli_exponentials),
              _pin_fails(test_phase_gates_are_projector_exponentials),
              _pin_fails(test_rotation_gates_on_basis_states_closed_form),
              _pin_fails(test_qaoa_cost_block_is_zz_exponential)]
    assert any(caught), mistake


def test_pins_catch_a_transposed_one_qubit_update(monkeypatch):
    orig = statevector.apply_1q
    monkeypatch.setattr(statevector, "apply_1q", lambda psi, n, q, U: orig(psi, n, q, U.T))
    assert _pin_fails(test_one_and_two_qubit_matrices_act_by_columns)
    assert _pin_fails(test_rotation_gates_on_basis_states_closed_form)


@pytest.mark.parametrize("mistake", ["ddof0", "no_sqrt_n", "sd_not_sqrt"])
def test_pins_catch_a_wrong_standard_error(monkeypatch, mistake):
    def wrong(scores, flags):
        n = len(scores)
        sd = float(np.std(scores, ddof=0 if mistake == "ddof0" else 1))
        if mistake == "sd_not_sqrt":
            sd = sd * sd
        div = 1.0 if mistake == "no_sqrt_n" else math.sqrt(n)
        sdp = float(np.std(np.asarray(flags, float), ddof=0 if mistake == "ddof0" else 1))
        return {"mean": float(np.mean(scores)), "pass_frac": float(np.mean(flags)),
                "stderr_mean": sd / div, "stderr_pass": sdp / div}
    monkeypatch.setattr(montecarlo, "aggregate", wrong)
    assert _pin_fails(test_aggregate_standard_error_closed_form)


def test_pins_catch_a_dropped_channel_term(monkeypatch):
    c = C.identity_chain(5)
    p = 0.03
    exact = (1 + (1 - 4 * p / 3) ** 5) / 2
    rho = density.evolve(c, p / 3, p / 3, 0.0)  # Y term dropped
    assert abs(density.expected_score(c, rho, statevector.simulate(c)) - exact) > 1e-4


def test_pins_catch_a_transposed_cx():
    # a CX with control and target swapped breaks the GHZ pin
    psi = statevector.simulate(C.Circuit(3, [C.Gate("H", (0,)), C.Gate("CX", (1, 0)), C.Gate("CX", (2, 1))]))
    expect = np.zeros(8, dtype=complex)
    expect[0] = expect[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - expect)) > 0.1


def test_heavy_outputs_of_quantum_volume_circuits():
    # the heavy set is the upper half of the ideal distribution: 2^(n-1)
    # outcomes; a uniform state puts exactly 1/2 on it; for random QV circuits
    # the ideal heavy-output probability approaches (1 + ln 2) / 2 = 0.847
    # (Porter-Thomas statistics, Aaronson & Chen 2017), already near it at n = 6
    hops = []
    for s in range(40):
        circ = C.quantum_volume(6, s)
        assert circ.G == 18 and all(g.name == "U2" for g in circ.gates)
        psi = statevector.simulate(circ, [])
        assert abs(np.linalg.norm(psi) - 1) < 1e-12
        heavy = criteria.heavy_outputs(psi)
        assert len(heavy) == 32
        crit = C.Criterion("binning", basis_set=heavy.tolist(), threshold=2 / 3)
        hops.append(criteria.score(crit, psi))
        uniform = np.full(64, 1 / 8, dtype=np.complex128)
        assert abs(criteria.score(crit, uniform) - 0.5) < 1e-12
    assert 0.80 < np.mean(hops) < 0.90
    assert min(hops) > 0.5


def test_paper_families_closed_forms():
    # BV: the closing H gates map the data qubits to |secret> and the ancilla to |1>
    for n, secret in ((5, 0b1011), (8, 0b1100101)):
        circ = C.bernstein_vazirani(n, secret)
        psi = statevector.simulate(circ, [])
        assert abs(abs(psi[circ.criterion.target]) ** 2 - 1) < 1e-12
    # HLF is a Clifford circuit: its output distribution is uniform on a support of size 2^k
    for seed in range(4):
        pr = np.abs(statevector.simulate(C.hidden_linear_function(7, seed), [])) ** 2
        nz = pr[pr > 1e-12]
        assert abs(nz.sum() - 1) < 1e-12 and np.allclose(nz, nz[0], atol=1e-12)
        assert len(nz) & (len(nz) - 1) == 0
    # RYRZ: depth layers of 2n rotations and n-1 CX, plus a final rotation layer
    circ = C.ryrz_ansatz(6, 3, 1)
    assert circ.G == 3 * (2 * 6 + 5) + 2 * 6
    # UCCSD: every excitation conserves the number of occupied orbitals
    circ = C.uccsd_ansatz(8, 4, 2)
    psi = statevector.simulate(circ, [])
    weight = np.array([bin(i).count("1") for i in range(1 << 8)])
    assert np.sum(np.abs(psi[weight != 4]) ** 2) < 1e-20
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
