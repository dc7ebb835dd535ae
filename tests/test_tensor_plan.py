"""Host side of the tensor-core phases (no GPU): for every phase that runs as a
fused-unitary contraction, the operand image the library builds equals the real
64 x 64 form of the product of the phase's core gates, rebuilt here from the
oracle's gate matrices in the phase's record order; the high terms are integers;
and every gate left outside the unitary is diagonal and sits where running it
before or after the unitary equals the record order."""
import numpy as np
import pytest

from oracle import gates as og
from workloads import circuits as C

DIAGONAL = {"CZ", "CP", "Z", "S", "SDG", "T", "TDG", "RZ", "P", "ID"}

CASES = {
    "brickwork16_t13": (lambda: C.brickwork(16, 12, 3), 13, 4),
    "random16_t13": (lambda: C.random_circuit(16, 300, 6, two_qubit_frac=0.5), 13, 4),
    "qaoa16_t12": (lambda: C.qaoa_maxcut(16, 2), 12, 4),
}


@pytest.fixture(scope="module")
def arso():
    from paper_2301_07264_gb300 import arso as mod
    return mod


def _apply(U, m, pos):
    """U <- G U for the gate matrix m on register positions pos (index bit(pos[0]) +
    2 bit(pos[1]) for two-qubit gates), U indexed [output register, input register]."""
    out = U.copy()
    bits = [1 << p for p in pos]
    for l in range(32):
        if l & sum(bits):
            continue
        idx = [l, l | bits[0]] if len(bits) == 1 else [l, l | bits[0], l | bits[1], l | bits[0] | bits[1]]
        out[idx, :] = m @ U[idx, :]
    return out


def _real_form(U):
    """B[n][k] for output n = 4p + 2c + lane (register 2p + lane, c = 0 real, 1 imaginary)
    and input k likewise, so that D = A B^T applies U to rows of packed registers."""
    B = np.zeros((64, 64))
    for n in range(64):
        j, co = 2 * (n >> 2) + (n & 1), (n >> 1) & 1
        for k in range(64):
            l, ci = 2 * (k >> 2) + (k & 1), (k >> 1) & 1
            u = U[j, l]
            B[n, k] = (u.real if ci == 0 else -u.imag) if co == 0 else (u.imag if ci == 0 else u.real)
    return B


def _decode(image):
    h = image.view(np.float16).astype(np.float64)
    hi, lo = h[:4096], h[4096:]
    B = np.zeros((64, 64))
    Bhi = np.zeros((64, 64))
    for n in range(64):
        for k in range(64):
            i = (n // 8) * 512 + (k // 8) * 64 + (n % 8) * 8 + k % 8
            B[n, k] = hi[i] + lo[i]
            Bhi[n, k] = hi[i]
    return B, Bhi


@pytest.mark.parametrize("case", sorted(CASES))
def test_tensor_images_equal_the_product_of_the_core_gates(arso, case):
    make, tile, low = CASES[case]
    circ = make()
    perm, begin, masks = arso.plan_schedule(circ.n, circ.gates, tile_qubits=tile, low_qubits=low,
                                            flags=arso.OPT_TENSOR_PHASES)
    n_ph, n_t = arso.plan_phases(circ.n, circ.gates, tile_qubits=tile, low_qubits=low,
                                 flags=arso.OPT_TENSOR_PHASES, tensor=True)
    assert n_t > 0
    checked = 0
    for ph in range(n_ph):
        d = arso.plan_tensor_phase(circ.n, circ.gates, ph, tile_qubits=tile, low_qubits=low)
        if d["image"] is None:
            continue
        m = int(masks[d["pass"]])
        local = {q: i for i, q in enumerate(q for q in range(circ.n) if (m >> q) & 1)}
        R = d["R"]
        U = np.eye(32, dtype=np.complex128)
        started, core_dense = set(), []
        b, e = d["pos"]
        for pos in range(b, e):
            g = circ.gates[int(perm[pos])]
            qs = [local[q] for q in g.qubits]
            role = int(d["roles"][pos - b])
            if all(q in R for q in qs):
                assert role == 0
                U = _apply(U, og.matrix_of(g), [R.index(q) for q in qs])
                if g.name not in DIAGONAL:
                    core_dense.append((pos, set(qs)))
            else:
                assert g.name in DIAGONAL and role in (1, 2), (case, ph, g.name, role)
                rq = {q for q in qs if q in R}
                before = any(p < pos and rq & s for p, s in core_dense)
                assert before == (role == 2), (case, ph, pos)
                if role == 2:
                    started |= rq
        # no non-diagonal core gate acts on a register bit after a gate run after U touched it
        for pos in range(b, e):
            if int(d["roles"][pos - b]) != 2:
                continue
            g = circ.gates[int(perm[pos])]
            rq = {local[q] for q in g.qubits} & set(R)
            assert not any(p > pos and rq & s for p, s in core_dense), (case, ph, pos)
        B, Bhi = _decode(d["image"])
        assert np.array_equal(Bhi, np.rint(Bhi))
        assert np.max(np.abs(B - 256.0 * _real_form(U))) <= 2.0 ** -11, (case, ph)
        checked += 1
    assert checked == n_t


def test_no_images_without_the_flag(arso):
    circ = C.brickwork(16, 12, 3)
    n_ph = arso.plan_phases(circ.n, circ.gates, tile_qubits=13)
    for ph in range(n_ph):
        assert arso.plan_tensor_phase(circ.n, circ.gates, ph, tile_qubits=13, flags=0)["image"] is None
