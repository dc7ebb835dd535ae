"""Host-side checks that need no GPU: the C-ABI library loads, exports every
function declared in include/*.h, reports errors without a device, and the
pass scheduler keeps the circuit's dependencies."""
import glob
import os
import re

import numpy as np
import pytest

from workloads import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(arso_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def arso():
    from paper_2301_07264_gb300 import build
    build.build()
    from paper_2301_07264_gb300 import arso as mod
    return mod


def test_library_exports_every_declared_symbol(arso):
    declared = _declared()
    assert len(declared) >= 20
    missing = [n for n in declared if not hasattr(arso.lib, n)]
    assert not missing, missing


def test_version_and_errors_without_device(arso):
    assert "sm_103a" in arso.version()
    st = arso.lib.arso_circuit_get_info(None, None)
    assert st == arso.EINVAL
    assert arso.lib.arso_last_error()


def _check_schedule(circ, tile, low):
    from paper_2301_07264_gb300 import arso
    perm, begin, masks = arso.plan_schedule(circ.n, circ.gates, tile_qubits=tile, low_qubits=low)
    G = circ.G
    assert sorted(perm.tolist()) == list(range(G))
    # every gate's qubits are tile qubits of its pass; low qubits in every tile
    for p in range(len(masks)):
        m = int(masks[p])
        assert bin(m).count("1") == min(tile, circ.n)
        assert all((m >> q) & 1 for q in range(min(low, tile)))
        for pos in range(begin[p], begin[p + 1]):
            for q in circ.gates[perm[pos]].qubits:
                assert (m >> q) & 1
    # the engine order keeps the order of gates on every qubit
    last = {}
    for pos in range(G):
        g = int(perm[pos])
        for q in circ.gates[g].qubits:
            assert last.get(q, -1) < g
            last[q] = g
    return len(masks)


@pytest.mark.parametrize("n,G,tile,low,seed", [(14, 300, 8, 3, 1), (20, 400, 13, 4, 2), (24, 200, 14, 5, 3)])
def test_schedule_respects_dependencies(arso, n, G, tile, low, seed):
    _check_schedule(C.random_circuit(n, G, seed), tile, low)


def test_brickwork24_schedule_is_fused(arso):
    # the frontier-closure pass builder: 1420 gates in at most 23 HBM sweeps at 13-qubit tiles
    # and 26 at 12-qubit tiles (the circuit-order builder needed 46 at 13)
    assert _check_schedule(C.brickwork24(0), 13, 4) <= 23
    assert _check_schedule(C.brickwork24(0), 12, 4) <= 26


@pytest.mark.parametrize("n,G,tile,low,frac,seed", [
    (14, 500, 10, 1, 0.3, 21), (16, 800, 11, 2, 0.6, 22), (18, 600, 12, 3, 0.5, 23), (20, 900, 12, 4, 0.4, 24),
    (22, 700, 13, 5, 0.5, 25), (24, 1200, 14, 4, 0.5, 26), (19, 400, 6, 3, 0.7, 27), (15, 300, 14, 5, 0.2, 28)])
def test_frontier_schedules_of_random_circuits(arso, n, G, tile, low, frac, seed):
    # every gate kind, two-qubit fractions 0.2-0.7, tiles 6-14, 1-5 contiguous low qubits
    _check_schedule(C.random_circuit(n, G, seed, two_qubit_frac=frac), tile, low)


def test_plan_tensor_phase_rejects_a_phase_out_of_range(arso):
    circ = C.brickwork(16, 4, 1)
    n_ph = arso.plan_phases(16, circ.gates, tile_qubits=13, flags=arso.OPT_TENSOR_PHASES)
    with pytest.raises(arso.ArsoError) as e:
        arso.plan_tensor_phase(16, circ.gates, n_ph, tile_qubits=13)
    assert e.value.status == arso.EINVAL


@pytest.mark.parametrize("make,tile,low", [(lambda: C.qaoa_maxcut(24, 2), 13, 4),
                                           (lambda: C.qft_basis(20, 12345), 13, 4),
                                           (lambda: C.cuccaro_adder(9, 301, 177), 12, 3),
                                           (lambda: C.brickwork(16, 12, 3), 10, 2)])
def test_frontier_schedules_are_valid(arso, make, tile, low):
    _check_schedule(make(), tile, low)


def test_resident_circuits_plan_one_pass(arso):
    # one pass over the whole register; the phase planner may reorder gates on
    # disjoint qubits but keeps the order of the gates on every qubit
    assert _check_schedule(C.grover12(0), 12, 4) == 1


def test_phase_planner_counts(arso):
    # the list-scheduling planner: brickwork-24 at 13-qubit tiles needs at most
    # 160 phases for 1420 gates; Grover-12's 60,771 gates need at least
    # ceil(60,771 / 64) phases of at most 64 gates, and at most 1,310
    assert arso.plan_phases(24, C.brickwork24(0).gates, tile_qubits=13) <= 160
    assert 950 <= arso.plan_phases(12, C.grover12(0).gates) <= 1310


def test_tensor_phase_plans(arso):
    # tensor-core phases: brickwork-24 at 13-qubit tiles plans at most 170 phases,
    # at least 120 of them fused unitaries; without the flag, and for resident
    # circuits, none
    n, nt = arso.plan_phases(24, C.brickwork24(0).gates, tile_qubits=13, flags=arso.OPT_TENSOR_PHASES, tensor=True)
    assert n <= 170 and 120 <= nt <= n
    assert arso.plan_phases(24, C.brickwork24(0).gates, tile_qubits=13, tensor=True)[1] == 0
    assert arso.plan_phases(12, C.grover12(0).gates, flags=arso.OPT_TENSOR_PHASES, tensor=True)[1] == 0
    # tiles below 12 qubits never take the route
    assert arso.plan_phases(16, C.brickwork(16, 8, 1).gates, tile_qubits=11, flags=arso.OPT_TENSOR_PHASES,
                            tensor=True)[1] == 0


def test_inverse_gate_count_fit():
    # the Sec. V-B fit: data exactly b / G returns b with zero residual and a
    # zero intercept; data a + b / G returns (a, b) from the affine fit
    from paper_2301_07264_gb300.bench_workloads import fit_inverse_gate_count
    Gs = [40, 90, 200, 350, 800]
    f = fit_inverse_gate_count(Gs, [0.3 / g for g in Gs], 3000)
    assert abs(f["b"] - 0.3) < 1e-12 and f["mse"] < 1e-30
    assert abs(f["affine_a"]) < 1e-12 and abs(f["affine_b"] - 0.3) < 1e-10
    assert f["G_56"] == 3000 and abs(f["p_tol_56_extrapolated"] - 1e-4) < 1e-15
    f = fit_inverse_gate_count(Gs, [2e-4 + 0.25 / g for g in Gs], 1000)
    assert abs(f["affine_a"] - 2e-4) < 1e-12 and abs(f["affine_b"] - 0.25) < 1e-10 and f["affine_mse"] < 1e-28
    assert f["mse"] > 0
