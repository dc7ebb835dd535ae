"""The allocation-free scoring entry point against the allocating one.

arso_score_state_noalloc serves callers that cannot call cudaMalloc (code
running inside another allocator's arena, or on paths where allocating would
synchronise or fail); it keeps its scratch in fixed-size device arrays. This
test calls it through the C ABI twice in a row for every criterion and
compares each result with arso_score_state, within the score tolerance the
parity tests use, and checks that repeated calls leave the device's free
memory and the default memory pool's counters unchanged. The file sorts last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import circuits as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCORE_TOL = 1e-5


def test_noalloc_score_matches_allocating_entry_point():
    from paper_2301_07264_gb300 import arso
    fn = arso.lib.arso_score_state_noalloc
    fn.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.POINTER(arso.Criterion), C.c_void_p,
                   C.POINTER(C.c_double)]
    fn.restype = C.c_int
    rng = np.random.default_rng(7)
    for n in (5, 16, 20):
        psi = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
        psi /= np.linalg.norm(psi)
        ref = psi + 0.05 * (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n))
        ref /= np.linalg.norm(ref)
        d_psi = torch.from_numpy(psi.astype(np.complex64)).cuda()
        d_ref = torch.from_numpy(ref.astype(np.complex64)).cuda()
        top = int(np.argmax(np.abs(psi)))
        heavy = tuple(int(i) for i in np.nonzero(np.abs(psi) ** 2 > np.median(np.abs(psi) ** 2))[0])
        crits = [W.Criterion("fidelity"), W.Criterion("outcome", target=top),
                 W.Criterion("binning", basis_set=heavy), W.Criterion("argmax", target=top),
                 W.Criterion("binning", basis_set=(0, 3))]
        for crit in crits:
            c = arso.make_criterion(crit)
            expect = arso.score_state(n, d_psi, d_ref, c)
            for _ in range(2):
                out = C.c_double(-1.0)
                st = fn(n, d_psi.data_ptr(), d_ref.data_ptr(), C.byref(c), None, C.byref(out))
                assert st == arso.OK, arso.lib.arso_last_error().decode()
                assert abs(out.value - expect) < SCORE_TOL, (n, crit.kind)


def test_noalloc_rejects_oversized_binning():
    from paper_2301_07264_gb300 import arso
    fn = arso.lib.arso_score_state_noalloc
    fn.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.POINTER(arso.Criterion), C.c_void_p,
                   C.POINTER(C.c_double)]
    fn.restype = C.c_int
    d = torch.zeros(1 << 21, dtype=torch.complex64, device="cuda")
    c = arso.make_criterion(W.Criterion("binning", basis_set=(1,)))
    out = C.c_double()
    assert fn(21, d.data_ptr(), None, C.byref(c), None, C.byref(out)) == arso.EINVAL
    assert b"20 qubits" in arso.lib.arso_last_error()


def _driver_memory():
    """(free device bytes, default pool reserved bytes, default pool used bytes)
    read through the CUDA driver in the current context."""
    cu = C.CDLL("libcuda.so.1")
    free, total = C.c_size_t(), C.c_size_t()
    assert cu.cuMemGetInfo_v2(C.byref(free), C.byref(total)) == 0
    dev = C.c_int()
    assert cu.cuCtxGetDevice(C.byref(dev)) == 0
    pool = C.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(C.byref(pool), dev) == 0
    reserved, used = C.c_uint64(), C.c_uint64()
    assert cu.cuMemPoolGetAttribute(pool, 5, C.byref(reserved)) == 0  # RESERVED_MEM_CURRENT
    assert cu.cuMemPoolGetAttribute(pool, 7, C.byref(used)) == 0  # USED_MEM_CURRENT
    return free.value, reserved.value, used.value


def test_noalloc_leaves_device_memory_unchanged():
    # the entry point exists for callers that must not grow device memory, so
    # after a first round (which loads the kernels into the context) repeated
    # calls over every criterion and size must leave the driver's free memory
    # and the default memory pool's reserved and used bytes exactly as they were
    from paper_2301_07264_gb300 import arso
    fn = arso.lib.arso_score_state_noalloc
    fn.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.POINTER(arso.Criterion), C.c_void_p,
                   C.POINTER(C.c_double)]
    fn.restype = C.c_int
    rng = np.random.default_rng(8)
    cases = []
    for n in (6, 18, 20):
        psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
        d_psi = torch.from_numpy(psi).cuda()
        crits = [W.Criterion("fidelity"), W.Criterion("outcome", target=3), W.Criterion("argmax", target=1),
                 W.Criterion("binning", basis_set=tuple(range(0, 1 << n, 3)))]
        cases += [(n, d_psi, arso.make_criterion(c)) for c in crits]
    torch.cuda.synchronize()

    def round_():
        vals = []
        for n, d_psi, c in cases:
            out = C.c_double(-1.0)
            st = fn(n, d_psi.data_ptr(), d_psi.data_ptr(), C.byref(c), None, C.byref(out))
            assert st == arso.OK, arso.lib.arso_last_error().decode()
            vals.append(out.value)
        return vals

    first = round_()
    before = _driver_memory()
    torch_before = torch.cuda.memory_reserved()
    for _ in range(3):
        assert round_() == first
    assert _driver_memory() == before
    assert torch.cuda.memory_reserved() == torch_before
