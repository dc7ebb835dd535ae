"""Python binding of the C ABI declared in include/arso.h.

Argument marshalling only: every step of the simulation, sampling, scoring and
search runs inside libarso.so. Functions carry the ABI's names without the
``arso_`` prefix. Device buffers are torch CUDA tensors (or raw integer device
pointers); host buffers are numpy arrays. Streams are ``torch.cuda.Stream``
objects, raw ``cudaStream_t`` integers, or None (legacy default stream).

Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libarso.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libarso.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
lib = C.CDLL(_LIB_PATH)

# ------------------------------------------------------------------ enums --
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED, ENOTCONVERGED = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EUNSUPPORTED", "ENOTCONVERGED"]

GATE_KIND = {
    "ID": 0, "H": 1, "X": 2, "Y": 3, "Z": 4, "S": 5, "SDG": 6, "T": 7, "TDG": 8,
    "RX": 9, "RY": 10, "RZ": 11, "P": 12, "U": 13,
    "CX": 32, "CZ": 33, "CP": 34, "SWAP": 35, "U2": 36,
}
C64, C128 = 0, 1
CRIT_KIND = {"fidelity": 0, "outcome": 1, "binning": 2, "argmax": 3}
AGGREGATE = {"mean": 0, "pass": 1}
MODE = {"auto": 0, "mc": 1, "exhaustive": 2}


class ArsoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


# --------------------------------------------------------------- structs --
class Gate(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("q", C.c_uint32 * 2), ("param", C.c_double),
                ("matrix", C.POINTER(C.c_double))]


class CompileOpts(C.Structure):
    _fields_ = [("precision", C.c_uint32), ("tile_qubits", C.c_uint32), ("low_qubits", C.c_uint32),
                ("max_batch", C.c_uint32), ("cache_bytes", C.c_uint64), ("flags", C.c_uint32)]


class CircuitInfo(C.Structure):
    _fields_ = [("n_qubits", C.c_uint32), ("G", C.c_uint64), ("k", C.c_uint64), ("m", C.c_uint64),
                ("L", C.c_uint64), ("engine", C.c_uint32), ("n_passes", C.c_uint32),
                ("tile_qubits", C.c_uint32), ("precision", C.c_uint32), ("checkpoint_every", C.c_uint64),
                ("n_phases", C.c_uint32), ("tensor_phases", C.c_uint32)]


class Criterion(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("aggregate", C.c_uint32), ("target", C.c_uint64),
                ("set", C.POINTER(C.c_uint64)), ("set_len", C.c_size_t), ("threshold", C.c_double)]


class Result(C.Structure):
    _fields_ = [("value", C.c_double), ("mean", C.c_double), ("pass_frac", C.c_double),
                ("stderr_value", C.c_double), ("expected_errors", C.c_double), ("mode_used", C.c_uint32),
                ("n_traj", C.c_uint64), ("P_R", C.c_double), ("P_X", C.c_double), ("P_Z", C.c_double),
                ("P_Y", C.c_double)]


class SearchOpts(C.Structure):
    _fields_ = [("p_lo", C.c_double), ("p_hi", C.c_double), ("rel_tol", C.c_double), ("n_traj", C.c_uint64),
                ("seed", C.c_uint64), ("max_probes", C.c_uint32), ("mode", C.c_uint32),
                ("surrogate", C.c_void_p), ("features", C.POINTER(C.c_float)), ("surrogate_margin", C.c_double),
                ("flags", C.c_uint32)]


class RateResult(C.Structure):
    _fields_ = [("p", C.c_double), ("lo", C.c_double), ("hi", C.c_double), ("value_lo", C.c_double),
                ("value_hi", C.c_double), ("probes", C.c_uint32), ("mode_used", C.c_uint32),
                ("used_surrogate", C.c_uint32), ("verified", C.c_uint32), ("converged", C.c_uint32),
                ("P1", C.c_double)]


_vp = C.c_void_p
_sigs = {
    "arso_compile_circuit": [C.c_uint32, C.POINTER(Gate), C.c_size_t, C.POINTER(CompileOpts), C.POINTER(_vp)],
    "arso_circuit_get_info": [_vp, C.POINTER(CircuitInfo)],
    "arso_plan_schedule": [C.c_uint32, C.POINTER(Gate), C.c_size_t, C.POINTER(CompileOpts), C.POINTER(C.c_uint32),
                           C.c_uint32, _vp, _vp, _vp],
    "arso_sample_errors": [_vp, C.c_double, C.c_double, C.c_double, C.c_uint64, C.c_uint64, C.c_uint64, _vp,
                           C.POINTER(_vp)],
    "arso_sample_errors_batch": [C.c_size_t, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "arso_error_list_from_host": [_vp, C.c_uint64, _vp, _vp, _vp, C.POINTER(_vp)],
    "arso_error_list_info": [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)],
    "arso_error_list_copy": [_vp, _vp, _vp, _vp],
    "arso_run_trajectories": [_vp, _vp, C.POINTER(Criterion), _vp, _vp, _vp],
    "arso_trajectory_states": [_vp, _vp, C.c_uint64, C.c_uint64, _vp, _vp],
    "arso_reference_state": [_vp, _vp, _vp],
    "arso_exhaustive": [_vp, C.POINTER(Criterion), _vp, _vp, _vp],
    "arso_success_prob": [_vp, C.POINTER(Criterion), C.c_double, C.c_uint32, C.c_uint64, C.c_uint64, _vp,
                          C.POINTER(Result)],
    "arso_tolerable_rate": [_vp, C.POINTER(Criterion), C.c_double, C.POINTER(SearchOpts), _vp,
                            C.POINTER(RateResult)],
    "arso_apply_gate": [C.c_uint32, _vp, C.POINTER(Gate), _vp],
    "arso_apply_pauli": [C.c_uint32, _vp, C.c_uint32, C.c_uint32, _vp],
    "arso_score_state": [C.c_uint32, _vp, _vp, C.POINTER(Criterion), _vp, C.POINTER(C.c_double)],
    "arso_aggregate": [_vp, _vp, C.c_uint64, _vp, _vp],
    "arso_profile_enable": [C.c_int],
    "arso_profile_reset": [],
    "arso_profile_read": [C.c_uint32, _vp],
    "arso_profile_counters": [_vp, _vp, _vp],
}
for _name, _args in _sigs.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.arso_circuit_free.argtypes = [_vp]
lib.arso_circuit_free.restype = None
lib.arso_error_list_free.argtypes = [_vp]
lib.arso_error_list_free.restype = None
lib.arso_last_error.restype = C.c_char_p
lib.arso_version.restype = C.c_char_p


def _check(status):
    if status != OK:
        raise ArsoError(status, lib.arso_last_error().decode())


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _ptr(buf):
    """Device pointer of a torch tensor, host pointer of a numpy array, or an int."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if isinstance(buf, np.ndarray):
        assert buf.flags["C_CONTIGUOUS"]
        return buf.ctypes.data
    assert buf.is_contiguous()
    return int(buf.data_ptr())


# ---------------------------------------------------------------- handles --
class CompiledCircuit:
    def __init__(self, handle, n):
        self.handle = handle
        self.n = n

    def info(self) -> CircuitInfo:
        return circuit_get_info(self)

    def __del__(self):
        if getattr(self, "handle", None):
            lib.arso_circuit_free(self.handle)
            self.handle = None


class ErrorList:
    def __init__(self, handle, circuit):
        self.handle = handle
        self.circuit = circuit  # keep the circuit alive

    def info(self):
        nt, ne = C.c_uint64(), C.c_uint64()
        _check(lib.arso_error_list_info(self.handle, C.byref(nt), C.byref(ne)))
        return nt.value, ne.value

    def __del__(self):
        if getattr(self, "handle", None):
            lib.arso_error_list_free(self.handle)
            self.handle = None


def _gates_array(gates):
    arr = (Gate * max(len(gates), 1))()
    keep = []
    for i, g in enumerate(gates):
        arr[i].kind = GATE_KIND[g.name]
        arr[i].q[0] = g.qubits[0]
        arr[i].q[1] = g.qubits[1] if len(g.qubits) > 1 else 0
        arr[i].param = g.params[0] if g.params else 0.0
        if g.matrix is not None:
            m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128)).view(np.float64).ravel().copy()
            keep.append(m)
            arr[i].matrix = m.ctypes.data_as(C.POINTER(C.c_double))
    return arr, keep


OPT_NO_SUFFIX_REUSE = 1
OPT_NO_GRAPHS = 2
OPT_NO_FAST_EXHAUSTIVE = 4
OPT_NO_PERSISTENT = 8
OPT_TENSOR_PHASES = 16


def compile_circuit(n, gates, precision=C64, tile_qubits=0, low_qubits=0, max_batch=0, cache_bytes=0, flags=0):
    arr, keep = _gates_array(gates)
    opts = CompileOpts(precision, tile_qubits, low_qubits, max_batch, cache_bytes, flags)
    h = _vp()
    _check(lib.arso_compile_circuit(n, arr, len(gates), C.byref(opts), C.byref(h)))
    del keep
    return CompiledCircuit(h.value, n)


def plan_schedule(n, gates, precision=C64, tile_qubits=0, low_qubits=0, flags=0):
    """Host-only: (perm, pass_begin, tile_masks) of the fused pass schedule (the engine
    order depends on the phase planner, so on ARSO_OPT_TENSOR_PHASES in flags)."""
    arr, keep = _gates_array(gates)
    opts = CompileOpts(precision, tile_qubits, low_qubits, 0, 0, flags)
    P = C.c_uint32()
    _check(lib.arso_plan_schedule(n, arr, len(gates), C.byref(opts), C.byref(P), 0, None, None, None))
    perm = np.zeros(max(len(gates), 1), dtype=np.uint32)
    begin = np.zeros(P.value + 1, dtype=np.uint32)
    masks = np.zeros(max(P.value, 1), dtype=np.uint64)
    _check(lib.arso_plan_schedule(n, arr, len(gates), C.byref(opts), C.byref(P), P.value, perm.ctypes.data,
                                  begin.ctypes.data, masks.ctypes.data))
    return perm[: len(gates)], begin, masks[: P.value]


def circuit_get_info(circ) -> CircuitInfo:
    info = CircuitInfo()
    _check(lib.arso_circuit_get_info(circ.handle, C.byref(info)))
    return info


def make_criterion(crit):
    """Criterion from an object/dict with kind, target, basis_set, threshold, aggregate."""
    get = (lambda k, d=None: crit.get(k, d)) if isinstance(crit, dict) else (lambda k, d=None: getattr(crit, k, d))
    s = np.ascontiguousarray(np.asarray(get("basis_set", ()) or (), dtype=np.uint64))
    c = Criterion(CRIT_KIND[get("kind", "fidelity")], AGGREGATE[get("aggregate", "mean")], int(get("target", 0)),
                  s.ctypes.data_as(C.POINTER(C.c_uint64)) if s.size else None, s.size,
                  float(get("threshold", 0.5)))
    c._keep = s
    return c


def sample_errors(circ, p_x, p_z, p_y, seed, traj_begin, n_traj, stream=None) -> ErrorList:
    h = _vp()
    _check(lib.arso_sample_errors(circ.handle, p_x, p_z, p_y, seed, traj_begin, n_traj, _stream(stream),
                                  C.byref(h)))
    return ErrorList(h.value, circ)


def sample_errors_batch(circuits, p_x, p_z, p_y, seeds, traj_begin, n_traj, stream=None):
    """Error lists of many circuits in one call (include/arso.h, arso_sample_errors_batch);
    scalar arguments apply to every entry."""
    n = len(circuits)

    def arr(v, ct):
        v = list(v) if hasattr(v, "__len__") else [v] * n
        return (ct * n)(*v)
    hs = (_vp * n)(*[c.handle for c in circuits])
    outs = (_vp * n)()
    _check(lib.arso_sample_errors_batch(n, hs, arr(p_x, C.c_double), arr(p_z, C.c_double), arr(p_y, C.c_double),
                                        arr(seeds, C.c_uint64), arr(traj_begin, C.c_uint64), arr(n_traj, C.c_uint64),
                                        _stream(stream), outs))
    return [ErrorList(outs[i], circuits[i]) for i in range(n)]


def error_list_from_host(circ, lists, stream=None) -> ErrorList:
    """lists: per trajectory, a sorted list of (location, code)."""
    off = np.zeros(len(lists) + 1, dtype=np.uint64)
    ev = []
    for i, l in enumerate(lists):
        off[i + 1] = off[i] + len(l)
        ev += [(loc << 2) | code for loc, code in l]
    evs = np.asarray(ev if ev else [0], dtype=np.uint32)
    h = _vp()
    _check(lib.arso_error_list_from_host(circ.handle, len(lists), off.ctypes.data, evs.ctypes.data,
                                         _stream(stream), C.byref(h)))
    return ErrorList(h.value, circ)


def error_list_copy(errs, stream=None):
    nt, ne = errs.info()
    off = np.zeros(nt + 1, dtype=np.uint64)
    ev = np.zeros(max(ne, 1), dtype=np.uint32)
    _check(lib.arso_error_list_copy(errs.handle, off.ctypes.data, ev.ctypes.data, _stream(stream)))
    return off, ev[:ne]


def run_trajectories(circ, errs, crit, score_out, pass_out=None, stream=None):
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    _check(lib.arso_run_trajectories(circ.handle, errs.handle, C.byref(c), _stream(stream), _ptr(score_out),
                                     _ptr(pass_out)))


def aggregate(score, pass_flags=None, stream=None):
    """(mean, pass_frac, stderr_mean, stderr_pass, n) of device score / flag arrays."""
    out = np.zeros(5)
    n = score.numel() if hasattr(score, "numel") else len(score)
    _check(lib.arso_aggregate(_ptr(score), _ptr(pass_flags), n, _stream(stream), out.ctypes.data))
    return tuple(out)


class KernelStats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("ms", C.c_double), ("bytes", C.c_double), ("flops", C.c_double),
                ("smem_bytes", C.c_double)]


K_PASS, K_PASS_LAST, K_RESIDENT, K_SAMPLE, K_REDUCE, K_OTHER, K_GEMM, K_MIX = range(8)


def profile_enable(on=True):
    _check(lib.arso_profile_enable(1 if on else 0))


def profile_reset():
    _check(lib.arso_profile_reset())


def profile_read(kernel) -> KernelStats:
    s = KernelStats()
    _check(lib.arso_profile_read(kernel, C.byref(s)))
    return s


def profile_counters():
    a, b, c = C.c_uint64(), C.c_uint64(), C.c_uint64()
    _check(lib.arso_profile_counters(C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def trajectory_states(circ, errs, first, count, amps_out, stream=None):
    _check(lib.arso_trajectory_states(circ.handle, errs.handle, first, count, _stream(stream), _ptr(amps_out)))


def reference_state(circ, amps_out, stream=None):
    _check(lib.arso_reference_state(circ.handle, _stream(stream), _ptr(amps_out)))


def exhaustive(circ, crit, per_location=True, stream=None):
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    P = np.zeros(4)
    info = circ.info()
    per = np.zeros(max(3 * info.L, 1)) if per_location else None
    _check(lib.arso_exhaustive(circ.handle, C.byref(c), _stream(stream), P.ctypes.data,
                               per.ctypes.data if per is not None else None))
    return P, (per[: 3 * info.L] if per is not None else None)


def success_prob(circ, crit, p, mode="auto", n_traj=1000, seed=0, stream=None) -> Result:
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    r = Result()
    _check(lib.arso_success_prob(circ.handle, C.byref(c), p, MODE[mode], n_traj, seed, _stream(stream),
                                 C.byref(r)))
    return r


SEARCH_NO_REUSE = 1


def tolerable_rate(circ, crit, P_target, p_lo=0.0, p_hi=0.0, rel_tol=0.0, n_traj=0, seed=0, max_probes=0,
                   mode="auto", stream=None, check=True, reuse=True) -> RateResult:
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    o = SearchOpts(p_lo, p_hi, rel_tol, n_traj, seed, max_probes, MODE[mode], None, None, 0.0,
                   0 if reuse else SEARCH_NO_REUSE)
    r = RateResult()
    st = lib.arso_tolerable_rate(circ.handle, C.byref(c), P_target, C.byref(o), _stream(stream), C.byref(r))
    if check:
        _check(st)
    return r


def apply_gate(n, amps, gate, stream=None):
    arr, keep = _gates_array([gate])
    _check(lib.arso_apply_gate(n, _ptr(amps), arr, _stream(stream)))


def apply_pauli(n, amps, qubit, code, stream=None):
    _check(lib.arso_apply_pauli(n, _ptr(amps), qubit, code, _stream(stream)))


def score_state(n, amps, ref, crit, stream=None) -> float:
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    out = C.c_double()
    _check(lib.arso_score_state(n, _ptr(amps), _ptr(ref), C.byref(c), _stream(stream), C.byref(out)))
    return out.value


def version() -> str:
    return lib.arso_version().decode()


# ------------------------------------------------------------- surrogate --
N_FEATURES = 32
SURROGATE_INPUTS = 33
SURROGATE_PARAMS = 33 * 256 + 256 + 256 * 256 + 256 + 256 + 1

for _name, _args in {
    "arso_circuit_features": [_vp, C.POINTER(Criterion), _vp],
    "arso_surrogate_create": [C.c_uint64, C.POINTER(_vp)],
    "arso_surrogate_train": [_vp, _vp, _vp, C.c_uint64, C.c_uint32, C.c_uint32, C.c_double, C.c_uint64, _vp, _vp],
    "arso_surrogate_predict": [_vp, _vp, C.c_uint64, _vp, _vp],
    "arso_surrogate_get_params": [_vp, _vp],
    "arso_surrogate_set_params": [_vp, _vp],
    "arso_surrogate_set_norm": [_vp, _vp, _vp],
    "arso_surrogate_grads": [_vp, _vp, _vp, C.c_uint64, _vp, _vp, _vp],
    "arso_debug_stall_next_gemm": [],
    "arso_debug_stall_next_batch": [],
    "arso_tolerable_rate_surrogate": [_vp, C.POINTER(Criterion), C.c_double, C.POINTER(SearchOpts), _vp,
                                      C.POINTER(RateResult)],
}.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.arso_surrogate_free.argtypes = [_vp]
lib.arso_surrogate_free.restype = None


class Surrogate:
    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None):
            lib.arso_surrogate_free(self.handle)
            self.handle = None


def circuit_features(circ, crit):
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    out = np.zeros(N_FEATURES, dtype=np.float32)
    _check(lib.arso_circuit_features(circ.handle, C.byref(c), out.ctypes.data))
    return out


def surrogate_create(seed=0) -> Surrogate:
    h = _vp()
    _check(lib.arso_surrogate_create(seed, C.byref(h)))
    return Surrogate(h.value)


def surrogate_train(s, x, y, epochs=1, batch=4096, lr=1e-3, seed=0, stream=None):
    """x: device (n, 33) float32; y: device (n,) float32 pass flags. Returns the last epoch's mean loss."""
    loss = C.c_double()
    n = x.shape[0]
    _check(lib.arso_surrogate_train(s.handle, _ptr(x), _ptr(y), n, epochs, batch, lr, seed, _stream(stream),
                                    C.byref(loss)))
    return loss.value


def surrogate_predict(s, x, out, stream=None):
    _check(lib.arso_surrogate_predict(s.handle, _ptr(x), x.shape[0], _ptr(out), _stream(stream)))


def surrogate_get_params(s):
    out = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
    _check(lib.arso_surrogate_get_params(s.handle, out.ctypes.data))
    return out


def surrogate_set_params(s, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(lib.arso_surrogate_set_params(s.handle, p.ctypes.data))


def surrogate_set_norm(s, mean, sd):
    m = np.ascontiguousarray(mean, dtype=np.float32)
    d = np.ascontiguousarray(sd, dtype=np.float32)
    _check(lib.arso_surrogate_set_norm(s.handle, m.ctypes.data, d.ctypes.data))


def surrogate_grads(s, x, y, stream=None):
    g = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
    loss = C.c_double()
    _check(lib.arso_surrogate_grads(s.handle, _ptr(x), _ptr(y), x.shape[0], _stream(stream), g.ctypes.data,
                                    C.byref(loss)))
    return g, loss.value


def debug_stall_next_gemm():
    """Make the next tensor-core GEMM with a TMA operand give up its bounded wait
    (see include/arso.h); the call that launches it raises ArsoError(ETIMEOUT)."""
    _check(lib.arso_debug_stall_next_gemm())


def debug_stall_next_batch():
    """Make the next persistent batch launch's dependency waits run out (see
    include/arso.h); that run_batch call raises ArsoError(ETIMEOUT)."""
    _check(lib.arso_debug_stall_next_batch())


def tolerable_rate_surrogate(circ, crit, P_target, surrogate, p_lo=0.0, p_hi=0.0, n_traj=0, seed=0, margin=0.0,
                             rel_tol=0.0, max_probes=0, stream=None, reuse=True) -> RateResult:
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    o = SearchOpts(p_lo, p_hi, rel_tol, n_traj, seed, max_probes, MODE["mc"], surrogate.handle, None, margin,
                   0 if reuse else SEARCH_NO_REUSE)
    r = RateResult()
    _check(lib.arso_tolerable_rate_surrogate(circ.handle, C.byref(c), P_target, C.byref(o), _stream(stream),
                                             C.byref(r)))
    return r


lib.arso_run_batch.argtypes = [C.c_size_t, _vp, _vp, _vp, _vp, _vp, _vp]
lib.arso_run_batch.restype = C.c_int


def run_batch(circuits, error_lists, crits, score_outs, pass_outs=None, stream=None):
    """One call over many circuits (see include/arso.h, arso_run_batch)."""
    n = len(circuits)
    ch = (C.c_void_p * n)(*[c.handle for c in circuits])
    eh = (C.c_void_p * n)(*[e.handle for e in error_lists])
    cs = (Criterion * n)()
    keep = []
    for i, cr in enumerate(crits):
        c = cr if isinstance(cr, Criterion) else make_criterion(cr)
        keep.append(c)
        cs[i] = c
    so = (C.c_void_p * n)(*[_ptr(x) for x in score_outs])
    po = (C.c_void_p * n)(*[_ptr(x) for x in pass_outs]) if pass_outs is not None else None
    _check(lib.arso_run_batch(n, ch, eh, cs, _stream(stream), so, po))


lib.arso_autotune.argtypes = [C.c_uint32, C.POINTER(Gate), C.c_size_t, C.POINTER(Criterion), C.c_double, C.c_uint64,
                              C.c_uint64, C.POINTER(CompileOpts), _vp, C.POINTER(CompileOpts), _vp, _vp]
lib.arso_autotune.restype = C.c_int


def autotune(n, gates, crit, p, n_traj=64, seed=0, precision=C64, stream=None):
    """Measured best (tile_qubits, low_qubits) for a circuit; returns (opts dict, per-candidate ms)."""
    arr, keep = _gates_array(gates)
    c = crit if isinstance(crit, Criterion) else make_criterion(crit)
    base = CompileOpts(precision, 0, 0, 0, 0, 0)
    best = CompileOpts()
    ms = np.zeros(16)
    cnt = C.c_uint32()
    _check(lib.arso_autotune(n, arr, len(gates), C.byref(c), p, n_traj, seed, C.byref(base), _stream(stream),
                             C.byref(best), ms.ctypes.data, C.byref(cnt)))
    return {"tile_qubits": best.tile_qubits, "low_qubits": best.low_qubits}, ms[: cnt.value]


lib.arso_plan_phases.argtypes = [C.c_uint32, C.POINTER(Gate), C.c_size_t, C.POINTER(CompileOpts), C.POINTER(C.c_uint32),
                                 C.POINTER(C.c_uint32)]
lib.arso_plan_phases.restype = C.c_int


lib.arso_plan_tensor_phase.argtypes = [C.c_uint32, C.POINTER(Gate), C.c_size_t, C.POINTER(CompileOpts), C.c_uint32,
                                       C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                       C.POINTER(C.c_uint32), _vp, C.c_uint32, _vp, C.POINTER(C.c_uint32)]
lib.arso_plan_tensor_phase.restype = C.c_int


def plan_tensor_phase(n, gates, phase, tile_qubits=0, low_qubits=0, flags=OPT_TENSOR_PHASES):
    """Host-only (see include/arso.h): a register phase's register bits, engine-position
    range, pass, per-gate roles and, when it runs on the tensor cores, its operand image
    (8192 binary16 values: hi then lo)."""
    arr, keep = _gates_array(gates)
    opts = CompileOpts(C64, tile_qubits, low_qubits, 0, 0, flags)
    rb, pb, pe, ps, has = (C.c_uint32() for _ in range(5))
    roles = np.zeros(max(len(gates), 1), dtype=np.uint8)
    image = np.zeros(8192, dtype=np.uint16)
    _check(lib.arso_plan_tensor_phase(n, arr, len(gates), C.byref(opts), phase, C.byref(rb), C.byref(pb),
                                      C.byref(pe), C.byref(ps), roles.ctypes.data, roles.size,
                                      image.ctypes.data, C.byref(has)))
    R = [(rb.value >> (5 * b)) & 31 for b in range(5)]
    return {"R": R, "pos": (pb.value, pe.value), "pass": ps.value, "roles": roles[: pe.value - pb.value].copy(),
            "image": image if has.value else None}


def plan_phases(n, gates, precision=C64, tile_qubits=0, low_qubits=0, flags=0, tensor=False):
    """Host-only: number of register-bit phases the compile step plans (with
    tensor=True, the pair (phases, phases on the tensor cores))."""
    arr, keep = _gates_array(gates)
    opts = CompileOpts(precision, tile_qubits, low_qubits, 0, 0, flags)
    out, nt = C.c_uint32(), C.c_uint32()
    _check(lib.arso_plan_phases(n, arr, len(gates), C.byref(opts), C.byref(out), C.byref(nt)))
    return (out.value, nt.value) if tensor else out.value
