"""Python binding of the GB300 state-vector library (``libqsgb300.so``).

Argument marshalling only: every step on a state runs in the library's CUDA
kernels. The ``qs_*`` functions here mirror the C ABI in
``include/qsim_gb300.h`` one to one; ``State``, ``Plan`` and ``Expval``
(a ``torch.autograd.Function`` whose backward is the library's adjoint
gradient) are conveniences over them.

The library is built in-tree by ``paper_2509_04955_gb300.build.build()``;
importing this package never compiles anything, and there is no CPU path: a
missing library or a missing GPU raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsgb300.so")

QS_OK, QS_ERR_ARG, QS_ERR_OOM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
QS_C64, QS_C128 = 0, 1
QS_MODE_PER_GATE, QS_MODE_FUSED, QS_MODE_TENSOR, QS_MODE_SMGP = 0, 1, 2, 3
KIND = {"h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8, "rx": 9, "ry": 10,
        "rz": 11, "p": 12, "u1": 13, "swap": 14, "u2": 15}
DTYPES = {"c64": QS_C64, "c128": QS_C128, "complex64": QS_C64, "complex128": QS_C128}
NP_DTYPE = {QS_C64: np.complex64, QS_C128: np.complex128}


class QsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qs status {status}: {msg}")
        self.status = status


class QsGate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nq", C.c_int32), ("q", C.c_int32 * 2), ("nctrl", C.c_int32),
                ("ctrl", C.c_int32 * 2), ("param_index", C.c_int32), ("param", C.c_double),
                ("scale", C.c_double), ("mat", C.c_double * 32)]


class QsPauliTerm(C.Structure):
    _fields_ = [("coeff", C.c_double), ("xmask", C.c_uint64), ("zmask", C.c_uint64)]


class QsPlanOpts(C.Structure):
    _fields_ = [("mode", C.c_int32), ("fuse_k", C.c_int32), ("tile_qubits", C.c_int32),
                ("low_qubits", C.c_int32), ("paper_mode", C.c_int32), ("tc_precision", C.c_int32),
                ("threads", C.c_int32), ("fuse_parametric", C.c_int32), ("reserved", C.c_int32 * 8)]


class QsPlanInfo(C.Structure):
    _fields_ = [("gates", C.c_int64), ("blocks", C.c_int64), ("passes", C.c_int64), ("launches", C.c_int64),
                ("sweeps", C.c_double), ("per_gate_sweeps", C.c_double), ("flops_per_amp", C.c_double),
                ("max_block_qubits", C.c_int32), ("tile_qubits", C.c_int32), ("low_qubits", C.c_int32),
                ("reserved", C.c_int32 * 5)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}
        d["bulk_tile_passes"] = self.reserved[0]
        return d


class QsStreamInfo(C.Structure):
    _fields_ = [("passes", C.c_int64), ("groups", C.c_int64), ("copies", C.c_int64), ("bytes_h2d", C.c_double),
                ("bytes_d2h", C.c_double), ("device_bytes", C.c_double), ("reserved", C.c_int64 * 4)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


_VP, _I64P, _I32P, _DP = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)

# name -> (restype, argtypes)
_SIGS = {
    "qs_state_alloc": (C.c_int, [C.c_int, C.c_int, _VP, C.POINTER(_VP)]),
    "qs_state_wrap": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.POINTER(_VP)]),
    "qs_state_free": (C.c_int, [_VP]),
    "qs_state_info": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(_VP)]),
    "qs_state_set_stream": (C.c_int, [_VP, _VP]),
    "qs_state_set_basis": (C.c_int, [_VP, C.c_uint64]),
    "qs_state_copy_from_host": (C.c_int, [_VP, _VP, C.c_size_t]),
    "qs_state_copy_to_host": (C.c_int, [_VP, _VP, C.c_size_t]),
    "qs_state_copy": (C.c_int, [_VP, _VP]),
    "qs_state_get_amplitudes": (C.c_int, [_VP, C.POINTER(C.c_uint64), C.c_size_t, _VP]),
    "qs_plan_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(QsGate), C.c_size_t, C.POINTER(QsPlanOpts),
                                 C.POINTER(_VP)]),
    "qs_plan_info_get": (C.c_int, [_VP, C.POINTER(QsPlanInfo)]),
    "qs_plan_free": (C.c_int, [_VP]),
    "qs_plan_execute": (C.c_int, [_VP, _VP, _DP, C.c_size_t]),
    "qs_plan_autotune": (C.c_int, [_VP, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t, C.POINTER(QsPlanOpts), _DP]),
    "qs_apply_circuit": (C.c_int, [_VP, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t, C.POINTER(QsPlanOpts)]),
    "qs_norm": (C.c_int, [_VP, _DP]),
    "qs_expval_pauli_sum": (C.c_int, [_VP, C.POINTER(QsPauliTerm), C.c_size_t, _DP]),
    "qs_apply_pauli_sum": (C.c_int, [_VP, C.POINTER(QsPauliTerm), C.c_size_t, _VP]),
    "qs_inner": (C.c_int, [_VP, _VP, _DP, _DP]),
    "qs_state_diff": (C.c_int, [_VP, _VP, _DP, _DP]),
    "qs_adjoint_grad": (C.c_int, [_VP, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t, C.POINTER(QsPauliTerm),
                                  C.c_size_t, _DP, _DP]),
    "qs_adjoint_grad_opts": (C.c_int, [_VP, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t, C.POINTER(QsPauliTerm),
                                       C.c_size_t, C.POINTER(QsPlanOpts), _DP, _DP]),
    "qs_plan_execute_batched": (C.c_int, [_VP, C.POINTER(_VP), C.c_int, _DP, C.c_size_t, C.POINTER(QsPauliTerm),
                                          C.c_size_t, _DP]),
    "qs_plan_check_device_blocks": (C.c_int, [_VP, _VP, _DP, C.c_size_t, _DP, _I64P]),
    "qs_plan_op_count": (C.c_int, [_VP, _I64P, _I64P]),
    "qs_plan_op_get": (C.c_int, [_VP, C.c_int64, _I32P, _I32P, _I32P, _I32P, _DP]),
    "qs_plan_pass_get": (C.c_int, [_VP, C.c_int64, _I32P, _I32P, _I64P, _I64P]),
    "qs_plan_execute_host": (C.c_int, [_VP, C.POINTER(_VP), C.c_int, C.POINTER(_VP), C.POINTER(_VP), C.c_int, _DP,
                                       C.c_size_t, _DP]),
    "qs_stream_apply": (C.c_int, [_VP, C.c_int, C.c_int, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t,
                                  C.POINTER(QsPlanOpts), C.c_int, C.c_int, C.POINTER(QsStreamInfo)]),
    "qs_stream_plan": (C.c_int, [C.c_int, C.POINTER(QsGate), C.c_size_t, C.c_int, C.c_int, _I64P,
                                 C.POINTER(C.c_uint64), _I64P, C.c_int64, _I32P]),
    "qs_plan_phase_terms": (C.c_int, [_VP, C.c_int64, C.POINTER(C.c_uint64), _I32P, _DP, _DP, C.c_int64, _I64P]),
    "qs_plan_set_timing": (C.c_int, [_VP, C.c_int]),
    "qs_plan_timing_read": (C.c_int, [_VP, _DP, _I64P]),
    "qs_plan_timing_read_kinds": (C.c_int, [_VP, _DP, _I64P, _DP, _I64P]),
    "qs_expval_pauli_sum_noalloc": (C.c_int, [_VP, C.c_int, C.c_int, _VP, C.POINTER(QsPauliTerm), C.c_size_t,
                                              _DP]),
    "qs_apply_circuit_batched": (C.c_int, [C.POINTER(_VP), C.c_int, C.POINTER(QsGate), C.c_size_t, _DP, C.c_size_t,
                                           C.POINTER(QsPlanOpts)]),
    "qs_tune_cache_lookup": (C.c_int, [C.c_int, C.c_int, C.POINTER(QsGate), C.c_size_t, C.POINTER(QsPlanOpts), _DP,
                                       C.POINTER(C.c_int)]),
    "qs_tune_cache_put": (C.c_int, [C.c_int, C.c_int, C.POINTER(QsGate), C.c_size_t, C.POINTER(QsPlanOpts),
                                    C.c_double]),
    "qs_tune_cache_save": (C.c_int, [C.c_char_p, _I64P]),
    "qs_tune_cache_load": (C.c_int, [C.c_char_p, _I64P]),
    "qs_tune_cache_clear": (C.c_int, []),
    "qs_last_error": (C.c_char_p, []),
    "qs_launch_count": (C.c_int64, []),
    "qs_plan_set_wait_limit": (C.c_int, [_VP, C.c_uint32]),
    "qs_device_alloc_count": (C.c_int64, []),
    "qs_version": (C.c_char_p, []),
}

_lib = None


def lib():
    """Loads the in-tree library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2509_04955_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGS)


def _check(status: int):
    if status != QS_OK:
        raise QsError(status, lib().qs_last_error().decode(errors="replace"))


# ---------------------------------------------------------------- marshalling

def pack_gates(gates) -> C.Array:
    arr = (QsGate * max(1, len(gates)))()
    for k, g in enumerate(gates):
        o = arr[k]
        o.kind = KIND[g.kind]
        o.nq = len(g.targets)
        for j, q in enumerate(g.targets[:2]):
            o.q[j] = q
        o.nctrl = len(g.controls)           # the library rejects more than two
        for j, q in enumerate(g.controls[:2]):
            o.ctrl[j] = q
        o.param_index = g.param_index
        o.param = g.angle
        o.scale = g.scale
        if g.matrix is not None:
            m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
            for j, v in enumerate(m):
                o.mat[2 * j] = v.real
                o.mat[2 * j + 1] = v.imag
    return arr


def pack_terms(coeff, xmask, zmask) -> C.Array:
    n = len(coeff)
    arr = (QsPauliTerm * max(1, n))()
    for j in range(n):
        arr[j].coeff = float(coeff[j])
        arr[j].xmask = int(xmask[j])
        arr[j].zmask = int(zmask[j])
    return arr


def _dptr(a):
    if a is None:
        return None, 0
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.size


def make_opts(mode=QS_MODE_FUSED, fuse_k=0, tile_qubits=0, low_qubits=0, paper_mode=0, tc_precision=0,
              fuse_parametric=0, tc_min_gates=0, tc_pipeline=0, phase_min_gates=0, c128_pairs=0,
              batch_l2_waves=0, tile_staging=0):
    """qs_plan_opts; tc_min_gates, tc_pipeline, phase_min_gates, c128_pairs and batch_l2_waves fill
    reserved[0..4] (c128_pairs: 0 or 1 = complex128 CUDA-core passes in FP32 pairs, the default;
    2 = in FP64; tile_staging fills reserved[5]: 2 = tile passes staged by bulk copies)."""
    o = QsPlanOpts()
    o.mode, o.fuse_k, o.tile_qubits, o.low_qubits = mode, fuse_k, tile_qubits, low_qubits
    o.paper_mode, o.tc_precision, o.fuse_parametric = paper_mode, tc_precision, fuse_parametric
    o.reserved[0] = tc_min_gates
    o.reserved[1] = tc_pipeline
    o.reserved[2] = phase_min_gates
    o.reserved[3] = c128_pairs
    o.reserved[4] = batch_l2_waves
    o.reserved[5] = tile_staging
    return o


# ---------------------------------------------------------------- C ABI mirrors

def qs_state_alloc(n: int, dtype: int, stream=None) -> int:
    h = _VP()
    _check(lib().qs_state_alloc(n, dtype, stream, C.byref(h)))
    return h.value


def qs_state_wrap(dev_ptr: int, n: int, dtype: int, stream=None) -> int:
    h = _VP()
    _check(lib().qs_state_wrap(dev_ptr, n, dtype, stream, C.byref(h)))
    return h.value


def qs_state_free(h: int):
    _check(lib().qs_state_free(h))


def qs_state_set_basis(h: int, x: int):
    _check(lib().qs_state_set_basis(h, x))


def qs_state_set_stream(h: int, stream):
    _check(lib().qs_state_set_stream(h, stream))


def qs_state_copy_from_host(h: int, arr: np.ndarray):
    arr = np.ascontiguousarray(arr)
    _check(lib().qs_state_copy_from_host(h, arr.ctypes.data, arr.nbytes))


def qs_state_copy_to_host(h: int, out: np.ndarray):
    assert out.flags.c_contiguous
    _check(lib().qs_state_copy_to_host(h, out.ctypes.data, out.nbytes))


def qs_state_copy(dst: int, src: int):
    _check(lib().qs_state_copy(dst, src))


def qs_state_get_amplitudes(h: int, idx, dtype: int) -> np.ndarray:
    """psi[idx] gathered on the device (dtype: the state's QS_C64 / QS_C128)."""
    ix = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(len(ix), dtype=NP_DTYPE[dtype])
    _check(lib().qs_state_get_amplitudes(h, ix.ctypes.data_as(C.POINTER(C.c_uint64)), len(ix), out.ctypes.data))
    return out


def qs_plan_create(n: int, dtype: int, gates, opts: QsPlanOpts | None = None) -> int:
    h = _VP()
    arr = pack_gates(gates)
    _check(lib().qs_plan_create(n, dtype, arr, len(gates), C.byref(opts) if opts is not None else None, C.byref(h)))
    return h.value


def qs_plan_info_get(plan: int) -> dict:
    info = QsPlanInfo()
    _check(lib().qs_plan_info_get(plan, C.byref(info)))
    return info.as_dict()


def qs_plan_free(plan: int):
    _check(lib().qs_plan_free(plan))


def qs_plan_execute(plan: int, state: int, theta=None):
    th, nt = _dptr(theta)
    _check(lib().qs_plan_execute(plan, state, th.ctypes.data_as(_DP) if th is not None else None, nt))


def qs_plan_autotune(state: int, gates, theta=None) -> tuple[QsPlanOpts, float]:
    """Device-timed choice of plan options for this circuit (cached per process)."""
    th, nt = _dptr(theta)
    best = QsPlanOpts()
    ms = C.c_double()
    _check(lib().qs_plan_autotune(state, pack_gates(gates), len(gates),
                                  th.ctypes.data_as(_DP) if th is not None else None, nt, C.byref(best),
                                  C.byref(ms)))
    return best, ms.value


def qs_tune_cache_lookup(n: int, dtype: int, gates):
    """(options, ms) cached for this circuit, or None."""
    o, ms, found = QsPlanOpts(), C.c_double(), C.c_int()
    _check(lib().qs_tune_cache_lookup(n, dtype, pack_gates(gates), len(gates), C.byref(o), C.byref(ms),
                                      C.byref(found)))
    return (o, ms.value) if found.value else None


def qs_tune_cache_put(n: int, dtype: int, gates, opts: QsPlanOpts, ms: float):
    _check(lib().qs_tune_cache_put(n, dtype, pack_gates(gates), len(gates), C.byref(opts), ms))


def qs_tune_cache_save(path: str) -> int:
    cnt = C.c_int64()
    _check(lib().qs_tune_cache_save(os.fsencode(path), C.byref(cnt)))
    return cnt.value


def qs_tune_cache_load(path: str) -> int:
    cnt = C.c_int64()
    _check(lib().qs_tune_cache_load(os.fsencode(path), C.byref(cnt)))
    return cnt.value


def qs_tune_cache_clear():
    _check(lib().qs_tune_cache_clear())


def opts_dict(o: QsPlanOpts) -> dict:
    return {"mode": o.mode, "fuse_k": o.fuse_k, "tile_qubits": o.tile_qubits, "low_qubits": o.low_qubits,
            "tc_min_gates": o.reserved[0], "tc_precision": o.tc_precision, "tc_pipeline": o.reserved[1],
            "phase_min_gates": o.reserved[2], "c128_pairs": o.reserved[3],
            "tile_staging": o.reserved[5]}


def qs_apply_circuit(state: int, gates, theta=None, opts: QsPlanOpts | None = None):
    th, nt = _dptr(theta)
    _check(lib().qs_apply_circuit(state, pack_gates(gates), len(gates),
                                  th.ctypes.data_as(_DP) if th is not None else None, nt,
                                  C.byref(opts) if opts is not None else None))


def _host_ptr(a) -> int:
    """Address of a host buffer: a contiguous numpy array or a (pinned) CPU torch tensor."""
    if hasattr(a, "data_ptr"):
        assert not a.is_cuda and a.is_contiguous()
        return a.data_ptr()
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def qs_stream_apply(host_psi, n: int, dtype: int, gates, theta=None, opts: QsPlanOpts | None = None,
                    batch_qubits: int = 0, pass_qubits: int = 2) -> dict:
    """Applies the circuit to a host-resident state in place, streaming it through
    three device buffers (qs_stream_apply); returns the stream statistics."""
    th, nt = _dptr(theta)
    info = QsStreamInfo()
    _check(lib().qs_stream_apply(_host_ptr(host_psi), n, dtype, pack_gates(gates), len(gates),
                                 th.ctypes.data_as(_DP) if th is not None else None, nt,
                                 C.byref(opts) if opts is not None else None, batch_qubits, pass_qubits,
                                 C.byref(info)))
    return info.as_dict()


def qs_plan_execute_host(plan: int, work: list[int], host_in: list, host_out: list | None = None, theta=None,
                         want_norms: bool = True):
    """Runs the plan on len(host_in) host-resident states through the device states
    `work`, overlapping the copies with the circuit (qs_plan_execute_host); returns
    the norms (or None)."""
    th, nt = _dptr(theta)
    cnt = len(host_in)
    w = (_VP * len(work))(*work)
    hin = (_VP * max(1, cnt))(*[_host_ptr(a) for a in host_in])
    hout = None
    if host_out is not None:
        hout = (_VP * max(1, cnt))(*[_host_ptr(a) if a is not None else None for a in host_out])
    norms = np.zeros(max(1, cnt)) if want_norms else None
    _check(lib().qs_plan_execute_host(plan, w, len(work), hin, hout, cnt,
                                      th.ctypes.data_as(_DP) if th is not None else None, nt,
                                      norms.ctypes.data_as(_DP) if norms is not None else None))
    return norms[:cnt] if want_norms else None


def qs_stream_plan(n: int, gates, batch_qubits: int, pass_qubits: int) -> list[tuple[int, list[int]]]:
    """Streamed passes (host only): (batch-index qubit mask, gate indices in execution order)."""
    cnt = C.c_int64()
    pg = pack_gates(gates)
    _check(lib().qs_stream_plan(n, pg, len(gates), batch_qubits, pass_qubits, C.byref(cnt), None, None, 0, None))
    k = max(1, cnt.value)
    m, e = (C.c_uint64 * k)(), (C.c_int64 * k)()
    order = (C.c_int32 * max(1, len(gates)))()
    _check(lib().qs_stream_plan(n, pg, len(gates), batch_qubits, pass_qubits, C.byref(cnt), m, e, cnt.value, order))
    out, b = [], 0
    for i in range(cnt.value):
        out.append((int(m[i]), [int(order[j]) for j in range(b, e[i])]))
        b = e[i]
    return out


def qs_norm(state: int) -> float:
    v = C.c_double()
    _check(lib().qs_norm(state, C.byref(v)))
    return v.value


def qs_inner(a: int, b: int) -> complex:
    re, im = C.c_double(), C.c_double()
    _check(lib().qs_inner(a, b, C.byref(re), C.byref(im)))
    return complex(re.value, im.value)


def qs_state_diff(a: int, b: int) -> tuple[float, float]:
    m, l2 = C.c_double(), C.c_double()
    _check(lib().qs_state_diff(a, b, C.byref(m), C.byref(l2)))
    return m.value, l2.value


def qs_expval_pauli_sum(state: int, coeff, xmask, zmask) -> float:
    v = C.c_double()
    _check(lib().qs_expval_pauli_sum(state, pack_terms(coeff, xmask, zmask), len(coeff), C.byref(v)))
    return v.value


def qs_state_info(h: int) -> tuple[int, int, int]:
    n, dt, ptr = C.c_int(), C.c_int(), _VP()
    _check(lib().qs_state_info(h, C.byref(n), C.byref(dt), C.byref(ptr)))
    return n.value, dt.value, ptr.value


def qs_expval_pauli_sum_noalloc(dev_state: int, n: int, dtype: int, stream, coeff, xmask, zmask) -> float:
    """<H> of a state given by raw device pointer, with no device allocation
    (for callers that must not allocate; up to 1024 terms)."""
    v = C.c_double()
    _check(lib().qs_expval_pauli_sum_noalloc(dev_state, n, dtype, stream, pack_terms(coeff, xmask, zmask),
                                             len(coeff), C.byref(v)))
    return v.value


def qs_apply_pauli_sum(state: int, coeff, xmask, zmask, out: int):
    _check(lib().qs_apply_pauli_sum(state, pack_terms(coeff, xmask, zmask), len(coeff), out))


def qs_adjoint_grad(state: int, gates, theta, coeff, xmask, zmask, opts: QsPlanOpts | None = None):
    """<H> and its gradient (qs_adjoint_grad, or qs_adjoint_grad_opts when opts is given)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    grad = np.zeros(max(1, th.size))
    e = C.c_double()
    if opts is None:
        _check(lib().qs_adjoint_grad(state, pack_gates(gates), len(gates), th.ctypes.data_as(_DP), th.size,
                                     pack_terms(coeff, xmask, zmask), len(coeff), C.byref(e),
                                     grad.ctypes.data_as(_DP)))
    else:
        _check(lib().qs_adjoint_grad_opts(state, pack_gates(gates), len(gates), th.ctypes.data_as(_DP), th.size,
                                          pack_terms(coeff, xmask, zmask), len(coeff), C.byref(opts), C.byref(e),
                                          grad.ctypes.data_as(_DP)))
    return e.value, grad[: th.size]


def qs_plan_execute_batched(plan: int, states: list[int], theta=None, terms=None):
    B = len(states)
    arr = (_VP * B)(*states)
    th, nt = (None, 0)
    if theta is not None:
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(B, -1)
        nt = th.shape[1]
    ex = np.zeros(B)
    tp, ntm = (None, 0)
    if terms is not None:
        tp, ntm = pack_terms(*terms), len(terms[0])
    _check(lib().qs_plan_execute_batched(plan, arr, B, th.ctypes.data_as(_DP) if th is not None else None, nt,
                                         tp, ntm, ex.ctypes.data_as(_DP) if terms is not None else None))
    return ex if terms is not None else None


def qs_apply_circuit_batched(states: list[int], gates, theta=None, opts: QsPlanOpts | None = None):
    """One-shot: plan, apply to every state with its own theta row, free."""
    B = len(states)
    arr = (_VP * B)(*states)
    th, nt = (None, 0)
    if theta is not None:
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(B, -1)
        nt = th.shape[1]
    _check(lib().qs_apply_circuit_batched(arr, B, pack_gates(gates), len(gates),
                                          th.ctypes.data_as(_DP) if th is not None else None, nt,
                                          C.byref(opts) if opts is not None else None))


def qs_plan_check_device_blocks(plan: int, state: int, theta) -> tuple[float, int]:
    th, nt = _dptr(theta)
    d, nb = C.c_double(), C.c_int64()
    _check(lib().qs_plan_check_device_blocks(plan, state, th.ctypes.data_as(_DP) if th is not None else None, nt,
                                             C.byref(d), C.byref(nb)))
    return d.value, nb.value


def qs_plan_ops(plan: int) -> list[dict]:
    """Ops of a plan in execution order (host only)."""
    n_ops, n_pass = C.c_int64(), C.c_int64()
    _check(lib().qs_plan_op_count(plan, C.byref(n_ops), C.byref(n_pass)))
    out = []
    mat = np.zeros(2 * 4096)
    for i in range(n_ops.value):
        t, nq, gi = C.c_int32(), C.c_int32(), C.c_int32()
        qs = (C.c_int32 * 64)()
        _check(lib().qs_plan_op_get(plan, i, C.byref(t), qs, C.byref(nq), C.byref(gi), mat.ctypes.data_as(_DP)))
        d = {"type": t.value, "qubits": tuple(qs[j] for j in range(nq.value)), "gate": gi.value}
        if t.value == 4:
            d["terms"] = qs_plan_phase_terms(plan, i)
        elif t.value != 0:
            cnt = (1 << nq.value) if t.value == 2 else (1 << (2 * nq.value))
            v = mat[: 2 * cnt].view(np.complex128).copy()
            d["matrix"] = v if t.value == 2 else v.reshape(1 << nq.value, 1 << nq.value)
        out.append(d)
    return out


def qs_plan_passes(plan: int) -> list[dict]:
    n_ops, n_pass = C.c_int64(), C.c_int64()
    _check(lib().qs_plan_op_count(plan, C.byref(n_ops), C.byref(n_pass)))
    out = []
    for i in range(n_pass.value):
        tq = (C.c_int32 * 64)()
        m = C.c_int32()
        b, e = C.c_int64(), C.c_int64()
        _check(lib().qs_plan_pass_get(plan, i, tq, C.byref(m), C.byref(b), C.byref(e)))
        out.append({"tile": tuple(tq[j] for j in range(m.value)), "ops": (b.value, e.value)})
    return out


def qs_plan_phase_terms(plan: int, i: int) -> list[tuple[int, int, float, float]]:
    """Terms (mask, param_index, alpha0, coef) of phase-run op i."""
    cnt = C.c_int64()
    _check(lib().qs_plan_phase_terms(plan, i, None, None, None, None, 0, C.byref(cnt)))
    k = cnt.value
    m = (C.c_uint64 * max(1, k))()
    pi = (C.c_int32 * max(1, k))()
    a0 = np.zeros(max(1, k))
    cf = np.zeros(max(1, k))
    _check(lib().qs_plan_phase_terms(plan, i, m, pi, a0.ctypes.data_as(_DP), cf.ctypes.data_as(_DP), k,
                                     C.byref(cnt)))
    return [(int(m[j]), int(pi[j]), float(a0[j]), float(cf[j])) for j in range(k)]


def qs_plan_set_wait_limit(plan: int, polls: int):
    """Polls per tensor-core pipeline wait before the pass gives up (0 = default)."""
    _check(lib().qs_plan_set_wait_limit(plan, int(polls)))


def qs_plan_set_timing(plan: int, enable: bool):
    _check(lib().qs_plan_set_timing(plan, int(enable)))


def qs_plan_timing_read(plan: int) -> tuple[float, int]:
    ms, n = C.c_double(), C.c_int64()
    _check(lib().qs_plan_timing_read(plan, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def qs_plan_timing_read_kinds(plan: int) -> dict:
    ms, n = C.c_double(), C.c_int64()
    km, kn = (C.c_double * 2)(), (C.c_int64 * 2)()
    _check(lib().qs_plan_timing_read_kinds(plan, C.byref(ms), C.byref(n), km, kn))
    return {"ms": ms.value, "launches": n.value, "tile_ms": km[0], "tile_launches": kn[0], "tc_ms": km[1],
            "tc_launches": kn[1]}


def qs_launch_count() -> int:
    return lib().qs_launch_count()


def qs_device_alloc_count() -> int:
    """Device allocations (cudaMalloc) the library has made in this process."""
    return lib().qs_device_alloc_count()


def qs_version() -> str:
    return lib().qs_version().decode()


# ---------------------------------------------------------------- conveniences

def _torch_stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class State:
    """An n-qubit state in device memory owned by a torch tensor."""

    def __init__(self, n: int, dtype: str = "c64", basis: int | None = 0):
        import torch
        self.n, self.dtype = n, DTYPES[dtype]
        tdt = torch.complex64 if self.dtype == QS_C64 else torch.complex128
        self.tensor = torch.empty(1 << n, dtype=tdt, device="cuda")
        self.handle = qs_state_wrap(self.tensor.data_ptr(), n, self.dtype, _torch_stream())
        if basis is not None:
            qs_state_set_basis(self.handle, basis)

    def free(self):
        if self.handle:
            qs_state_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_basis(self, x: int):
        qs_state_set_basis(self.handle, x)

    def load(self, host: np.ndarray):
        qs_state_copy_from_host(self.handle, np.ascontiguousarray(host, dtype=NP_DTYPE[self.dtype]))

    def to_numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, dtype=NP_DTYPE[self.dtype])
        qs_state_copy_to_host(self.handle, out)
        return out

    def norm(self) -> float:
        return qs_norm(self.handle)

    def amplitudes(self, idx) -> np.ndarray:
        """psi[idx] for a list of basis indices, gathered on the device."""
        return qs_state_get_amplitudes(self.handle, idx, self.dtype)

    def expval(self, coeff, xmask, zmask) -> float:
        return qs_expval_pauli_sum(self.handle, coeff, xmask, zmask)


class Plan:
    def __init__(self, n: int, dtype: str, gates, mode: int = QS_MODE_FUSED, **opts):
        self.n, self.dtype = n, DTYPES[dtype]
        o = None if mode == QS_MODE_PER_GATE and not opts else make_opts(mode=mode, **opts)
        self.handle = qs_plan_create(n, self.dtype, gates, o)

    def info(self) -> dict:
        return qs_plan_info_get(self.handle)

    def ops(self) -> list[dict]:
        return qs_plan_ops(self.handle)

    def passes(self) -> list[dict]:
        return qs_plan_passes(self.handle)

    def execute(self, state: State, theta=None):
        qs_plan_execute(self.handle, state.handle, theta)

    def execute_batched(self, states: list[State], theta=None, terms=None):
        return qs_plan_execute_batched(self.handle, [s.handle for s in states], theta, terms)

    def free(self):
        if self.handle:
            qs_plan_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _make_expval_function():
    import torch

    class Expval(torch.autograd.Function):
        """E(theta) = <psi0| C(theta)^dagger H C(theta) |psi0>; backward is the
        adjoint gradient computed by the library (``qs_adjoint_grad``)."""

        @staticmethod
        def forward(ctx, theta, psi0: State, gates, terms, opts=None):
            th = theta.detach().to("cpu", torch.float64).numpy()
            e, g = qs_adjoint_grad(psi0.handle, gates, th, *terms, opts=opts)
            ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype))
            return theta.new_tensor(e)

        @staticmethod
        def backward(ctx, grad_out):
            (g,) = ctx.saved_tensors
            return grad_out * g.to(grad_out.device), None, None, None, None

    return Expval


_Expval = None


def expval(theta, psi0: State, gates, terms, opts: QsPlanOpts | None = None):
    """Differentiable <H>: ``expval(theta, psi0, gates, (coeff, xmask, zmask))``; ``opts``
    (optional) plans the forward execution and sets the complex128 arithmetic of the
    adjoint sweep (``qs_adjoint_grad_opts``)."""
    global _Expval
    if _Expval is None:
        _Expval = _make_expval_function()
    return _Expval.apply(theta, psi0, gates, terms, opts)
