"""Python access to the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``. The CUDA library never imports it.

``build()`` compiles ``oracle.c`` with gcc into ``liboracle.so`` beside it.
States are numpy complex128 vectors of length 2^n (qubit q = bit q).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_KIND = {"h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8,
         "rx": 9, "ry": 10, "rz": 11, "p": 12, "u1": 13, "swap": 14, "u2": 15}


class OrGate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ntarg", C.c_int32), ("targ", C.c_int32 * 2),
                ("nctrl", C.c_int32), ("ctrl", C.c_int32 * 2), ("param_index", C.c_int32),
                ("angle", C.c_double), ("scale", C.c_double), ("mat", C.c_double * 32)]


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", _SO, src, "-lm"]
        try:   # OpenMP only for the all-cores baseline timing; plain C without it
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
    return _SO


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp, u64p = C.POINTER(C.c_double), C.POINTER(C.c_uint64)
        gp = C.POINTER(OrGate)
        L.or_gate_matrix.argtypes = [gp, dp, dp]
        L.or_gate_matrix.restype = C.c_int
        L.or_gate_dmatrix.argtypes = [gp, dp, dp]
        L.or_gate_dmatrix.restype = C.c_int
        L.or_set_basis.argtypes = [dp, C.c_int, C.c_uint64]
        L.or_set_threads.argtypes = [C.c_int]
        L.or_set_threads.restype = C.c_int
        L.or_apply_gate.argtypes = [dp, C.c_int, gp, dp]
        L.or_apply_gate_adjoint.argtypes = [dp, C.c_int, gp, dp]
        L.or_apply_circuit.argtypes = [dp, C.c_int, gp, C.c_int64, dp]
        L.or_norm2.argtypes = [dp, C.c_int]
        L.or_norm2.restype = C.c_double
        L.or_unitary.argtypes = [C.c_int, gp, C.c_int64, dp, dp]
        L.or_expval.argtypes = [dp, C.c_int, dp, u64p, u64p, C.c_int64, dp]
        L.or_expval.restype = C.c_double
        L.or_apply_pauli_sum.argtypes = [dp, C.c_int, dp, u64p, u64p, C.c_int64, dp]
        L.or_adjoint_grad.argtypes = [dp, C.c_int, gp, C.c_int64, dp, C.c_int64, dp, u64p, u64p,
                                      C.c_int64, dp, dp]
        L.or_adjoint_grad.restype = C.c_int
        _lib = L
    return _lib


def pack(gates) -> C.Array:
    arr = (OrGate * max(1, len(gates)))()
    for k, g in enumerate(gates):
        o = arr[k]
        o.kind = _KIND[g.kind]
        o.ntarg = len(g.targets)
        for j, q in enumerate(g.targets):
            o.targ[j] = q
        o.nctrl = len(g.controls)
        for j, q in enumerate(g.controls):
            o.ctrl[j] = q
        o.param_index = g.param_index
        o.angle = g.angle
        o.scale = g.scale
        if g.matrix is not None:
            m = np.asarray(g.matrix, dtype=np.complex128).reshape(-1)
            for j, v in enumerate(m):
                o.mat[2 * j] = v.real
                o.mat[2 * j + 1] = v.imag
    return arr


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u64p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _theta(theta) -> np.ndarray:
    if theta is None:
        return np.zeros(1)
    t = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
    return t if t.size else np.zeros(1)


def gate_matrix(g, theta=None) -> np.ndarray:
    m = np.zeros(16, dtype=np.complex128)
    d = lib().or_gate_matrix(pack([g]), _dp(_theta(theta)), _dp(m.view(np.float64)))
    return m[: d * d].reshape(d, d)


def gate_dmatrix(g, theta=None) -> np.ndarray:
    m = np.zeros(16, dtype=np.complex128)
    d = lib().or_gate_dmatrix(pack([g]), _dp(_theta(theta)), _dp(m.view(np.float64)))
    return m[: d * d].reshape(d, d)


def basis(n: int, x: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().or_set_basis(_dp(psi.view(np.float64)), n, x)
    return psi


def apply_circuit(psi: np.ndarray, n: int, gates, theta=None) -> np.ndarray:
    """Returns a new state: the circuit applied gate by gate to ``psi``."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    lib().or_apply_circuit(_dp(out.view(np.float64)), n, pack(gates), len(gates), _dp(_theta(theta)))
    return out


def norm2(psi: np.ndarray, n: int) -> float:
    return lib().or_norm2(_dp(np.ascontiguousarray(psi).view(np.float64)), n)


def unitary(n: int, gates, theta=None) -> np.ndarray:
    assert n <= 9
    U = np.empty((1 << n, 1 << n), dtype=np.complex128)
    lib().or_unitary(n, pack(gates), len(gates), _dp(_theta(theta)), _dp(U.view(np.float64)))
    return U


def _terms(coeff, xm, zm):
    return (np.ascontiguousarray(coeff, dtype=np.float64), np.ascontiguousarray(xm, dtype=np.uint64),
            np.ascontiguousarray(zm, dtype=np.uint64))


def expval(psi: np.ndarray, n: int, coeff, xm, zm) -> complex:
    c, x, z = _terms(coeff, xm, zm)
    im = C.c_double(0)
    re = lib().or_expval(_dp(np.ascontiguousarray(psi).view(np.float64)), n, _dp(c), _u64p(x), _u64p(z),
                         len(c), C.byref(im))
    return complex(re, im.value)


def apply_pauli_sum(psi: np.ndarray, n: int, coeff, xm, zm) -> np.ndarray:
    c, x, z = _terms(coeff, xm, zm)
    out = np.empty(1 << n, dtype=np.complex128)
    lib().or_apply_pauli_sum(_dp(np.ascontiguousarray(psi).view(np.float64)), n, _dp(c), _u64p(x),
                             _u64p(z), len(c), _dp(out.view(np.float64)))
    return out


def adjoint_grad(psi0: np.ndarray, n: int, gates, theta, coeff, xm, zm):
    """Returns (expval, grad[len(theta)])."""
    c, x, z = _terms(coeff, xm, zm)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    grad = np.zeros(max(1, th.size))
    e = C.c_double(0)
    rc = lib().or_adjoint_grad(_dp(np.ascontiguousarray(psi0).view(np.float64)), n, pack(gates),
                               len(gates), _dp(_theta(th)), th.size, _dp(c), _u64p(x), _u64p(z),
                               len(c), C.byref(e), _dp(grad))
    if rc != 0:
        raise MemoryError("oracle adjoint: allocation failed")
    return e.value, grad[: th.size]


def expval_of_circuit(psi0, n, gates, theta, coeff, xm, zm) -> float:
    return expval(apply_circuit(psi0, n, gates, theta), n, coeff, xm, zm).real
