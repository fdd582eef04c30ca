"""CPU oracle for the two-stage Hessenberg-triangular reduction (Steel & Vandebril).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it to check and time the GPU library.  The GPU library never imports it.

The arithmetic lives in ``hts_oracle_body.inc`` (plain C, compiled into ``liboracle.so``);
this module only marshals numpy arrays.  Every routine follows the paper's algorithm text:

* ``stage0``  -- QR of B (Section "Experiments": B is QR-factorised first; Alg. 1 requires
  B upper triangular).
* ``stage1``  -- Alg. 1, blocked reduction to r-Hessenberg-triangular form, with every
  reflector applied on its own.
* ``stage2``  -- Alg. 2, unblocked reduction of an r-HT pencil to HT form.
* ``reduce``  -- stage0 + stage1 (n_b = r) + stage2.

All routines take and return Fortran-ordered arrays; ``precision='d'`` runs in FP64,
``precision='ld'`` in the platform's C ``long double`` (80-bit on x86-64, binary128 on
AArch64).  Q and Z are returned so that A_in = Q H Z^T and B_in = Q T Z^T.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "hts_oracle.c"), os.path.join(_HERE, "hts_oracle_body.inc")]
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C, OpenMP, no FP contraction)."""
    stale = not os.path.exists(_LIB_PATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in _SOURCES)
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               _SOURCES[0], "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    for suf, ct in (("d", ctypes.c_double), ("ld", ctypes.c_longdouble)):
        p = ctypes.POINTER(ct)
        getattr(lib, "oracle_larfg_" + suf).restype = ct
        getattr(lib, "oracle_larfg_" + suf).argtypes = [ctypes.c_int, p, p, ctypes.c_ssize_t]
        getattr(lib, "oracle_stage0_" + suf).argtypes = [ctypes.c_int, p, ctypes.c_int, p, ctypes.c_int,
                                                         p, ctypes.c_int]
        getattr(lib, "oracle_stage1_" + suf).argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                         p, ctypes.c_int, p, ctypes.c_int,
                                                         p, ctypes.c_int, p, ctypes.c_int]
        getattr(lib, "oracle_stage2_" + suf).argtypes = [ctypes.c_int, ctypes.c_int,
                                                         p, ctypes.c_int, p, ctypes.c_int,
                                                         p, ctypes.c_int, p, ctypes.c_int, ctypes.c_long]
    lib.oracle_threads.restype = ctypes.c_int
    lib.oracle_ldbl_mant_dig.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


@contextlib.contextmanager
def using_library(path):
    """Run the wrappers against another build of the oracle source (used by the tests that
    plant mistakes in a copy of the oracle and check that the pins catch them)."""
    global _lib
    old = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = old


def _dtype(precision):
    if precision == "d":
        return np.float64, ctypes.c_double
    if precision == "ld":
        return np.longdouble, ctypes.c_longdouble
    raise ValueError("precision must be 'd' or 'ld'")


def _arr(M, dt):
    return np.array(M, dtype=dt, order="F", copy=True)


def _ptr(M, ct):
    if M is None:
        return None
    return M.ctypes.data_as(ctypes.POINTER(ct))


def _ld(M):
    return max(1, M.shape[0])


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return _load().oracle_threads()


def ldbl_mant_dig() -> int:
    return _load().oracle_ldbl_mant_dig()


def larfg(x, precision="d"):
    """Householder reflector for vector x: returns (beta, v, tau) with v[0] = 1 and
    (I - tau v v^T) x = beta e_1."""
    dt, ct = _dtype(precision)
    x = np.array(x, dtype=dt).copy()
    m = x.size
    alpha = ct(x[0])
    rest = np.ascontiguousarray(x[1:]) if m > 1 else np.zeros(1, dtype=dt)
    tau = getattr(_load(), "oracle_larfg_" + precision)(m, ctypes.byref(alpha), _ptr(rest, ct), 1)
    v = np.ones(m, dtype=dt)
    if m > 1:
        v[1:] = rest[: m - 1]
    return dt(alpha.value), v, dt(tau)


def stage0(A, B, Q=None, precision="d"):
    """QR of B: returns (A', R, Q') with A' = Q0^T A, R = Q0^T B, Q' = Q Q0 (Q defaults to I)."""
    dt, ct = _dtype(precision)
    n = A.shape[0]
    A, B = _arr(A, dt), _arr(B, dt)
    Q = np.eye(n, dtype=dt, order="F") if Q is None else _arr(Q, dt)
    getattr(_load(), "oracle_stage0_" + precision)(n, _ptr(A, ct), _ld(A), _ptr(B, ct), _ld(B),
                                                   _ptr(Q, ct), _ld(Q))
    return A, B, Q


def stage1(A, B, nb, p=8, Q=None, Z=None, accumulate=True, precision="d"):
    """Alg. 1 on (A, B) with B upper triangular: returns (A', B', Q', Z') in r-HT form, r = nb."""
    dt, ct = _dtype(precision)
    n = A.shape[0]
    A, B = _arr(A, dt), _arr(B, dt)
    if accumulate:
        Q = np.eye(n, dtype=dt, order="F") if Q is None else _arr(Q, dt)
        Z = np.eye(n, dtype=dt, order="F") if Z is None else _arr(Z, dt)
    else:
        Q = Z = None
    getattr(_load(), "oracle_stage1_" + precision)(
        n, nb, p, _ptr(A, ct), _ld(A), _ptr(B, ct), _ld(B),
        _ptr(Q, ct), _ld(Q) if Q is not None else 1, _ptr(Z, ct), _ld(Z) if Z is not None else 1)
    return A, B, Q, Z


def stage2(A, B, r, Q=None, Z=None, accumulate=True, precision="d", max_half_steps=-1):
    """Alg. 2 on an r-HT pencil: returns (H, T, Q', Z').  ``max_half_steps`` >= 0 stops early."""
    dt, ct = _dtype(precision)
    n = A.shape[0]
    A, B = _arr(A, dt), _arr(B, dt)
    if accumulate:
        Q = np.eye(n, dtype=dt, order="F") if Q is None else _arr(Q, dt)
        Z = np.eye(n, dtype=dt, order="F") if Z is None else _arr(Z, dt)
    else:
        Q = Z = None
    getattr(_load(), "oracle_stage2_" + precision)(
        n, r, _ptr(A, ct), _ld(A), _ptr(B, ct), _ld(B),
        _ptr(Q, ct), _ld(Q) if Q is not None else 1, _ptr(Z, ct), _ld(Z) if Z is not None else 1,
        int(max_half_steps))
    return A, B, Q, Z


def reduce(A, B, r, p=8, precision="d"):
    """Full two-stage reduction of a dense pencil: QR(B), Alg. 1 with n_b = r, Alg. 2."""
    A1, B1, Q = stage0(A, B, precision=precision)
    A2, B2, Q, Z = stage1(A1, B1, r, p, Q=Q, precision=precision)
    return stage2(A2, B2, r, Q=Q, Z=Z, precision=precision)
