"""FP64 CPU oracle for the POD / TSQR-SVD path (pyLOM, arXiv 2405.15529).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg (and its ``--impl reference`` arm) may import
this module.  It shares no code with the CUDA library and never imports it.

The numerical work is in ``oracle.c`` (plain C, binary64); this module only
builds and loads it and marshals numpy arrays (Fortran order = column-major).
Each wrapper names the section of the paper its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        # a test that plants a mistake in a copy of oracle.c points this at
        # the mutated build to show that the pins catch it
        override = os.environ.get("PYLOM_ORACLE_LIB")
        if override:
            lib = ctypes.CDLL(override)
        else:
            build()
            lib = ctypes.CDLL(_LIB)
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_center_weight.argtypes = [_dp, _i64, _i64, _i64, _dp, ctypes.c_int, _dp, _i64, _dp]
        lib.oracle_householder_qr.argtypes = [_dp, _i64, _i64, _i64, _dp]
        lib.oracle_apply_q.argtypes = [_dp, _i64, _i64, _i64, _dp, _dp, _i64, _i64]
        lib.oracle_jacobi_svd.argtypes = [_dp, _i64, _i64, _i64, _dp, _dp, _i64, ctypes.c_int]
        lib.oracle_jacobi_svd.restype = ctypes.c_int
        lib.oracle_svd_jacobi_sorted.argtypes = [_dp, _i64, _i64, _i64, _dp, _dp, _i64, ctypes.c_int]
        lib.oracle_svd_jacobi_sorted.restype = ctypes.c_int
        lib.oracle_truncation_rank.argtypes = [_dp, _i64, ctypes.c_double, _i64]
        lib.oracle_truncation_rank.restype = _i64
        lib.oracle_pod.argtypes = [_dp, _i64, _i64, _i64, _dp, ctypes.c_int, ctypes.c_double, _i64,
                                   ctypes.c_int, _dp, _i64, _dp, _dp, _i64, _dp,
                                   ctypes.POINTER(_i64), ctypes.c_int]
        lib.oracle_pod.restype = ctypes.c_int
        lib.oracle_tsqr.argtypes = [_dp, _i64, _i64, _i64, _dp, _i64, _dp, _i64]
        lib.oracle_matmul.argtypes = [ctypes.c_int, _dp, _dp, _dp, _i64, _i64, _i64, _i64, _i64, _i64]
        lib.oracle_pod_loss_grad.argtypes = [_dp, _i64, _i64, _i64, _dp, ctypes.c_int, _i64, _dp, _i64]
        lib.oracle_pod_loss_grad.restype = ctypes.c_double
        lib.oracle_zsvd.argtypes = [ctypes.c_void_p, _i64, _i64, _i64, _i64, ctypes.c_void_p, _i64, _dp,
                                    ctypes.c_void_p, _i64, ctypes.c_int]
        lib.oracle_zsvd.restype = ctypes.c_int
        lib.oracle_zhouseholder_qr.argtypes = [ctypes.c_void_p, _i64, _i64, _i64, ctypes.c_void_p]
        _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _p(a):
    return None if a is None else a.ctypes.data_as(_dp)


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def center_weight(X, w=None, remove_mean=True):
    """Y_w = diag(sqrt w)(X - xbar 1^T) and xbar (Alg. 2 mean removal)."""
    X = _f64(X)
    N, M = X.shape
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    Y = np.zeros((N, M), dtype=np.float64, order="F")
    mean = np.zeros(N, dtype=np.float64)
    _load().oracle_center_weight(_p(X), N, M, N, _p(wv), int(bool(remove_mean)), _p(Y), N, _p(mean))
    return Y, mean


def householder_qr(A):
    """Unblocked Householder QR (Eq. svdqr1): returns (packed, tau)."""
    A = _f64(A).copy(order="F")
    n, m = A.shape
    tau = np.zeros(m, dtype=np.float64)
    _load().oracle_householder_qr(_p(A), n, m, n, _p(tau))
    return A, tau


def apply_q(packed, tau, C):
    """Q C for the reflectors of householder_qr."""
    packed = _f64(packed)
    C = _f64(C).copy(order="F")
    n, m = packed.shape
    k = C.shape[1]
    _load().oracle_apply_q(_p(packed), n, m, n, _p(np.ascontiguousarray(tau)), _p(C), k, n)
    return C


def jacobi_svd_raw(A, max_sweeps=60):
    """One-sided Jacobi (unsorted): returns (A_rot, S, V, sweeps)."""
    A = _f64(A).copy(order="F")
    n, m = A.shape
    S = np.zeros(m)
    V = np.zeros((m, m), order="F")
    sw = _load().oracle_jacobi_svd(_p(A), n, m, n, _p(S), _p(V), m, max_sweeps)
    return A, S, V, sw


def svd(A, max_sweeps=60):
    """Sorted, sign-fixed SVD A = U diag(S) V^T of an n x m (n >= m) matrix by
    one-sided Jacobi (Eq. svdqr2 applied to R).  Returns (U, S, V, sweeps)."""
    A = _f64(A).copy(order="F")
    n, m = A.shape
    S = np.zeros(m)
    V = np.zeros((m, m), order="F")
    sw = _load().oracle_svd_jacobi_sorted(_p(A), n, m, n, _p(S), _p(V), m, max_sweeps)
    return A, S, V, sw


def truncation_rank(S, energy, r_max):
    """Smallest r whose cumulative energy reaches ``energy`` (Sec. 3.1)."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    return int(_load().oracle_truncation_rank(_p(S), S.shape[0], float(energy), int(r_max)))


def pod(X, w=None, remove_mean=True, energy=0.0, r_max=None, mode_kind=0, max_sweeps=60):
    """POD of Alg. 2 via Eqs. svdqr1-svdqr3 (no tree, no blocking).

    Returns dict(U (N x r), S (M), VT (M x M), mean (N), r, sweeps)."""
    X = _f64(X)
    N, M = X.shape
    if r_max is None:
        r_max = M
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    U = np.zeros((N, r_max), dtype=np.float64, order="F")
    S = np.zeros(M)
    VT = np.zeros((M, M), order="F")
    mean = np.zeros(N)
    r = _i64(0)
    sw = _load().oracle_pod(_p(X), N, M, N, _p(wv), int(bool(remove_mean)), float(energy), int(r_max),
                            int(mode_kind), _p(U), N, _p(S), _p(VT), M, _p(mean), ctypes.byref(r),
                            int(max_sweeps))
    return dict(U=U[:, : r.value].copy(order="F"), S=S, VT=VT, mean=mean, r=int(r.value), sweeps=sw)


def tsqr(A, want_q=True):
    """Alg. 1's result by definition: (R, Q) of the Householder QR."""
    A = _f64(A)
    N, M = A.shape
    R = np.zeros((M, M), order="F")
    Q = np.zeros((N, M), order="F") if want_q else None
    _load().oracle_tsqr(_p(A), N, M, N, _p(R), M, _p(Q), N)
    return R, Q


def matmul(A, B, transA=False):
    """Alg. 4's local product C = op(A) B."""
    A = _f64(A)
    B = _f64(B)
    if transA:
        k, m = A.shape
    else:
        m, k = A.shape
    n = B.shape[1]
    C = np.zeros((m, n), order="F")
    _load().oracle_matmul(int(bool(transA)), _p(A), _p(B), _p(C), m, n, k, A.shape[0], B.shape[0], m)
    return C


def pod_loss_grad(X, r, w=None, remove_mean=False, want_grad=True):
    """Truncated-POD reconstruction loss L = sum_{i>r} s_i^2 of Y_w and its
    closed-form gradient dL/dX (valid where s_r > s_{r+1})."""
    X = _f64(X)
    N, M = X.shape
    wv = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    G = np.zeros((N, M), order="F") if want_grad else None
    L = _load().oracle_pod_loss_grad(_p(X), N, M, N, _p(wv), int(bool(remove_mean)), int(r), _p(G), N)
    return float(L), G


def zsvd(X, k=None, max_sweeps=60):
    """Complex SVD X = U diag(S) V^H (binary64) by Householder QR and one-sided
    Jacobi (the per-frequency SVD of SPOD, Alg. 6).  Returns (U (N x k), S, V,
    sweeps) with the phase rule: the largest |entry| of each v_i is real > 0."""
    X = np.asfortranarray(np.asarray(X, dtype=np.complex128))
    N, M = X.shape
    k = M if k is None else int(k)
    U = np.zeros((N, max(k, 1)), dtype=np.complex128, order="F")
    S = np.zeros(M)
    V = np.zeros((M, M), dtype=np.complex128, order="F")
    sw = _load().oracle_zsvd(X.ctypes.data, N, M, N, k, U.ctypes.data, N, _p(S), V.ctypes.data, M,
                             int(max_sweeps))
    return U[:, :k], S, V, sw


def zhouseholder_qr(A):
    """Complex Householder QR (packed reflectors + R, tau)."""
    A = np.asfortranarray(np.asarray(A, dtype=np.complex128)).copy(order="F")
    n, m = A.shape
    tau = np.zeros(m, dtype=np.complex128)
    _load().oracle_zhouseholder_qr(A.ctypes.data, n, m, n, tau.ctypes.data)
    return A, tau
