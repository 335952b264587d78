"""GB300-native POD / TSQR-SVD (the hot path of pyLOM, arXiv 2405.15529).

Thin Python binding over the C ABI of ``libpylom.so`` (declared in
``include/pylom.h``).  This module only marshals arguments: every step of the
path (mean removal and weights, leaf Householder QR, the tree reduction of
Alg. 1, the Jacobi SVD of R, the top-down pass and U = Q U_r) runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.

There is no CPU fallback: importing works without the library, but every
call raises if ``libpylom.so`` has not been built or no CUDA device exists.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpylom.so")

# pylom_status
OK, ERR_ARG, ERR_SHAPE, ERR_WORKSPACE, ERR_CUDA, ERR_NONFINITE, ERR_NOCONV, ERR_TIMEOUT, \
    ERR_UNSUPPORTED, ERR_SINGULAR = range(10)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_WORKSPACE", 4: "ERR_CUDA",
                5: "ERR_NONFINITE", 6: "ERR_NOCONV", 7: "ERR_TIMEOUT", 8: "ERR_UNSUPPORTED",
                9: "ERR_SINGULAR"}
# pylom_dtype / pylom_prec / pylom_mode_kind
F32, F64, C64, C128 = 0, 1, 2, 3
PREC_FP64, PREC_MIXED_3XTF32 = 0, 1
MODES_ORTHONORMAL, MODES_PHYSICAL = 0, 1

# Every symbol include/pylom.h declares (checked by the tests).
EXPORTS = (
    "pylom_version", "pylom_last_error", "pylom_leaf_count", "pylom_workspace_status",
    "pylom_pod_workspace_size", "pylom_pod", "pylom_tsqr_workspace_size", "pylom_tsqr",
    "pylom_svd_small_workspace_size", "pylom_svd_small", "pylom_matmul_workspace_size",
    "pylom_matmul", "pylom_profile_begin", "pylom_profile_end",
    "pylom_svd_small_noalloc",
    "pylom_pod_backward_workspace_size", "pylom_pod_backward",
    "pylom_svd_batched_plan", "pylom_svd_batched_bind", "pylom_svd_batched_run",
    "pylom_svd_batched_plan_info", "pylom_svd_batched_plan_destroy", "pylom_svd_batched_max_leaf_rows",
    "pylom_svd_batched_bind_items",
    "pylom_spod_shape", "pylom_spod_blocks_workspace_size", "pylom_spod_blocks", "pylom_spod_order",
    "pylom_pod_streamed_workspace_size", "pylom_pod_streamed", "pylom_pod_streamed_leaf_rows",
    "pylom_dmd_workspace_size", "pylom_dmd",
    "pylom_wait_selftest_workspace_size", "pylom_wait_selftest",
    "pylom_pod_shard_workspace_size", "pylom_pod_shard_factor", "pylom_pod_rstack_workspace_size",
    "pylom_pod_rstack", "pylom_pod_shard_modes",
)
PROFILE_PHASES = ("leaf_qr", "tree", "svd_small", "down_pass", "modes")


class PylomError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_int = ctypes.c_int
_dbl = ctypes.c_double


def load_library(path: str = LIB_PATH):
    """Load libpylom.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    lib.pylom_version.restype = ctypes.c_char_p
    lib.pylom_last_error.restype = ctypes.c_char_p
    lib.pylom_leaf_count.restype = _i64
    lib.pylom_leaf_count.argtypes = [_i64, _i64, _i64]
    lib.pylom_workspace_status.restype = _int
    lib.pylom_workspace_status.argtypes = [_vp, _vp, ctypes.POINTER(_i64), ctypes.POINTER(_int)]
    lib.pylom_pod_workspace_size.restype = _sz
    lib.pylom_pod_workspace_size.argtypes = [_i64, _i64, _i64, _i64, _int, _int]
    lib.pylom_pod.restype = _int
    lib.pylom_pod.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _int, _dbl, _i64, _int, _i64,
                              _vp, _i64, _vp, _vp, _i64, _vp, _vp, _int, _vp, _sz, _vp]
    lib.pylom_tsqr_workspace_size.restype = _sz
    lib.pylom_tsqr_workspace_size.argtypes = [_i64, _i64, _i64, _int, _int, _int]
    lib.pylom_tsqr.restype = _int
    lib.pylom_tsqr.argtypes = [_vp, _i64, _i64, _i64, _int, _i64, _vp, _i64, _vp, _i64, _int,
                               _vp, _sz, _vp]
    lib.pylom_svd_small_workspace_size.restype = _sz
    lib.pylom_svd_small_workspace_size.argtypes = [_i64]
    lib.pylom_svd_small.restype = _int
    lib.pylom_svd_small.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _int, _vp, _sz, _vp]
    lib.pylom_matmul_workspace_size.restype = _sz
    lib.pylom_matmul_workspace_size.argtypes = [_i64, _i64, _i64]
    lib.pylom_matmul.restype = _int
    lib.pylom_matmul.argtypes = [_int, _vp, _vp, _vp, _i64, _i64, _i64, _i64, _i64, _i64, _vp, _sz, _vp]
    lib.pylom_profile_begin.restype = _int
    lib.pylom_profile_begin.argtypes = [_int]
    lib.pylom_profile_end.restype = _int
    lib.pylom_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_int)]
    lib.pylom_pod_backward_workspace_size.restype = _sz
    lib.pylom_pod_backward_workspace_size.argtypes = [_i64, _i64, _i64, _i64, _int]
    lib.pylom_pod_backward.restype = _int
    lib.pylom_pod_backward.argtypes = [_vp, _sz, _i64, _i64, _i64, _i64, _i64, _vp, _int, _int, _int, _vp, _vp,
                                       _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _int, _vp, _sz, _vp]
    lib.pylom_spod_shape.restype = _int
    lib.pylom_spod_shape.argtypes = [_i64, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    lib.pylom_spod_blocks_workspace_size.restype = _sz
    lib.pylom_spod_blocks_workspace_size.argtypes = [_i64, _i64]
    lib.pylom_spod_blocks.restype = _int
    lib.pylom_spod_blocks.argtypes = [_vp, _i64, _i64, _i64, _int, _i64, _i64, _int, _vp, _i64, _vp, _vp, _sz, _vp]
    lib.pylom_spod_order.restype = _int
    lib.pylom_pod_streamed_workspace_size.restype = _sz
    lib.pylom_pod_streamed_workspace_size.argtypes = [_i64, _i64, _i64, _i64, _i64, _int]
    lib.pylom_dmd_workspace_size.restype = _sz
    lib.pylom_dmd_workspace_size.argtypes = [_i64, _i64, _i64, _i64, _int]
    lib.pylom_dmd.restype = _int
    lib.pylom_dmd.argtypes = [_vp, _i64, _i64, _i64, _int, _int, _dbl, _i64, _i64, _vp, _vp, _vp, _i64, _vp, _vp,
                              _vp, _vp, _sz, _vp]
    lib.pylom_pod_streamed_leaf_rows.restype = _i64
    lib.pylom_pod_streamed_leaf_rows.argtypes = [_i64, _i64, _i64, _i64]
    lib.pylom_pod_streamed.restype = _int
    lib.pylom_pod_streamed.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _int, _dbl, _i64, _int, _i64, _i64,
                                       _vp, _vp, _i64, _vp, _vp, _i64, _vp, ctypes.POINTER(_i64), _vp, _sz, _vp]
    lib.pylom_spod_order.argtypes = [_vp, _i64, _i64, _vp, _vp]
    lib.pylom_svd_batched_plan.restype = _int
    lib.pylom_svd_batched_plan.argtypes = [_int, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                                           _i64, _int, ctypes.POINTER(_vp), ctypes.POINTER(_sz)]
    lib.pylom_svd_batched_bind.restype = _int
    lib.pylom_svd_batched_bind.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_vp),
                                           ctypes.POINTER(_i64), _vp, _sz, _vp]
    lib.pylom_svd_batched_run.restype = _int
    lib.pylom_svd_batched_run.argtypes = [_vp, _vp, _vp, _int, _vp]
    lib.pylom_svd_batched_plan_info.restype = _i64
    lib.pylom_svd_batched_plan_info.argtypes = [_vp, _int, _int]
    lib.pylom_svd_batched_plan_destroy.restype = None
    lib.pylom_svd_batched_plan_destroy.argtypes = [_vp]
    lib.pylom_svd_small_noalloc.restype = _int
    lib.pylom_svd_small_noalloc.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _int, _vp, _vp]
    lib.pylom_svd_batched_bind_items.restype = _int
    lib.pylom_svd_batched_bind_items.argtypes = [_vp, ctypes.c_void_p, _vp, _sz, _vp]
    lib.pylom_svd_batched_max_leaf_rows.restype = _i64
    lib.pylom_svd_batched_max_leaf_rows.argtypes = [_int]
    lib.pylom_pod_shard_workspace_size.restype = _sz
    lib.pylom_pod_shard_workspace_size.argtypes = [_i64, _i64, _i64, _i64, _int, _int]
    lib.pylom_pod_shard_factor.restype = _int
    lib.pylom_pod_shard_factor.argtypes = [_vp, _i64, _i64, _i64, _int, _vp, _int, _i64, _i64, _vp, _vp, _i64,
                                           _int, _vp, _sz, _vp]
    lib.pylom_pod_rstack_workspace_size.restype = _sz
    lib.pylom_pod_rstack_workspace_size.argtypes = [_i64, _i64, _i64]
    lib.pylom_pod_rstack.restype = _int
    lib.pylom_pod_rstack.argtypes = [_vp, _i64, _i64, _dbl, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _sz, _vp]
    lib.pylom_pod_shard_modes.restype = _int
    lib.pylom_pod_shard_modes.argtypes = [_vp, _vp, _i64, _i64, _i64, _i64, _vp, _int, _vp, _i64, _int, _vp, _sz,
                                          _vp]
    lib.pylom_wait_selftest_workspace_size.restype = _sz
    lib.pylom_wait_selftest_workspace_size.argtypes = []
    lib.pylom_wait_selftest.restype = _int
    lib.pylom_wait_selftest.argtypes = [_int, _int, _dbl, _vp, _vp, _sz, _vp]
    _lib = lib
    return lib


def _raise(status: int, what: str):
    if status != OK:
        msg = load_library().pylom_last_error().decode(errors="replace")
        raise PylomError(status, f"{what}: {msg}")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the POD path runs only on the GPU (no CPU fallback)")
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _colmajor(t):
    """Column-major view of a 2-D tensor (copies only if needed).  Strides of
    size-1 dimensions carry no layout information and are ignored."""
    if t.dim() != 2:
        raise ValueError("expected a 2-D tensor")
    rows, cols = t.shape
    if (rows == 1 or t.stride(0) == 1) and (cols == 1 or t.stride(1) >= rows):
        return t
    return t.t().contiguous().t()


def _ld(t):
    """Leading dimension of a column-major 2-D tensor."""
    rows, cols = t.shape
    return max(1, rows) if cols == 1 else t.stride(1)


def empty_colmajor(rows: int, cols: int, dtype, device):
    torch = _torch()
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _dptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def profile_begin(max_calls: int) -> None:
    _raise(load_library().pylom_profile_begin(int(max_calls)), "pylom_profile_begin")


def profile_end():
    """Summed milliseconds per phase of the profiled pylom_pod calls."""
    arr = (ctypes.c_double * len(PROFILE_PHASES))()
    n = _int(0)
    _raise(load_library().pylom_profile_end(arr, ctypes.byref(n)), "pylom_profile_end")
    out = dict(zip(PROFILE_PHASES, list(arr)))
    out["leaf_qr_tree"] = out["leaf_qr"] + out["tree"]     # the leaves and the whole reduction
    return out, int(n.value)


def wait_selftest(kind: str = "grid", blocks: int = 16, limit_ms: float = 2.0, stream=None):
    """Run one bounded device wait into its limit (pylom_wait_selftest):
    kind 'grid' (the grid barrier) or 'mbarrier' (the tcgen05 commit wait).
    Returns (device status, number of blocks whose waits gave up)."""
    torch = _torch()
    lib = load_library()
    ws = torch.zeros(lib.pylom_wait_selftest_workspace_size(), dtype=torch.uint8, device="cuda")
    gave = torch.zeros(1, dtype=torch.int32, device="cuda")
    _raise(lib.pylom_wait_selftest({"grid": 0, "mbarrier": 1}[kind], int(blocks), float(limit_ms), _dptr(gave),
                                   _dptr(ws), ws.numel(), _stream(stream)), "pylom_wait_selftest")
    st = lib.pylom_workspace_status(_dptr(ws), _stream(stream), None, None)
    return int(st), int(gave.item())


def upload(dst, src, chunk_bytes: int = 256 << 20, stream=None):
    """Host-to-device copy of a page-locked host tensor into a device tensor
    of the same size, issued as one cudaMemcpyAsync per chunk_bytes slice.
    On GB300 one copy of several GB from page-locked memory ran at 20-55
    GB/s while 256 MB pieces ran at 211 GB/s (measured inside the
    benchmark), so large inputs are moved in pieces."""
    torch = _torch()
    if not (dst.is_contiguous() and src.is_contiguous()) or dst.numel() * dst.element_size() != \
            src.numel() * src.element_size():
        raise ValueError("upload needs contiguous tensors of the same size in bytes")
    d = dst.view(-1).view(torch.uint8)
    s = src.view(-1).view(torch.uint8)
    ctx = torch.cuda.stream(stream) if stream is not None else None
    if ctx:
        ctx.__enter__()
    try:
        for o in range(0, d.numel(), chunk_bytes):
            e = min(d.numel(), o + chunk_bytes)
            d[o:e].copy_(s[o:e], non_blocking=True)
    finally:
        if ctx:
            ctx.__exit__(None, None, None)
    return dst


def leaf_count(N: int, M: int, leaf_rows: int = 0) -> int:
    return int(load_library().pylom_leaf_count(N, M, leaf_rows))


def workspace_status(ws, stream=None):
    """(status, r, sweeps) recorded in a workspace; synchronises the stream."""
    r = _i64(0)
    sw = _int(0)
    st = load_library().pylom_workspace_status(_dptr(ws), _stream(stream), ctypes.byref(r), ctypes.byref(sw))
    return st, int(r.value), int(sw.value)


@dataclass
class PodResult:
    U: "torch.Tensor"        # N x r (column-major view)
    S: "torch.Tensor"        # M
    VT: "torch.Tensor"       # M x M
    mean: Optional["torch.Tensor"]
    r: int
    sweeps: int
    workspace: "torch.Tensor"
    prec: int = 0            # PREC_FP64 or PREC_MIXED_3XTF32 (the backward needs it)


def pod_workspace_size(N, M, leaf_rows=0, r_max=None, xtype=F64, prec=PREC_FP64) -> int:
    r_max = M if r_max is None else r_max
    return int(load_library().pylom_pod_workspace_size(N, M, leaf_rows, r_max, xtype, prec))


def pod(X, w=None, remove_mean=True, energy=0.0, r_max=None, mode_kind=MODES_ORTHONORMAL,
        leaf_rows=0, prec=PREC_FP64, workspace=None, out=None, stream=None, check=True) -> PodResult:
    """POD of the N x M snapshot matrix X (Alg. 2 of the paper) on the GPU.

    X: CUDA tensor (float32 or float64), any 2-D layout (column-major used
    as is), or a column-major page-locked host tensor (pin_memory): the leaf
    kernel then reads it across the host link, with no separate upload.
    w: N cell volumes (float64) or None.  Returns U (N x r), S, VT, mean.
    With check=False the call stays asynchronous and U holds r_max columns
    (r is then read later from the workspace)."""
    torch = _torch()
    lib = load_library()
    if X.device.type == "cpu":
        if not (X.is_pinned() and X.dim() == 2 and X.stride(0) == 1 and X.stride(1) >= X.shape[0]):
            raise ValueError("a host X must be a column-major page-locked tensor (e.g. "
                             "torch.empty((M, N), pin_memory=True).t())")
        dev = torch.device("cuda", torch.cuda.current_device())
    else:
        X = _colmajor(X)
        dev = X.device
    N, M = X.shape
    xtype = {torch.float32: F32, torch.float64: F64}.get(X.dtype)
    if xtype is None:
        raise TypeError("X must be float32 or float64")
    r_max = M if r_max is None else int(r_max)
    if w is not None:
        w = w.to(device=dev, dtype=torch.float64).contiguous()
    need = lib.pylom_pod_workspace_size(N, M, leaf_rows, r_max, xtype, prec)
    if need == 0:
        _raise(ERR_SHAPE if prec == PREC_FP64 else ERR_UNSUPPORTED,
               f"pylom_pod_workspace_size(N={N}, M={M}, b={leaf_rows}, r_max={r_max}, prec={prec})")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if out is None:
        U = empty_colmajor(N, r_max, torch.float32 if prec == PREC_MIXED_3XTF32 else torch.float64, dev)
        S = torch.empty(M, dtype=torch.float64, device=dev)
        VT = empty_colmajor(M, M, torch.float64, dev)
        mean = torch.empty(N, dtype=torch.float64, device=dev)
        r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    else:
        U, S, VT, mean, r_dev = out
    st = lib.pylom_pod(_dptr(X), N, M, _ld(X), xtype, _dptr(w), int(bool(remove_mean)),
                       float(energy), r_max, int(mode_kind), int(leaf_rows), _dptr(U), _ld(U),
                       _dptr(S), _dptr(VT), _ld(VT), _dptr(mean), _dptr(r_dev), int(prec),
                       _dptr(workspace), workspace.numel(), _stream(stream))
    _raise(st, "pylom_pod")
    r, sweeps = r_max, -1
    if check:
        st, r, sweeps = workspace_status(workspace, stream)
        _raise(st, "pylom_pod (device)")
        U = U[:, :r]
    return PodResult(U=U, S=S, VT=VT, mean=mean, r=r, sweeps=sweeps, workspace=workspace, prec=int(prec))


@dataclass
class DmdResult:
    mu: "torch.Tensor"          # r complex eigenvalues (sorted)
    b: "torch.Tensor"           # r complex amplitudes
    Phi_packed: "torch.Tensor"  # N x r real (conjugate pairs as Re / Im columns)
    S: "torch.Tensor"           # M-1 singular values of Y1
    mean: Optional["torch.Tensor"]
    r: int
    workspace: "torch.Tensor"

    @property
    def Phi(self):
        """The modes as an N x r complex tensor (a layout change of Phi_packed)."""
        torch = _torch()
        mu = self.mu
        P = self.Phi_packed
        out = torch.empty((P.shape[0], self.r), dtype=torch.complex128, device=P.device)
        p = 0
        im = mu.imag.cpu()
        while p < self.r:
            if im[p] > 0.0:
                out[:, p] = torch.complex(P[:, p], P[:, p + 1])
                out[:, p + 1] = torch.complex(P[:, p], -P[:, p + 1])
                p += 2
            else:
                out[:, p] = torch.complex(P[:, p], torch.zeros_like(P[:, p]))
                p += 1
        return out


def dmd_workspace_size(N, M, leaf_rows=0, r_max=None, xtype=F64) -> int:
    r_max = M - 1 if r_max is None else r_max
    return int(load_library().pylom_dmd_workspace_size(N, M, leaf_rows, r_max, xtype))


def dmd(X, remove_mean=True, energy=0.0, r_max=None, leaf_rows=0, workspace=None, out=None, stream=None,
        check=True) -> DmdResult:
    """Exact DMD of the N x M snapshot matrix X (Alg. 3, amplitudes of
    Alg. 5) on the GPU.  X: CUDA tensor, float32 or float64.  With
    check=False the call stays asynchronous (r is read later from the
    workspace; the outputs then hold r_max entries)."""
    torch = _torch()
    lib = load_library()
    X = _colmajor(X)
    N, M = X.shape
    xtype = {torch.float32: F32, torch.float64: F64}.get(X.dtype)
    if xtype is None:
        raise TypeError("X must be float32 or float64")
    r_max = M - 1 if r_max is None else int(r_max)
    dev = X.device
    need = lib.pylom_dmd_workspace_size(N, M, leaf_rows, r_max, xtype)
    if need == 0:
        _raise(ERR_SHAPE, f"pylom_dmd_workspace_size(N={N}, M={M}, b={leaf_rows}, r_max={r_max})")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    if out is None:
        mu = torch.empty(2 * r_max, dtype=torch.float64, device=dev)
        b = torch.empty(2 * r_max, dtype=torch.float64, device=dev)
        Phi = empty_colmajor(N, r_max, torch.float64, dev)
        S = torch.empty(max(M - 1, 1), dtype=torch.float64, device=dev)
        mean = torch.empty(N, dtype=torch.float64, device=dev)
        r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    else:
        mu, b, Phi, S, mean, r_dev = out
    st = lib.pylom_dmd(_dptr(X), N, M, _ld(X), xtype, int(bool(remove_mean)), float(energy), r_max, int(leaf_rows),
                       _dptr(mu), _dptr(b), _dptr(Phi), _ld(Phi), _dptr(S), _dptr(mean), _dptr(r_dev),
                       _dptr(workspace), workspace.numel(), _stream(stream))
    _raise(st, "pylom_dmd")
    r = r_max
    if check:
        st, r, _ = workspace_status(workspace, stream)
        _raise(st, "pylom_dmd (device)")
    muc = torch.view_as_complex(mu.view(-1, 2))[:r]
    bc = torch.view_as_complex(b.view(-1, 2))[:r]
    return DmdResult(mu=muc, b=bc, Phi_packed=Phi[:, :r], S=S, mean=mean if remove_mean else None, r=r,
                     workspace=workspace)


def pod_streamed_leaf_rows(N, M, leaf_rows=0, chunk_rows=1 << 22) -> int:
    """Leaf height of a streamed POD call (its results equal pod() with this leaf_rows)."""
    return int(load_library().pylom_pod_streamed_leaf_rows(N, M, leaf_rows, chunk_rows))


@dataclass
class StreamedPodResult:
    U: "torch.Tensor"        # host N x r (column-major view of page-locked memory)
    S: "torch.Tensor"        # device, M
    VT: "torch.Tensor"       # device, M x M
    mean: Optional["torch.Tensor"]   # host, N
    r: int
    workspace: "torch.Tensor"


def _pinned_colmajor(A, dtype=None):
    """A host column-major copy in page-locked memory (no copy if A already is one)."""
    torch = _torch()
    if not torch.is_tensor(A):
        A = torch.as_tensor(A)
    if dtype is not None and A.dtype != dtype:
        A = A.to(dtype)
    if A.device.type != "cpu":
        raise ValueError("the streamed POD takes X in host memory")
    if A.dim() != 2:
        raise ValueError("expected a 2-D array")
    rows, cols = A.shape
    if (rows == 1 or A.stride(0) == 1) and (cols == 1 or A.stride(1) >= rows) and A.is_pinned():
        return A
    out = torch.empty((A.shape[1], A.shape[0]), dtype=A.dtype, pin_memory=True).t()
    out.copy_(A)
    return out


def pod_streamed(X, w=None, remove_mean=True, energy=0.0, r_max=None, mode_kind=MODES_ORTHONORMAL,
                 leaf_rows=0, chunk_rows=1 << 22, device=None, stream=None, workspace=None, host_scratch=None,
                 out=None):
    """POD (binary64 path) of an N x M snapshot matrix held in HOST memory,
    streamed through the device in chunks of whole leaves of about
    chunk_rows rows; the modes come back to host memory.  Same results as
    pod() with the same leaf partition.  X: float32/float64 numpy array or
    CPU tensor (copied to page-locked memory unless it already is).
    host_scratch: page-locked float64 host tensor of at least N*M entries
    (the leaves' reflectors between the passes); out: a page-locked
    column-major float64 host tensor of N x >= r_max for the modes.  Both
    are allocated per call when None (page-locking 2 N M doubles is slow:
    pass them in for repeated calls)."""
    torch = _torch()
    lib = load_library()
    X = _pinned_colmajor(X)
    N, M = X.shape
    xtype = {torch.float32: F32, torch.float64: F64}.get(X.dtype)
    if xtype is None:
        raise TypeError("X must be float32 or float64")
    r_max = M if r_max is None else int(r_max)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if w is not None:
        w = _pinned_colmajor(torch.as_tensor(w).to(torch.float64).reshape(-1, 1)).reshape(-1)
    need = lib.pylom_pod_streamed_workspace_size(N, M, leaf_rows, chunk_rows, r_max, xtype)
    if need == 0:
        _raise(ERR_SHAPE, f"pylom_pod_streamed_workspace_size(N={N}, M={M}, b={leaf_rows}, "
                          f"chunk={chunk_rows}, r_max={r_max})")
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    Yh = host_scratch
    if Yh is None:
        Yh = torch.empty(N * M, dtype=torch.float64, pin_memory=True)
    elif Yh.dtype != torch.float64 or Yh.device.type != "cpu" or Yh.numel() < N * M or not Yh.is_contiguous():
        raise ValueError("host_scratch must be a contiguous float64 host tensor of at least N*M entries")
    U = out
    if U is None:
        U = torch.empty((r_max, N), dtype=torch.float64, pin_memory=True).t()
    elif (U.dtype != torch.float64 or U.device.type != "cpu" or U.dim() != 2 or U.shape[0] != N
          or U.shape[1] < r_max or U.stride(0) != 1):
        raise ValueError("out must be a column-major float64 host tensor of N x >= r_max")
    mean = torch.empty(N, dtype=torch.float64, pin_memory=True)
    S = torch.empty(M, dtype=torch.float64, device=dev)
    VT = empty_colmajor(M, M, torch.float64, dev)
    r = _i64(0)
    st = lib.pylom_pod_streamed(_dptr(X), N, M, _ld(X), xtype, _dptr(w), int(bool(remove_mean)), float(energy),
                                r_max, int(mode_kind), int(leaf_rows), int(chunk_rows), _dptr(Yh), _dptr(U), _ld(U),
                                _dptr(S), _dptr(VT), _ld(VT), _dptr(mean), ctypes.byref(r), _dptr(workspace),
                                workspace.numel(), _stream(stream))
    _raise(st, "pylom_pod_streamed")
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    return StreamedPodResult(U=U[:, :int(r.value)], S=S, VT=VT, mean=mean, r=int(r.value), workspace=workspace)


def tsqr(A, leaf_rows=0, want_q=True, prec=PREC_FP64, stream=None, check=True):
    """TSQR of Alg. 1: returns (R, Q or None)."""
    torch = _torch()
    lib = load_library()
    A = _colmajor(A)
    N, M = A.shape
    xtype = {torch.float32: F32, torch.float64: F64}.get(A.dtype)
    if xtype is None:
        raise TypeError("A must be float32 or float64")
    need = lib.pylom_tsqr_workspace_size(N, M, leaf_rows, int(want_q), xtype, prec)
    if need == 0:
        _raise(ERR_SHAPE, f"pylom_tsqr_workspace_size(N={N}, M={M}, b={leaf_rows})")
    ws = torch.empty(need, dtype=torch.uint8, device=A.device)
    R = empty_colmajor(M, M, torch.float64, A.device)
    Q = empty_colmajor(N, M, torch.float64, A.device) if want_q else None
    st = lib.pylom_tsqr(_dptr(A), N, M, _ld(A), xtype, leaf_rows, _dptr(R), _ld(R),
                        _dptr(Q), _ld(Q) if Q is not None else N, prec, _dptr(ws), ws.numel(),
                        _stream(stream))
    _raise(st, "pylom_tsqr")
    if check:
        st, _, _ = workspace_status(ws, stream)
        _raise(st, "pylom_tsqr (device)")
    return R, Q


def svd_small(R, max_sweeps=60, stream=None, check=True):
    """SVD of a small square FP64 matrix (Eq. svdqr2): returns (U, S, VT, sweeps)."""
    torch = _torch()
    lib = load_library()
    R = _colmajor(R.to(torch.float64))
    M = R.shape[0]
    if R.shape[1] != M:
        raise ValueError("svd_small expects a square matrix")
    need = lib.pylom_svd_small_workspace_size(M)
    ws = torch.empty(max(need, 512), dtype=torch.uint8, device=R.device)
    U = empty_colmajor(M, M, torch.float64, R.device)
    VT = empty_colmajor(M, M, torch.float64, R.device)
    S = torch.empty(M, dtype=torch.float64, device=R.device)
    st = lib.pylom_svd_small(_dptr(R), M, _ld(R), _dptr(U), _ld(U), _dptr(S), _dptr(VT),
                             _ld(VT), int(max_sweeps), _dptr(ws), ws.numel(), _stream(stream))
    _raise(st, "pylom_svd_small")
    sweeps = -1
    if check:
        st, _, sweeps = workspace_status(ws, stream)
        _raise(st, "pylom_svd_small (device)")
    return U, S, VT, sweeps


def svd_small_noalloc(R, max_sweeps=60, stream=None):
    """pylom_svd_small_noalloc: the small SVD with the library's fixed scratch
    (M <= 256; no workspace).  Returns (U, S, VT, status, sweeps) after
    synchronising the stream."""
    torch = _torch()
    lib = load_library()
    R = _colmajor(R.to(torch.float64))
    M = R.shape[0]
    if R.shape[1] != M:
        raise ValueError("svd_small_noalloc expects a square matrix")
    U = empty_colmajor(M, M, torch.float64, R.device)
    VT = empty_colmajor(M, M, torch.float64, R.device)
    S = torch.empty(M, dtype=torch.float64, device=R.device)
    info = torch.full((2,), -1, dtype=torch.int32, device=R.device)
    st = lib.pylom_svd_small_noalloc(_dptr(R), M, _ld(R), _dptr(U), _ld(U), _dptr(S), _dptr(VT),
                                     _ld(VT), int(max_sweeps), _dptr(info), _stream(stream))
    _raise(st, "pylom_svd_small_noalloc")
    (stream if stream is not None else torch.cuda.current_stream()).synchronize()
    inf = info.cpu().tolist()
    return U, S, VT, int(inf[0]), int(inf[1])


def matmul(A, B, transA=False, stream=None):
    """Alg. 4's local product C = op(A) B (FP64)."""
    torch = _torch()
    lib = load_library()
    A = _colmajor(A.to(torch.float64))
    B = _colmajor(B.to(torch.float64))
    m, k = (A.shape[1], A.shape[0]) if transA else A.shape
    if B.shape[0] != k:
        raise ValueError("inner dimensions differ")
    n = B.shape[1]
    need = lib.pylom_matmul_workspace_size(m, n, k)
    ws = torch.empty(max(need, 256), dtype=torch.uint8, device=A.device)
    C = empty_colmajor(m, n, torch.float64, A.device)
    st = lib.pylom_matmul(int(bool(transA)), _dptr(A), _dptr(B), _dptr(C), m, n, k, _ld(A),
                          _ld(B), _ld(C), _dptr(ws), ws.numel(), _stream(stream))
    _raise(st, "pylom_matmul")
    return C


def pod_backward(fwd: PodResult, X_shape, w, remove_mean, mode_kind, leaf_rows, r_max, dU=None, dS=None,
                 dVT=None, dx_dtype=None, stream=None, check=True):
    """Cotangent of X for the pylom_pod call that produced `fwd` (its
    workspace must be unchanged).  dU: N x r (r = fwd.r), dS: M, dVT: M x M."""
    torch = _torch()
    lib = load_library()
    N, M = X_shape
    dev = fwd.S.device
    dx_dtype = dx_dtype or torch.float64
    dxt = {torch.float32: F32, torch.float64: F64}[dx_dtype]
    r = fwd.r
    if dU is not None:
        dU = _colmajor(dU.to(torch.float64))
    if dS is not None:
        dS = dS.to(torch.float64).contiguous()
    if dVT is not None:
        dVT = _colmajor(dVT.to(torch.float64))
    if w is not None:
        w = w.to(device=dev, dtype=torch.float64).contiguous()
    need = lib.pylom_pod_backward_workspace_size(N, M, leaf_rows, r, int(fwd.prec))
    if need == 0:
        _raise(ERR_SHAPE, "pylom_pod_backward_workspace_size")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    dX = empty_colmajor(N, M, dx_dtype, dev)
    st = lib.pylom_pod_backward(_dptr(fwd.workspace), fwd.workspace.numel(), N, M, leaf_rows, r_max, r,
                                _dptr(w), int(bool(remove_mean)), int(mode_kind), int(fwd.prec), _dptr(fwd.S),
                                _dptr(fwd.VT),
                                _ld(fwd.VT), _dptr(dU), _ld(dU) if dU is not None else N, _dptr(dS),
                                _dptr(dVT), _ld(dVT) if dVT is not None else M, _dptr(dX), _ld(dX), dxt,
                                _dptr(ws), ws.numel(), _stream(stream))
    _raise(st, "pylom_pod_backward")
    if check:
        st, _, _ = workspace_status(ws, stream)
        _raise(st, "pylom_pod_backward (device)")
    return dX


def _make_pod_function():
    import torch

    class PodFn(torch.autograd.Function):
        """POD as a differentiable operation: forward = pylom_pod (modes,
        singular values, right vectors), backward = pylom_pod_backward, the
        hand-written TSQR + small-SVD adjoint.  Returns (U_r, S, VT)."""

        @staticmethod
        def forward(ctx, X, w, r, remove_mean, mode_kind, leaf_rows, prec):
            res = pod(X.detach(), w=w, remove_mean=remove_mean, energy=0.0, r_max=r, mode_kind=mode_kind,
                      leaf_rows=leaf_rows, prec=prec, check=True)
            ctx.fwd = res
            ctx.meta = (tuple(X.shape), X.dtype, w, remove_mean, mode_kind, leaf_rows, r)
            return res.U.clone(), res.S.clone(), res.VT.clone()

        @staticmethod
        def backward(ctx, gU, gS, gVT):
            shape, dtype, w, remove_mean, mode_kind, leaf_rows, r = ctx.meta
            dX = pod_backward(ctx.fwd, shape, w, remove_mean, mode_kind, leaf_rows, r, dU=gU, dS=gS, dVT=gVT,
                              dx_dtype=dtype)
            return dX, None, None, None, None, None, None

    return PodFn


_PodFn = None


def pod_autograd(X, r, w=None, remove_mean=False, mode_kind=MODES_ORTHONORMAL, leaf_rows=0, prec=PREC_FP64):
    """Differentiable POD: (U_r, S, VT) with the hand-written adjoint (prec:
    PREC_FP64, or PREC_MIXED_3XTF32 for FP32 modes and a tcgen05 adjoint)."""
    global _PodFn
    if _PodFn is None:
        _PodFn = _make_pod_function()
    return _PodFn.apply(X, w, int(r), bool(remove_mean), int(mode_kind), int(leaf_rows), int(prec))


def batched_max_leaf_rows(prec: int) -> int:
    """Longest leaf of a batched-SVD bin at this precision (host query)."""
    return int(load_library().pylom_svd_batched_max_leaf_rows(int(prec)))


class BatchedSVD:
    """Batched complex SVDs (the per-frequency SVDs of SPOD) in one
    persistent launch.  Q: list of column-major complex64 CUDA tensors
    (N_f x Nb_f).  After run(): S[f] (Nb_f,) descending, U[f] (N_f x k_f).
    capture() records run() in a CUDA graph; replay() re-runs it."""

    def __init__(self, Q, kmodes=8, prec=PREC_MIXED_3XTF32, leaf_rows=None, max_sweeps=60):
        torch = _torch()
        lib = load_library()
        self.lib = lib
        self.Q = [_colmajor(q) for q in Q]
        for q in self.Q:
            if q.dtype != torch.complex64:
                raise TypeError("bins must be complex64")
        n = len(self.Q)
        self.N = [int(q.shape[0]) for q in self.Q]
        self.Nb = [int(q.shape[1]) for q in self.Q]
        Na = (_i64 * n)(*self.N)
        Nba = (_i64 * n)(*self.Nb)
        lr = None
        if leaf_rows is not None:
            lr = (_i64 * n)(*[int(x) for x in leaf_rows])
        plan = _vp()
        wsb = _sz(0)
        _raise(lib.pylom_svd_batched_plan(n, Na, Nba, lr, int(kmodes), int(prec), ctypes.byref(plan),
                                          ctypes.byref(wsb)), "pylom_svd_batched_plan")
        self.plan = plan
        self.max_sweeps = int(max_sweeps)
        dev = self.Q[0].device
        self.ws = torch.empty(int(wsb.value), dtype=torch.uint8, device=dev)
        self.S_all = torch.zeros(sum(self.Nb), dtype=torch.float64, device=dev)
        self.k = [min(int(kmodes), nb) for nb in self.Nb]
        self.U = [empty_colmajor(N_f, max(k, 1), torch.complex64, dev) for N_f, k in zip(self.N, self.k)]
        qp = (_vp * n)(*[q.data_ptr() for q in self.Q])
        ldq = (_i64 * n)(*[_ld(q) for q in self.Q])
        up = (_vp * n)(*[u.data_ptr() for u in self.U])
        ldu = (_i64 * n)(*[_ld(u) for u in self.U])
        _raise(lib.pylom_svd_batched_bind(plan, qp, ldq, up, ldu, _dptr(self.ws), self.ws.numel(),
                                          _stream(None)), "pylom_svd_batched_bind")
        self.graph = None

    def info(self, f, what):
        return int(self.lib.pylom_svd_batched_plan_info(self.plan, int(f), int(what)))

    @property
    def S(self):
        return [self.S_all[self.info(f, 2): self.info(f, 2) + nb] for f, nb in enumerate(self.Nb)]

    @property
    def modes(self):
        return [u[:, :k] for u, k in zip(self.U, self.k)]

    def run(self, stream=None):
        _raise(self.lib.pylom_svd_batched_run(self.plan, _dptr(self.ws), _dptr(self.S_all), self.max_sweeps,
                                              _stream(stream)), "pylom_svd_batched_run")

    def status(self, stream=None):
        st, _, _ = workspace_status(self.ws, stream)
        return st

    def capture(self):
        torch = _torch()
        self.run()                       # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(torch.cuda.current_stream())
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                self.lib.pylom_svd_batched_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass


class BatchedItem(ctypes.Structure):
    """pylom_batched_item (include/pylom.h)."""
    _fields_ = [("xtype", _int), ("remove_mean", _int), ("mode_kind", _int), ("reserved", _int),
                ("X", _vp), ("ldx", _i64), ("w", _vp), ("mean", _vp), ("U", _vp), ("ldu", _i64),
                ("VT", _vp), ("ldvt", _i64)]


class BatchedPOD:
    """PODs of several real snapshot windows of different N x M (M <= 128)
    -- each with its own temporal mean removal and cell-volume weights
    (Alg. 2 per window) -- and, optionally, complex64 SPOD bins, all in one
    persistent launch (pylom_svd_batched_plan / _bind_items / _run).

    windows: list of real CUDA tensors (float32 or float64), N_i x M_i.
    weights: None or a list with None or an N_i float64 tensor per window.
    bins:    complex64 CUDA tensors (SPOD bins) run in the same launch,
             after the windows.
    After run(): S[i] (M_i,), modes[i] (N_i x k_i; binary64 with
    prec=PREC_FP64, binary32 with PREC_MIXED_3XTF32; complex64 for bins),
    VT[i] (M_i x M_i right vectors of window i), mean[i] (N_i)."""

    def __init__(self, windows, weights=None, remove_mean=True, mode_kind=MODES_ORTHONORMAL, kmodes=8,
                 prec=PREC_FP64, leaf_rows=None, bins=(), max_sweeps=60):
        torch = _torch()
        lib = load_library()
        self.lib = lib
        self.X = [_colmajor(x) for x in list(windows) + list(bins)]
        nwin = len(windows)
        self.nwin = nwin
        n = len(self.X)
        kinds = []
        for i, x in enumerate(self.X):
            kind = {torch.float32: F32, torch.float64: F64, torch.complex64: C64}.get(x.dtype)
            if kind is None or (i < nwin) == (kind == C64):
                raise TypeError("windows must be float32/float64, bins complex64")
            kinds.append(kind)
        weights = list(weights) if weights is not None else [None] * nwin
        if len(weights) != nwin:
            raise ValueError("one weights entry per window")
        dev = self.X[0].device
        self.w = [None if wt is None else wt.to(device=dev, dtype=torch.float64).contiguous() for wt in weights]
        self.N = [int(x.shape[0]) for x in self.X]
        self.Nb = [int(x.shape[1]) for x in self.X]
        Na, Nba = (_i64 * n)(*self.N), (_i64 * n)(*self.Nb)
        lr = None if leaf_rows is None else (_i64 * n)(*[int(v) for v in leaf_rows])
        plan, wsb = _vp(), _sz(0)
        _raise(lib.pylom_svd_batched_plan(n, Na, Nba, lr, int(kmodes), int(prec), ctypes.byref(plan),
                                          ctypes.byref(wsb)), "pylom_svd_batched_plan")
        self.plan = plan
        self.max_sweeps = int(max_sweeps)
        self.ws = torch.empty(int(wsb.value), dtype=torch.uint8, device=dev)
        self.S_all = torch.zeros(sum(self.Nb), dtype=torch.float64, device=dev)
        self.k = [min(int(kmodes), nb) for nb in self.Nb]
        real_t = torch.float64 if prec == PREC_FP64 else torch.float32
        self.U, self.VT, self.mean = [], [], []
        items = (BatchedItem * n)()
        for i, x in enumerate(self.X):
            real = i < nwin
            U = empty_colmajor(self.N[i], max(self.k[i], 1), real_t if real else torch.complex64, dev)
            VT = empty_colmajor(self.Nb[i], self.Nb[i], torch.float64, dev) if real else None
            mean = torch.zeros(self.N[i], dtype=torch.float64, device=dev) if real else None
            self.U.append(U)
            self.VT.append(VT)
            self.mean.append(mean)
            it = items[i]
            it.xtype, it.remove_mean, it.mode_kind, it.reserved = kinds[i], int(bool(remove_mean)), int(mode_kind), 0
            it.X, it.ldx = x.data_ptr(), _ld(x)
            it.w = self.w[i].data_ptr() if real and self.w[i] is not None else None
            it.mean = mean.data_ptr() if real else None
            it.U, it.ldu = U.data_ptr(), _ld(U)
            it.VT, it.ldvt = (VT.data_ptr(), _ld(VT)) if real else (None, 0)
        self._items = items
        _raise(lib.pylom_svd_batched_bind_items(plan, ctypes.cast(items, ctypes.c_void_p), _dptr(self.ws),
                                                self.ws.numel(), _stream(None)), "pylom_svd_batched_bind_items")
        self.graph = None

    def info(self, f, what):
        return int(self.lib.pylom_svd_batched_plan_info(self.plan, int(f), int(what)))

    @property
    def S(self):
        return [self.S_all[self.info(f, 2): self.info(f, 2) + nb] for f, nb in enumerate(self.Nb)]

    @property
    def modes(self):
        return [u[:, :k] for u, k in zip(self.U, self.k)]

    def run(self, stream=None):
        _raise(self.lib.pylom_svd_batched_run(self.plan, _dptr(self.ws), _dptr(self.S_all), self.max_sweeps,
                                              _stream(stream)), "pylom_svd_batched_run")

    def status(self, stream=None):
        st, _, _ = workspace_status(self.ws, stream)
        return st

    def capture(self):
        torch = _torch()
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(torch.cuda.current_stream())
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                self.lib.pylom_svd_batched_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass


# ---------------------------------------------------------------------------
# SPOD (Sec. 2.3, Alg. 6): front end + batched SVDs + ordering
# ---------------------------------------------------------------------------

def spod_shape(T: int, npwin: int, nolap: int):
    """(nBlks, nfreq) of Alg. 6 for T snapshots, windows of npwin overlapping by nolap."""
    nb, nf = _i64(0), _i64(0)
    _raise(load_library().pylom_spod_shape(int(T), int(npwin), int(nolap), ctypes.byref(nb), ctypes.byref(nf)),
           "pylom_spod_shape")
    return int(nb.value), int(nf.value)


def spod_blocks(D, npwin: int, nolap: int, remove_mean: bool = True, Q=None, mean=None, workspace=None,
                stream=None):
    """The matrices Q_f / sqrt(nBlks) of every frequency (Alg. 6) from the
    snapshots D (N x T CUDA tensor, float32 or float64): a complex64 tensor
    Q of shape (nfreq, nBlks, N), Q[f].t() being the N x nBlks matrix of
    frequency f (column-major)."""
    torch = _torch()
    lib = load_library()
    D = _colmajor(D)
    N, T = D.shape
    dt = {torch.float32: F32, torch.float64: F64}.get(D.dtype)
    if dt is None:
        raise TypeError("D must be float32 or float64")
    nblks, nfreq = spod_shape(T, npwin, nolap)
    dev = D.device
    if Q is None:
        Q = torch.empty((nfreq, nblks, N), dtype=torch.complex64, device=dev)
    need = lib.pylom_spod_blocks_workspace_size(N, int(npwin))
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    _raise(lib.pylom_spod_blocks(_dptr(D), N, T, _ld(D), dt, int(npwin), int(nolap), int(bool(remove_mean)),
                                 _dptr(Q), int(Q.shape[2]), _dptr(mean), _dptr(workspace), workspace.numel(),
                                 _stream(stream)), "pylom_spod_blocks")
    return Q


class SPOD:
    """SPOD of the snapshot matrix D (N points x T instants) on the GPU
    (Sec. 2.3, Alg. 6): the front end (blocks, Hamming window, one-sided
    transform, Q_f), the SVDs of all frequencies in one persistent launch,
    and the order of the frequencies by their leading energy.  run() is
    capturable as one CUDA graph (capture() / replay()).  After a run:
    L (nfreq x nBlks energies S^2, bin order), modes[f] (N x kmodes complex64),
    order (frequencies by leading energy), f (frequency axis, 1 / time)."""

    def __init__(self, D, dt: float, npwin: int, nolap: int, remove_mean: bool = True, kmodes: int = 8,
                 prec=PREC_MIXED_3XTF32, leaf_rows=None):
        torch = _torch()
        self.lib = load_library()
        self.D = _colmajor(D)
        N, T = self.D.shape
        self.npwin, self.nolap, self.remove_mean = int(npwin), int(nolap), bool(remove_mean)
        self.nblks, self.nfreq = spod_shape(T, npwin, nolap)
        dev = self.D.device
        self.Q = torch.empty((self.nfreq, self.nblks, N), dtype=torch.complex64, device=dev)
        self.ws = torch.empty(self.lib.pylom_spod_blocks_workspace_size(N, self.npwin), dtype=torch.uint8,
                              device=dev)
        self.svd = BatchedSVD([self.Q[f].t() for f in range(self.nfreq)], kmodes=kmodes, prec=prec,
                              leaf_rows=leaf_rows)
        self.order = torch.empty(self.nfreq, dtype=torch.int64, device=dev)
        self.f = torch.arange(self.nfreq, dtype=torch.float64, device=dev) / (float(dt) * self.npwin)
        self.graph = None

    def run(self, stream=None):
        spod_blocks(self.D, self.npwin, self.nolap, self.remove_mean, Q=self.Q, workspace=self.ws, stream=stream)
        self.svd.run(stream)
        _raise(self.lib.pylom_spod_order(_dptr(self.svd.S_all), self.nfreq, self.nblks, _dptr(self.order),
                                         _stream(stream)), "pylom_spod_order")

    @property
    def L(self):
        return self.svd.S_all.view(self.nfreq, self.nblks) ** 2

    @property
    def modes(self):
        return self.svd.modes

    def status(self, stream=None):
        return self.svd.status(stream)

    def capture(self):
        torch = _torch()
        self.run()                       # warm-up outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(torch.cuda.current_stream())
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

