"""Row-sharded POD: the paper's parallel form (Sec. 3.1, Alg. 1) with the
row blocks of the snapshot matrix on different devices (one process per
GPU) or in several calls on one device.

Per shard g (rows X_g):
  1. ``shard_factor``: mean / weights, leaf QR and the shard's own tree
     (pylom_pod_shard_factor) -> R_g (M x M);
  2. the G factors are gathered on every shard (``torch.distributed``
     all-gather: the only exchange, G M^2 doubles);
  3. ``rstack``: the top of the tree over the stacked factors, the SVD of R,
     the truncation and the top-down pass to every shard
     (pylom_pod_rstack, replicated) -> S, VT, r and B_g;
  4. ``shard_modes``: the top-down pass through the shard's tree and its
     leaf modes (pylom_pod_shard_modes) -> U_g.

This module marshals arguments and moves the R factors; the arithmetic runs
in libpylom.so.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

from . import (F32, F64, MODES_ORTHONORMAL, PREC_FP64, PREC_MIXED_3XTF32, _colmajor, _dptr, _ld, _raise,
               _stream, _torch, empty_colmajor, load_library, workspace_status)


@dataclass
class ShardState:
    ws: "torch.Tensor"          # the shard's workspace (reflectors, tree) until shard_modes
    R: "torch.Tensor"           # M x M factor R_g (column-major, zeros below the diagonal)
    mean: Optional["torch.Tensor"]
    N: int
    M: int
    leaf_rows: int
    r_max: int
    prec: int


@dataclass
class TopResult:
    S: "torch.Tensor"           # M
    VT: "torch.Tensor"          # M x M
    B: "torch.Tensor"           # G x r_max x M: B[g].T is shard g's M x r_max block
    r_dev: "torch.Tensor"       # device int64
    ws: "torch.Tensor"


def shard_factor(X, w=None, remove_mean=True, leaf_rows=0, r_max=None, prec=PREC_FP64, stream=None) -> ShardState:
    torch = _torch()
    lib = load_library()
    X = _colmajor(X)
    N, M = X.shape
    xtype = {torch.float32: F32, torch.float64: F64}.get(X.dtype)
    if xtype is None:
        raise TypeError("X must be float32 or float64")
    r_max = M if r_max is None else int(r_max)
    dev = X.device
    if w is not None:
        w = w.to(device=dev, dtype=torch.float64).contiguous()
    need = lib.pylom_pod_shard_workspace_size(N, M, int(leaf_rows), r_max, xtype, int(prec))
    if need == 0:
        _raise(2, f"pylom_pod_shard_workspace_size(N={N}, M={M}, b={leaf_rows}, r_max={r_max})")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    R = empty_colmajor(M, M, torch.float64, dev)
    mean = torch.empty(N, dtype=torch.float64, device=dev)
    st = lib.pylom_pod_shard_factor(_dptr(X), N, M, _ld(X), xtype, _dptr(w), int(bool(remove_mean)),
                                    int(leaf_rows), r_max, _dptr(mean), _dptr(R), _ld(R), int(prec), _dptr(ws),
                                    ws.numel(), _stream(stream))
    _raise(st, "pylom_pod_shard_factor")
    return ShardState(ws=ws, R=R, mean=mean, N=N, M=M, leaf_rows=int(leaf_rows), r_max=r_max, prec=int(prec))


def rstack(Rstack, energy=0.0, r_max=None, stream=None) -> TopResult:
    """Rstack: (G, M, M) tensor whose slice g is R_g^T (i.e. R_g column-major)."""
    torch = _torch()
    lib = load_library()
    Rstack = Rstack.to(torch.float64).contiguous()
    G, M, _ = Rstack.shape
    r_max = M if r_max is None else int(r_max)
    dev = Rstack.device
    need = lib.pylom_pod_rstack_workspace_size(G, M, r_max)
    if need == 0:
        _raise(2, f"pylom_pod_rstack_workspace_size(G={G}, M={M}, r_max={r_max})")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    S = torch.empty(M, dtype=torch.float64, device=dev)
    VT = empty_colmajor(M, M, torch.float64, dev)
    B = torch.zeros((G, r_max, M), dtype=torch.float64, device=dev)
    r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    st = lib.pylom_pod_rstack(_dptr(Rstack), G, M, float(energy), r_max, _dptr(S), _dptr(VT), _ld(VT), _dptr(B),
                              _dptr(r_dev), _dptr(ws), ws.numel(), _stream(stream))
    _raise(st, "pylom_pod_rstack")
    return TopResult(S=S, VT=VT, B=B, r_dev=r_dev, ws=ws)


def shard_modes(state: ShardState, Bg, r_dev, w=None, mode_kind=MODES_ORTHONORMAL, stream=None):
    """U_g (N_g x r_max, the first r columns valid) of the shard.  Bg: the
    shard's (r_max, M) slice of TopResult.B."""
    torch = _torch()
    lib = load_library()
    dev = state.R.device
    Bg = Bg.to(torch.float64).contiguous()
    if tuple(Bg.shape) != (state.r_max, state.M):
        raise ValueError("Bg must be the shard's (r_max, M) block")
    if w is not None:
        w = w.to(device=dev, dtype=torch.float64).contiguous()
    U = empty_colmajor(state.N, state.r_max, torch.float32 if state.prec == PREC_MIXED_3XTF32 else torch.float64,
                       dev)
    st = lib.pylom_pod_shard_modes(_dptr(Bg), _dptr(r_dev), state.N, state.M, state.leaf_rows, state.r_max,
                                   _dptr(w), int(mode_kind), _dptr(U), _ld(U), state.prec, _dptr(state.ws),
                                   state.ws.numel(), _stream(stream))
    _raise(st, "pylom_pod_shard_modes")
    return U


class GpuShardOps:
    """The three device steps of a shard, through libpylom.so."""

    def __init__(self, remove_mean=True, leaf_rows=0, r_max=None, energy=0.0, mode_kind=MODES_ORTHONORMAL,
                 prec=PREC_FP64):
        self.remove_mean, self.leaf_rows, self.r_max = remove_mean, leaf_rows, r_max
        self.energy, self.mode_kind, self.prec = energy, mode_kind, prec

    def factor(self, X, w):
        st = shard_factor(X, w, self.remove_mean, self.leaf_rows, self.r_max, self.prec)
        return st.R, st

    def top(self, Rstack):
        r_max = self.r_max if self.r_max is not None else Rstack.shape[1]
        t = rstack(Rstack, self.energy, r_max)
        return t.S, t.VT, t.B, t.r_dev, t

    def modes(self, state, Bg, r_dev, w):
        U = shard_modes(state, Bg, r_dev, w, self.mode_kind)
        st, _, _ = workspace_status(state.ws)
        _raise(st, "pylom_pod_shard_factor / pylom_pod_shard_modes (device)")
        return U


def pod_sharded(X_local, w=None, group=None, ops=None, **kw):
    """POD of the row-stacked matrix [X_0; X_1; ...; X_{G-1}] where this
    process holds X_local = X_rank (rank = its rank in `group`, the
    default process group if None).  Every rank returns S, VT and r (equal
    on all ranks) and its own rows U_local of the modes.

    ops: the three shard steps (default: GpuShardOps(**kw), the library on
    this process's device)."""
    import torch
    import torch.distributed as dist
    ops = ops if ops is not None else GpuShardOps(**kw)
    R, state = ops.factor(X_local, w)
    Rt = R.t().contiguous()                        # column-major R_g as a row-major (M, M) block
    if dist.is_available() and dist.is_initialized():
        G = dist.get_world_size(group)
        rank = dist.get_rank(group)
        parts = [torch.empty_like(Rt) for _ in range(G)]
        dist.all_gather(parts, Rt, group=group)    # shard g's factor lands in slot g on every rank
        Rstack = torch.stack(parts)
    else:
        rank, Rstack = 0, Rt[None]
    S, VT, B, r_dev, top = ops.top(Rstack)
    U = ops.modes(state, B[rank], r_dev, w)
    r = int(r_dev.reshape(-1)[0].item())
    return U[:, :r], S, VT, r
