"""GPU parity: the CUDA POD / TSQR / small-SVD / matmul path (through the C
ABI) against the FP64 CPU oracle on the same seeded inputs, element by
element, plus the full-size 4,194,304 x 256 workload against its closed-form
construction."""
import ctypes
import math

import numpy as np
import pytest

import oracle
import synth
from tests import closed_forms as cf
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")


def _dev(X):
    """numpy Fortran array -> column-major CUDA tensor."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda").t()


def _np(t):
    return t.detach().cpu().numpy()


def _compare_pod(X, res, ref, w=None, mode_kind=0, sigma_abs=parity.SIGMA_ABS):
    S, S_ref = _np(res.S), ref["S"]
    parity.check_sigma(S, S_ref, abs_tol=sigma_abs)
    assert res.r == ref["r"]
    U = _np(res.U)
    wt = w if (w is not None and mode_kind == 1) else None
    parity.check_vectors(U, ref["U"], S_ref, ncols=res.r, weight=wt)
    V = _np(res.VT).T
    parity.check_vectors(V, ref["VT"].T, S_ref, ncols=res.r)
    # signs of separated singular pairs agree with the oracle (same rule)
    for grp in parity.clusters(S_ref):
        if len(grp) == 1 and grp[0] < res.r:
            i = grp[0]
            assert np.dot(V[:, i], ref["VT"][i, :]) > 0.0
    np.testing.assert_allclose(_np(res.mean), ref["mean"], rtol=0, atol=1e-14 * np.abs(X).max())


@pytest.mark.parametrize("N,M,b,remove_mean,weighted,mode_kind", [
    (16384, 64, 1024, True, False, 0),     # the 16384 x 64 wave workload, P = 16
    (5037, 24, 600, False, True, 0),       # ragged leaves (P = 8, uneven heights)
    (3001, 37, 128, True, True, 1),        # odd M, not a panel multiple, P = 23
    (200, 40, 0, True, False, 0),          # a single leaf
    (64, 64, 0, False, False, 0),          # square
    (100, 1, 0, False, True, 1),           # one snapshot
    (2048, 17, 17, True, False, 0),        # leaves of exactly M rows, P = 120
])
def test_pod_matches_oracle(N, M, b, remove_mean, weighted, mode_kind):
    X = synth.waves(N, M, n_waves=min(8, max(1, M // 4)), noise=1e-3, seed=N + M)
    w = synth.log_uniform_weights(N, seed=7) if weighted else None
    ref = oracle.pod(X, w=w, remove_mean=remove_mean, mode_kind=mode_kind)
    res = pg.pod(_dev(X), w=None if w is None else torch.from_numpy(w).cuda(),
                 remove_mean=remove_mean, mode_kind=mode_kind, leaf_rows=b)
    _compare_pod(X, res, ref, w=w, mode_kind=mode_kind)


def test_pod_float32_input():
    N, M = 6000, 48
    X = synth.waves(N, M, n_waves=8, noise=1e-3, seed=3, dtype=np.float32)
    ref = oracle.pod(X.astype(np.float64), remove_mean=True)
    res = pg.pod(_dev(X), remove_mean=True, leaf_rows=700)
    _compare_pod(X.astype(np.float64), res, ref)


def test_pod_energy_truncation_and_known_spectrum():
    N, M = 8192, 64
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(51, 52, 53))
    ref = oracle.pod(X, w=w, remove_mean=False, energy=0.99, mode_kind=1)
    res = pg.pod(_dev(X), w=torch.from_numpy(w).cuda(), remove_mean=False, energy=0.99,
                 mode_kind=1, leaf_rows=512)
    assert res.r == ref["r"] == cf.truncation_rank(M, 6.0, 0.99)
    parity.check_sigma(_np(res.S), s)
    _compare_pod(X, res, ref, w=w, mode_kind=1)
    Phi = _np(res.U)
    assert parity.orthonormality(Phi, weight=w) < 1e-12


def test_pod_repeatable_and_leaf_invariant():
    N, M = 4096, 32
    X = synth.waves(N, M, n_waves=6, noise=1e-3, seed=9)
    Xd = _dev(X)
    a = pg.pod(Xd, leaf_rows=256)
    b = pg.pod(Xd, leaf_rows=256)
    assert torch.equal(a.S, b.S) and torch.equal(a.U, b.U) and torch.equal(a.VT, b.VT)
    S_ref = a.S.cpu().numpy()
    for lr in (32, 100, 1000, 4096):
        c = pg.pod(Xd, leaf_rows=lr)
        parity.check_sigma(_np(c.S), S_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_pod_graph_replay_is_repeatable(prec):
    """One pylom_pod call (leaves, the pipelined tree from 64 leaves, small
    SVD, top-down pass, modes) captured in a CUDA graph: replays agree with
    each other bit for bit and with the eager call."""
    N, M = 1 << 18, 64
    X = synth.waves(N, M, n_waves=8, noise=1e-3, seed=21)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = _dev(X).to(dt)
    res = pg.pod(Xd, energy=0.99, prec=prec)
    assert pg.leaf_count(N, M, 0) >= 64
    ws = res.workspace
    U = pg.empty_colmajor(N, M, dt, "cuda")
    S = torch.empty(M, dtype=torch.float64, device="cuda")
    VT = pg.empty_colmajor(M, M, torch.float64, "cuda")
    mean = torch.empty(N, dtype=torch.float64, device="cuda")
    r_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = (U, S, VT, mean, r_dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pg.pod(Xd, energy=0.99, prec=prec, workspace=ws, out=out, stream=s, check=False)   # warm-up
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pg.pod(Xd, energy=0.99, prec=prec, workspace=ws, out=out, stream=s, check=False)
    g.replay()
    torch.cuda.synchronize()
    st, r, _ = pg.workspace_status(ws)
    assert st == pg.OK and r == res.r
    first = (U[:, :r].clone(), S.clone(), VT.clone())
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(first[0], U[:, :r]) and torch.equal(first[1], S) and torch.equal(first[2], VT)
    assert torch.equal(S, res.S) and torch.equal(U[:, :r], res.U)


@pytest.mark.parametrize("prec", [0, 1])
def test_pod_reads_page_locked_host_x(prec):
    """X in page-locked host memory: the leaf kernel reads it across the host
    link; the results are those of the device-resident X bit for bit."""
    N, M = 1 << 17, 48
    X = synth.waves(N, M, n_waves=6, noise=1e-3, seed=23)
    dt = torch.float64 if prec == 0 else torch.float32
    Xd = _dev(X).to(dt)
    Xh = torch.empty((M, N), dtype=dt, pin_memory=True)
    Xh.copy_(Xd.t())
    Xh = Xh.t()
    a = pg.pod(Xd, energy=0.99, prec=prec)
    b = pg.pod(Xh, energy=0.99, prec=prec)
    assert a.r == b.r
    assert torch.equal(a.S, b.S) and torch.equal(a.U, b.U) and torch.equal(a.VT, b.VT)
    assert torch.equal(a.mean, b.mean)


def test_pod_rejects_pageable_host_x():
    """Pageable host memory is refused on the host, before any launch."""
    lib = pg.load_library()
    N, M = 2048, 16
    Xh = np.asfortranarray(np.random.default_rng(0).standard_normal((N, M)))
    need = pg.pod_workspace_size(N, M)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    U = pg.empty_colmajor(N, M, torch.float64, "cuda")
    S = torch.empty(M, dtype=torch.float64, device="cuda")
    VT = pg.empty_colmajor(M, M, torch.float64, "cuda")
    st = lib.pylom_pod(ctypes.c_void_p(Xh.ctypes.data), N, M, N, pg.F64, None, 1, 0.0, M, 0, 0, pg._dptr(U),
                       pg._ld(U), pg._dptr(S), pg._dptr(VT), pg._ld(VT), None, None, pg.PREC_FP64, pg._dptr(ws),
                       ws.numel(), None)
    assert st == pg.ERR_ARG
    assert b"pageable" in lib.pylom_last_error()
    with pytest.raises(ValueError):
        pg.pod(torch.from_numpy(Xh.T.copy()).t())      # a host tensor that is not page-locked


def test_pod_zero_and_constant_rows():
    X = np.repeat(np.round(100 * np.random.default_rng(4).standard_normal((300, 1))), 12, axis=1)
    X = np.asfortranarray(X)
    res = pg.pod(_dev(X), remove_mean=True, leaf_rows=100)
    assert torch.all(res.S == 0.0)
    U = _np(res.U)
    assert parity.orthonormality(U) < 1e-13
    np.testing.assert_array_equal(_np(res.mean), X[:, 0])


def test_pod_reports_nonfinite_input():
    X = synth.waves(1000, 10, n_waves=2, noise=0.0)
    X[17, 3] = np.nan
    with pytest.raises(pg.PylomError) as ei:
        pg.pod(_dev(X), leaf_rows=200)
    assert ei.value.status == pg.ERR_NONFINITE


def test_tsqr_is_fp64_only():
    X = _dev(synth.waves(1000, 10, n_waves=2, noise=0.0))
    with pytest.raises(pg.PylomError):
        pg.tsqr(X, prec=pg.PREC_MIXED_3XTF32)


# ---------------------------------------------------------------------------
# TSQR, small SVD, local product
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,M,b", [(4096, 64, 512), (3001, 37, 128), (500, 20, 0), (777, 16, 16)])
def test_tsqr_matches_oracle(N, M, b):
    A = np.asfortranarray(np.random.default_rng(N).standard_normal((N, M)))
    R, Q = pg.tsqr(_dev(A), leaf_rows=b)
    R, Q = _np(R), _np(Q)
    R_ref, _ = oracle.tsqr(A, want_q=False)
    nA = np.linalg.norm(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(R.T @ R - A.T @ A) <= 1e-13 * nA ** 2
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(R_ref)), rtol=1e-11, atol=1e-13 * nA)
    # the rows agree up to sign
    sg = np.sign(np.diag(R)) * np.sign(np.diag(R_ref))
    assert np.linalg.norm(sg[:, None] * R - R_ref) <= 1e-12 * np.linalg.norm(R_ref)
    assert np.linalg.norm(Q.T @ Q - np.eye(M)) <= 1e-13 * math.sqrt(M)
    assert np.linalg.norm(Q @ R - A) <= 1e-13 * nA


@pytest.mark.parametrize("M,triangular", [(64, True), (37, False), (256, True), (1, False), (2, True),
                                         (600, True), (513, False)])   # the last two: binary32 preconditioning
def test_svd_small_matches_oracle(M, triangular):
    R = np.random.default_rng(M).standard_normal((M, M)) * np.logspace(0, -4, M)[None, :]
    if triangular:
        R = np.triu(R)
    R = np.asfortranarray(R)
    U, S, VT, sweeps = pg.svd_small(_dev(R))
    U_ref, S_ref, V_ref, _ = oracle.svd(R)
    parity.check_sigma(_np(S), S_ref)
    parity.check_vectors(_np(U), U_ref, S_ref)
    parity.check_vectors(_np(VT).T, V_ref, S_ref)
    Un, Sn, Vn = _np(U), _np(S), _np(VT).T
    # Jacobi's rounding grows with the number of rotations (about M per column
    # per sweep): the oracle itself reaches 7.7e-14 on the 256 x 256 case
    rec_tol = max(1e-13, 1e-15 * M)
    assert np.linalg.norm(R - (Un * Sn) @ Vn.T) <= rec_tol * max(np.linalg.norm(R), 1e-300)
    # spectral norm of Q^T Q - I; the oracle's own Jacobi reaches 3.9e-13 at
    # M = 256 and 1.6e-12 at M = 600 on these graded matrices
    for Q in (Un, Vn):
        assert np.linalg.norm(Q.T @ Q - np.eye(M), 2) <= max(1e-13, 5e-15 * M)
    assert 1 <= sweeps <= 60


def test_svd_small_reports_nonconvergence():
    R = np.asfortranarray(np.random.default_rng(0).standard_normal((32, 32)))
    with pytest.raises(pg.PylomError) as ei:
        pg.svd_small(_dev(R), max_sweeps=1)
    assert ei.value.status == pg.ERR_NOCONV


@pytest.mark.parametrize("m,n,k,transA", [(43, 256, 100000, True), (7, 5, 3, False), (64, 64, 64, True),
                                          (33, 17, 5000, False)])
def test_matmul_matches_oracle(m, n, k, transA):
    rng = np.random.default_rng(m + n)
    A = np.asfortranarray(rng.standard_normal((k, m) if transA else (m, k)))
    B = np.asfortranarray(rng.standard_normal((k, n)))
    C = _np(pg.matmul(_dev(A), _dev(B), transA=transA))
    C_ref = oracle.matmul(A, B, transA=transA)
    scale = np.sqrt(k) * 1e-14 * 10
    np.testing.assert_allclose(C, C_ref, rtol=0, atol=scale)


# ---------------------------------------------------------------------------
# full size: the 4,194,304 x 256 known-spectrum workload (closed form)
# ---------------------------------------------------------------------------

def test_pod_full_size_known_spectrum():
    N, M = 1 << 22, 256
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda")
    X = XT.t()
    res = pg.pod(X, w=w, remove_mean=False, energy=0.99, mode_kind=pg.MODES_ORTHONORMAL)
    assert res.r == 43 == cf.truncation_rank(M, 6.0, 0.99)
    parity.check_sigma(_np(res.S), s)
    # the exact left vectors of diag(sqrt w) X are the columns of Q1, which
    # the generator rebuilds: U_w = sqrt(w) X Q2 diag(1/s)
    Q2 = torch.tensor(synth.haar_orthogonal(M, 3), dtype=torch.float64, device="cuda")
    Yw = X * torch.sqrt(w)[:, None]
    Q1r = (Yw @ Q2[:, :43]) / torch.tensor(s[:43], device="cuda")[None, :]
    U = res.U
    ov = torch.abs(torch.sum(U * Q1r, dim=0))
    assert torch.all(ov >= 1 - 1e-6), ov.min()
    G = U.T @ U
    assert torch.linalg.norm(G - torch.eye(43, dtype=torch.float64, device="cuda")) < 1e-12
    V = res.VT.t()[:, :43]
    ovv = torch.abs(torch.sum(V * Q2[:, :43], dim=0))
    assert torch.all(ovv >= 1 - 1e-6)
