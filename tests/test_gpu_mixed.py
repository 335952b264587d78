"""GPU parity of the mixed-precision POD path (FP32 leaves, 3xTF32 block
reflectors on tcgen05, binary64 tree / Jacobi / top-down pass) against the
FP64 oracle and against the FP64 GPU path on the same input, at the mixed
tolerances: |dS| <= 2e-6 S_max; modes with S >= 1e-3 S_max separated by
>= 1e-3 relatively to within 1 - 1e-6 overlap."""
import numpy as np
import pytest

import oracle
import synth
from tests import closed_forms as cf
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")

MIXED_SIGMA = 2e-6
MODE_FLOOR = 1e-3


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda").t()


def _check_modes(U, U_ref, S_ref, k, weight=None):
    for grp in parity.clusters(S_ref):
        grp = [i for i in grp if i < k and S_ref[i] >= MODE_FLOOR * S_ref[0]]
        if not grp:
            continue
        A, B = U[:, grp], U_ref[:, grp]
        G = A.T @ (B * weight[:, None]) if weight is not None else A.T @ B
        v = abs(G[0, 0]) if len(grp) == 1 else np.linalg.svd(G, compute_uv=False).min()
        assert v >= 1 - 1e-6, (grp, v)


@pytest.mark.parametrize("N,M,b,remove_mean,weighted,mode_kind,dtype", [
    (16384, 64, 1024, True, False, 0, np.float64),   # the 16384 x 64 wave workload
    (5037, 24, 600, False, True, 0, np.float32),     # one partial panel, ragged leaves
    (3001, 37, 128, True, True, 1, np.float32),      # two panels (32 + 5), P = 23
    (20000, 128, 2048, False, False, 0, np.float32), # several 128-column chunks
    (9001, 300, 1500, True, False, 0, np.float32),   # trailing chunks of 128, 128, 12 columns; odd N
])
def test_mixed_pod_matches_oracle_and_fp64_path(N, M, b, remove_mean, weighted, mode_kind, dtype):
    X = synth.waves(N, M, n_waves=min(8, max(1, M // 4)), noise=1e-3, seed=N + M, dtype=dtype)
    w = synth.log_uniform_weights(N, seed=7) if weighted else None
    ref = oracle.pod(X.astype(np.float64), w=w, remove_mean=remove_mean, mode_kind=mode_kind)
    wd = None if w is None else torch.from_numpy(w).cuda()
    mix = pg.pod(_dev(X), w=wd, remove_mean=remove_mean, mode_kind=mode_kind, leaf_rows=b,
                 prec=pg.PREC_MIXED_3XTF32)
    f64 = pg.pod(_dev(X), w=wd, remove_mean=remove_mean, mode_kind=mode_kind, leaf_rows=b)
    assert mix.U.dtype == torch.float32
    S, S_ref, S64 = mix.S.cpu().numpy(), ref["S"], f64.S.cpu().numpy()
    assert np.max(np.abs(S - S_ref)) <= MIXED_SIGMA * S_ref[0], np.max(np.abs(S - S_ref)) / S_ref[0]
    assert np.max(np.abs(S - S64)) <= MIXED_SIGMA * S64[0]
    assert mix.r == ref["r"]
    wt = w if (w is not None and mode_kind == 1) else None
    U = mix.U.double().cpu().numpy()
    _check_modes(U, ref["U"], S_ref, mix.r, weight=wt)
    _check_modes(U, f64.U.cpu().numpy(), S64, mix.r, weight=wt)
    np.testing.assert_allclose(mix.mean.cpu().numpy(), ref["mean"], rtol=0, atol=1e-13 * np.abs(X).max())


def test_mixed_pod_known_spectrum_truncation():
    N, M = 65536, 256
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(71, 72, 73), dtype=np.float32)
    res = pg.pod(_dev(X), w=torch.from_numpy(w).cuda(), remove_mean=False, energy=0.99, leaf_rows=8192,
                 prec=pg.PREC_MIXED_3XTF32)
    ref = oracle.pod(X.astype(np.float64), w=w, remove_mean=False, energy=0.99)
    assert res.r == ref["r"]
    S = res.S.cpu().numpy()
    assert np.max(np.abs(S - ref["S"])) <= MIXED_SIGMA * ref["S"][0]
    _check_modes(res.U.double().cpu().numpy(), ref["U"], ref["S"], res.r)


def test_mixed_pod_full_size_fp32():
    # 4,194,304 x 256 float32 known spectrum, weights, 99 % energy
    N, M = 1 << 22, 256
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda", dtype=torch.float32)
    X = XT.t()
    res = pg.pod(X, w=w, remove_mean=False, energy=0.99, prec=pg.PREC_MIXED_3XTF32)
    assert res.r == 43 == cf.truncation_rank(M, 6.0, 0.99)
    # the exact spectrum of the float32 matrix differs from s by its rounding
    S = res.S.cpu().numpy()
    assert np.max(np.abs(S - s)) <= MIXED_SIGMA * s[0], np.max(np.abs(S - s))
    f64 = pg.pod(X, w=w, remove_mean=False, energy=0.99)
    S64 = f64.S.cpu().numpy()
    assert np.max(np.abs(S - S64)) <= MIXED_SIGMA * S64[0]
    G = res.U.double().T @ res.U.double()
    E = (G - torch.eye(res.r, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.linalg.norm(E, 2) < 1e-5, np.linalg.norm(E, 2)
    _check_modes(res.U.double().cpu().numpy(), f64.U.cpu().numpy(), S64, res.r)


def test_mixed_pod_full_size_waves_1808():
    # 10,000,000 x 1808 float32 wake-like field: 64 traveling waves with
    # power-law amplitudes, noise 1e-4, mean removed, 99 % energy, <= 128 modes
    N, M, rmax = 10_000_000, 1808, 128
    torch.cuda.empty_cache()
    XT = synth.waves_torch(N, M, 64, "powerlaw", 1e-4, 5, "cuda", dtype=torch.float32, row_chunk=1 << 18)
    X = XT.t()
    mix = pg.pod(X, remove_mean=True, energy=0.99, r_max=rmax, prec=pg.PREC_MIXED_3XTF32)
    S = mix.S.cpu().numpy()
    U = mix.U
    del mix
    torch.cuda.empty_cache()
    f64 = pg.pod(X, remove_mean=True, energy=0.99, r_max=rmax)
    S64 = f64.S.cpu().numpy()
    U64 = f64.U
    r = f64.r
    del f64
    torch.cuda.empty_cache()
    assert U.shape[1] == r
    # mixed against the FP64 GPU path on the same X
    assert np.max(np.abs(S - S64)) <= MIXED_SIGMA * S64[0], np.max(np.abs(S - S64)) / S64[0]
    # both against the noise-free closed form a_j sqrt(NM)/2 (twice each), within
    # the noise's spectral norm (Weyl), ~1e-4 (sqrt N + sqrt M)
    a, _, _ = synth.wave_params(64, "powerlaw")
    s_cf = np.repeat(a * np.sqrt(N * M) / 2.0, 2)
    weyl = 1.5e-4 * (np.sqrt(N) + np.sqrt(M))
    assert np.max(np.abs(S64[:128] - s_cf)) <= weyl
    assert np.all(S64[128:] <= weyl)
    assert r == cf.truncation_rank_of(s_cf, 0.99)
    # orthonormal modes, and the same modes (pairs as subspaces) as the FP64 path
    G = torch.zeros((r, r), dtype=torch.float64, device="cuda")
    Gm = torch.zeros((r, r), dtype=torch.float64, device="cuda")
    for r0 in range(0, N, 1 << 20):
        blk = U[r0:r0 + (1 << 20)].double()
        G += blk.T @ U64[r0:r0 + (1 << 20)]
        Gm += blk.T @ blk
    # FP32 modes carry about 1e-7 per entry of U^T U - I; bound the spectral norm
    E = (Gm - torch.eye(r, dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.linalg.norm(E, 2) < 1e-5, np.linalg.norm(E, 2)
    Gn = G.cpu().numpy()
    for grp in parity.clusters(S64[:r]):
        grp = [i for i in grp if S64[i] >= MODE_FLOOR * S64[0]]
        if not grp:
            continue
        blk = Gn[np.ix_(grp, grp)]
        v = abs(blk[0, 0]) if len(grp) == 1 else np.linalg.svd(blk, compute_uv=False).min()
        assert v >= 1 - 1e-6, (grp, v)
