"""GPU parity of the batched multi-window POD: several real snapshot windows
of different N x M (each with its own temporal mean removal and cell-volume
weights, Alg. 2 per window) and complex SPOD bins in one persistent launch
(pylom_svd_batched_bind_items), each window against the FP64 oracle's POD of
that window, each bin against the complex oracle, element by element."""
import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")

# N, M, float type, weights, leaf-height hint
WINDOWS = [
    (3000, 24, np.float64, True, 0),
    (5000, 64, np.float32, False, 1024),
    (1500, 17, np.float64, False, 300),
    (4096, 128, np.float32, True, 0),
    (2100, 40, np.float64, True, 700),
]


def _dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda", dtype).t()


def _windows():
    out = []
    for i, (N, M, ft, weighted, _) in enumerate(WINDOWS):
        X = synth.waves(N, M, n_waves=min(6, M // 3), noise=1e-3, seed=300 + i)
        X = X.astype(ft).astype(np.float64)            # the values the device sees
        w = synth.log_uniform_weights(N, seed=310 + i) if weighted else None
        out.append((X, w, ft))
    return out


def _run(prec, kmodes, mode_kind=pg.MODES_ORTHONORMAL, with_bins=True):
    wins = _windows()
    bins = [np.asfortranarray(synth.spod_bin(2500, 30, seed=320)),
            np.asfortranarray(synth.complex_known_spectrum(3000, 50, seeds=(321, 322), dtype=np.complex64)[0])]
    Xd = [_dev(X, torch.float32 if ft == np.float32 else torch.float64) for X, _, ft in wins]
    Wd = [None if w is None else torch.from_numpy(w).cuda() for _, w, _ in wins]
    Bd = [_dev(B, torch.complex64) for B in bins] if with_bins else []
    hints = [h for *_, h in WINDOWS] + [0] * len(Bd)
    bp = pg.BatchedPOD(Xd, weights=Wd, remove_mean=True, mode_kind=mode_kind, kmodes=kmodes, prec=prec,
                       leaf_rows=hints, bins=Bd)
    bp.run()
    assert bp.status() == pg.OK
    return bp, wins, bins if with_bins else []


@pytest.mark.parametrize("kmodes", [8, 32])
def test_windows_fp64_match_oracle(kmodes):
    bp, wins, bins = _run(pg.PREC_FP64, kmodes)
    for i, (X, w, _) in enumerate(wins):
        ref = oracle.pod(X, w=w, remove_mean=True)
        k = bp.k[i]
        assert k == min(kmodes, X.shape[1])
        S = bp.S[i].cpu().numpy()
        parity.check_sigma(S, ref["S"])
        parity.check_vectors(bp.modes[i].cpu().numpy(), ref["U"], ref["S"], ncols=k)
        parity.check_vectors(bp.VT[i].cpu().numpy()[:k].T, ref["VT"][:k].T, ref["S"], ncols=k)
        np.testing.assert_allclose(bp.mean[i].cpu().numpy(), ref["mean"], rtol=0, atol=1e-13)
        # same sign rule as the oracle: separated modes agree as vectors
        U = bp.modes[i].cpu().numpy()
        for grp in parity.clusters(ref["S"]):
            if len(grp) == 1 and grp[0] < k:
                j = grp[0]
                assert np.linalg.norm(U[:, j] - ref["U"][:, j]) <= 1e-8, (i, j)
    for f, B in enumerate(bins):
        U_ref, S_ref, _, _ = oracle.zsvd(B.astype(np.complex128))
        S = bp.S[len(wins) + f].cpu().numpy()
        assert np.max(np.abs(S - S_ref)) <= 1e-12 * S_ref[0]


def test_windows_mixed_match_oracle():
    bp, wins, _ = _run(pg.PREC_MIXED_3XTF32, 8, with_bins=False)
    for i, (X, w, _) in enumerate(wins):
        ref = oracle.pod(X, w=w, remove_mean=True)
        S = bp.S[i].cpu().numpy()
        assert np.max(np.abs(S - ref["S"])) <= 2e-6 * ref["S"][0], i
        keep = [j for j in range(bp.k[i]) if ref["S"][j] >= 1e-3 * ref["S"][0]]
        parity.check_vectors(bp.modes[i].cpu().numpy().astype(np.float64)[:, keep], ref["U"][:, keep],
                             ref["S"][keep], ncols=len(keep))


def test_windows_physical_modes_and_graph_replay():
    bp, wins, _ = _run(pg.PREC_FP64, 8, mode_kind=pg.MODES_PHYSICAL, with_bins=False)
    for i, (X, w, _) in enumerate(wins):
        ref = oracle.pod(X, w=w, remove_mean=True, mode_kind=pg.MODES_PHYSICAL)
        parity.check_vectors(bp.modes[i].cpu().numpy(), ref["U"], ref["S"], ncols=bp.k[i],
                             weight=w if w is not None else None)
    torch.cuda.synchronize()
    S0 = bp.S_all.clone()
    U0 = [u.clone() for u in bp.U]
    bp.capture()
    bp.S_all.zero_()
    bp.replay()
    torch.cuda.synchronize()
    assert bp.status() == pg.OK
    assert torch.equal(bp.S_all, S0)
    for u, u0 in zip(bp.U, U0):
        assert torch.equal(u, u0)


def test_window_nonfinite_and_bad_weight():
    X = synth.waves(800, 10, n_waves=2, noise=1e-3, seed=330)
    X[3, 4] = np.inf
    bp = pg.BatchedPOD([_dev(X, torch.float64)], kmodes=2)
    bp.run()
    assert bp.status() == pg.ERR_NONFINITE
    X = synth.waves(800, 10, n_waves=2, noise=1e-3, seed=331)
    w = np.ones(800)
    w[7] = -1.0
    bp = pg.BatchedPOD([_dev(X, torch.float64)], weights=[torch.from_numpy(w).cuda()], kmodes=2)
    bp.run()
    assert bp.status() == pg.ERR_NONFINITE
