"""GPU parity of the SPOD front end (Sec. 2.3, Alg. 6) and of the whole SPOD
(front end + per-frequency SVDs in one persistent launch + ordering)
against the FP64 oracle of ``oracle/spod.py`` on the same seeded data.

Tolerances: the front end works in FP32 with a direct transform of npwin
terms, so each Q entry carries about sqrt(npwin) 2^-24 of the block's
windowed amplitude; 2e-6 of the largest |Q| of the frequency bounds it.
Energies of the complex64 SVDs: 2e-6 of the largest energy (the mixed
batched path's singular values are held to 2e-6 S_max)."""
import numpy as np
import pytest

from oracle import spod as osp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")


def _dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.float64).T)).to("cuda", dtype).t()


def _waves(N, T, seed):
    rng = np.random.default_rng(seed)
    x = np.linspace(0, 2 * np.pi, N, endpoint=False)
    t = np.arange(T)
    return (1.0 + 0.3 * np.cos(x)[:, None]
            + 2.0 * np.cos(3 * x[:, None] - 2 * np.pi * 3 * t[None, :] / 32)
            + 1.5 * np.cos(5 * x[:, None] - 2 * np.pi * 10 * t[None, :] / 32)
            + 0.05 * rng.standard_normal((N, T)))


@pytest.mark.parametrize("N,T,npwin,nolap,remove_mean,dtype", [
    (1000, 300, 32, 16, True, torch.float64),
    (777, 301, 60, 30, False, torch.float32),   # the paper's window and overlap
    (129, 64, 64, 0, True, torch.float32),      # one block
    (300, 250, 15, 5, True, torch.float64),     # odd window
    (500, 420, 100, 50, True, torch.float32),   # window above 64: the direct transform
])
def test_spod_blocks_match_oracle(N, T, npwin, nolap, remove_mean, dtype):
    D = _waves(N, T, seed=N + T)
    Q_ref = osp.spod_blocks(D, npwin, nolap, remove_mean)            # nfreq x N x nBlks
    Q = pg.spod_blocks(_dev(D, dtype), npwin, nolap, remove_mean)    # nfreq x nBlks x N
    Qn = Q.cpu().numpy().transpose(0, 2, 1).astype(np.complex128)
    assert Qn.shape == Q_ref.shape
    for k in range(Q_ref.shape[0]):
        # relative to the largest |Q| (the windowed amplitude of the data);
        # FP32 input adds its own rounding (2^-24 of the data amplitude)
        tol = 2e-6 if dtype == torch.float64 else 4e-6
        err = np.max(np.abs(Qn[k] - Q_ref[k])) / np.max(np.abs(Q_ref))
        assert err <= tol, (k, err)


def test_spod_blocks_rejects_bad_shapes():
    D = torch.zeros((10, 20), dtype=torch.float32, device="cuda")
    with pytest.raises(pg.PylomError):
        pg.spod_blocks(D, 32, 0)          # T < npwin
    with pytest.raises(pg.PylomError):
        pg.spod_blocks(D, 8, 8)           # nolap >= npwin


def test_spod_end_to_end_matches_oracle():
    N, T, npwin, nolap = 4096, 32 * 17 + 16, 32, 16
    D = _waves(N, T, seed=9)
    ref = osp.spod(D, 0.1, npwin, nolap, remove_mean=True, kmodes=4)
    sp = pg.SPOD(_dev(D, torch.float32), 0.1, npwin, nolap, remove_mean=True, kmodes=4)
    sp.run()
    assert sp.status() == pg.OK
    L = sp.L.cpu().numpy()
    Lmax = ref["L"].max()
    assert np.max(np.abs(L - ref["L"])) <= 2e-6 * Lmax
    order = sp.order.cpu().numpy()
    assert list(order[:2]) == list(ref["order"][:2]) == [3, 10]
    np.testing.assert_allclose(sp.f.cpu().numpy(), ref["f"], rtol=1e-15)
    # the leading mode of the two wave frequencies, up to phase
    for k in (3, 10):
        u = sp.modes[k][:, 0].cpu().numpy().astype(np.complex128)
        v = ref["U"][k][:, 0]
        assert abs(np.vdot(u, v)) >= 1 - 1e-5


def test_spod_graph_replay_is_repeatable():
    N, T, npwin, nolap = 2048, 32 * 9 + 16, 32, 16
    D = _dev(_waves(N, T, seed=4), torch.float32)
    sp = pg.SPOD(D, 0.1, npwin, nolap, kmodes=2)
    sp.capture()
    sp.replay()
    torch.cuda.synchronize()
    L1, U1, o1 = sp.L.clone(), sp.modes[3].clone(), sp.order.clone()
    sp.replay()
    torch.cuda.synchronize()
    assert torch.equal(L1, sp.L) and torch.equal(U1, sp.modes[3]) and torch.equal(o1, sp.order)
