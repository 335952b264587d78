"""GPU parity of the exact DMD (Sec. 3.2, Algs. 3-5) through the C ABI
against the FP64 oracle of ``oracle/dmd.py`` on the same seeded inputs, and
against the closed form of oscillation data.

Tolerances: the inputs are sums of K oscillations with random spatial
vectors (a nearly normal A, eigenvalues with condition numbers near 1) plus
small noise, so both sides' eigenvalues agree to about 1e-13; 1e-10 is
used.  Amplitudes and mode-times-amplitude products pass through the
Cholesky solve of P (condition number of P up to about 1e3 here): 1e-8 of
their largest entry."""
import numpy as np
import pytest

import synth
from oracle import dmd as odmd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")


def _dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda", dtype).t()


def _compare(res, ref, tol_mu=1e-10, tol_b=1e-8):
    r = ref["r"]
    assert res.r == r
    mu = res.mu.cpu().numpy()
    b = res.b.cpu().numpy()
    Phi = res.Phi.cpu().numpy()
    np.testing.assert_allclose(mu, ref["mu"], rtol=0, atol=tol_mu)
    bmax = np.max(np.abs(ref["b"]))
    np.testing.assert_allclose(b, ref["b"], rtol=0, atol=tol_b * bmax)
    pb = Phi * b[None, :]
    pb_ref = ref["Phi"] * ref["b"][None, :]
    assert np.max(np.abs(pb - pb_ref)) <= tol_b * np.max(np.abs(pb_ref))
    # each mode equals the oracle's up to a unit phase (the same normalisation)
    for p in range(r):
        u, v = Phi[:, p], ref["Phi"][:, p]
        c = abs(np.vdot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v))
        assert c >= 1 - 1e-10, (p, c)


@pytest.mark.parametrize("N,M,K,b,dtype,remove_mean,noise", [
    (3000, 40, 6, 500, torch.float64, True, 1e-6),      # 12 modes, 6 leaves
    (4097, 33, 5, 700, torch.float32, False, 1e-5),     # F32 input, ragged leaves
    (20000, 400, 8, 4000, torch.float64, True, 1e-6),   # cooperative tree (M >= 384)
    (6000, 600, 10, 1000, torch.float64, False, 1e-6),  # binary32-preconditioned SVD of Y1 (M-1 >= 512)
])
def test_dmd_matches_oracle(N, M, K, b, dtype, remove_mean, noise):
    lam, amp = synth.oscillation_params(K, seed=K)
    D, _ = synth.oscillations(N, M, lam, amp, seed=N + M, noise=noise, offset=0.5 if remove_mean else 0.0)
    r = 2 * K
    Din = np.asarray(_dev(D, dtype).cpu().numpy(), dtype=np.float64)   # what the device sees
    ref = odmd.dmd(Din, remove_mean=remove_mean, r_max=r)
    res = pg.dmd(_dev(D, dtype), remove_mean=remove_mean, r_max=r, leaf_rows=b)
    _compare(res, ref)
    np.testing.assert_allclose(res.S.cpu().numpy(), ref["S"], rtol=0, atol=1e-12 * ref["S"][0])


@pytest.mark.parametrize("K", [20, 65, 100])
def test_dmd_eigensolver_residency(K):
    """r = 40, 130, 200: the Schur form and vectors in shared memory, the
    Schur form only, and neither (global memory)."""
    N, M = 5000, 2 * K + 40
    lam, amp = synth.oscillation_params(K, seed=3)
    D, _ = synth.oscillations(N, M, lam, amp, seed=7, noise=1e-7)
    ref = odmd.dmd(D, remove_mean=False, r_max=2 * K)
    res = pg.dmd(_dev(D), remove_mean=False, r_max=2 * K)
    _compare(res, ref, tol_mu=1e-9, tol_b=1e-7)


def test_dmd_closed_form():
    N, M, K = 1 << 17, 64, 4
    lam, amp = synth.oscillation_params(K, seed=11)
    D, parts = synth.oscillations(N, M, lam, amp, seed=12)
    res = pg.dmd(_dev(D), remove_mean=False)
    assert res.r == 2 * K                          # numerical rank of Y1
    mu = res.mu.cpu().numpy()
    pb = res.Phi.cpu().numpy() * res.b.cpu().numpy()[None, :]
    for l_k, part in zip(lam, parts):
        i = int(np.argmin(np.abs(mu - l_k)))
        assert abs(mu[i] - l_k) <= 1e-11
        assert np.linalg.norm(pb[:, i] - part) <= 1e-9 * np.linalg.norm(part)
        j = int(np.argmin(np.abs(mu - np.conj(l_k))))
        assert np.linalg.norm(pb[:, j] - np.conj(part)) <= 1e-9 * np.linalg.norm(part)
    # order: |b| descending, conjugate pairs adjacent with Im > 0 first
    bb = np.abs(res.b.cpu().numpy())
    assert np.all(np.diff(bb[::2]) <= 1e-12 * bb[0])
    assert np.all(mu[::2].imag > 0) and np.allclose(mu[1::2], np.conj(mu[::2]), rtol=0, atol=0)


def test_dmd_real_decaying_mode_and_edges():
    rng = np.random.default_rng(1)
    N, M = 3000, 12
    psi = rng.standard_normal(N)
    D = np.asfortranarray(psi[:, None] * 0.9 ** np.arange(M)[None, :])
    res = pg.dmd(_dev(D), remove_mean=False)
    assert res.r == 1
    assert abs(res.mu.cpu().numpy()[0] - 0.9) <= 1e-13
    np.testing.assert_allclose(res.Phi.cpu().numpy()[:, 0] * res.b.cpu().numpy()[0], psi, rtol=0,
                               atol=1e-12 * np.abs(psi).max())
    # all-zero data: rank 0, no modes, no error
    z = pg.dmd(torch.zeros((500, 10), dtype=torch.float64, device="cuda"), remove_mean=False)
    assert z.r == 0
    # two snapshots: one real eigenvalue
    D2 = np.asfortranarray(np.stack([psi, 0.5 * psi + 1e-3 * rng.standard_normal(N)], axis=1))
    ref = odmd.dmd(D2, remove_mean=False)
    res2 = pg.dmd(_dev(D2), remove_mean=False)
    _compare(res2, ref)


def test_dmd_rejects_bad_shapes():
    X = torch.zeros((100, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(pg.PylomError):
        pg.dmd(X[:, :1])                 # one snapshot
    with pytest.raises(pg.PylomError):
        pg.dmd(X, r_max=10)              # r_max > M - 1


def test_dmd_graph_replay_is_repeatable():
    N, M, K = 8192, 48, 6
    lam, amp = synth.oscillation_params(K, seed=5)
    D, _ = synth.oscillations(N, M, lam, amp, seed=6, noise=1e-6)
    X = _dev(D)
    res = pg.dmd(X, r_max=2 * K)
    ws = res.workspace
    mu = torch.empty(4 * K, dtype=torch.float64, device="cuda")
    b = torch.empty_like(mu)
    Phi = pg.empty_colmajor(N, 2 * K, torch.float64, "cuda")
    S = torch.empty(M - 1, dtype=torch.float64, device="cuda")
    mean = torch.empty(N, dtype=torch.float64, device="cuda")
    r_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    out = (mu, b, Phi, S, mean, r_dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        pg.dmd(X, r_max=2 * K, workspace=ws, out=out, stream=s, check=False)   # warm-up outside the graph
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pg.dmd(X, r_max=2 * K, workspace=ws, out=out, stream=s, check=False)
    g.replay()
    torch.cuda.synchronize()
    first = (mu.clone(), b.clone(), Phi.clone())
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(first[0], mu) and torch.equal(first[1], b) and torch.equal(first[2], Phi)
    assert torch.equal(mu[: 4 * K], torch.view_as_real(res.mu).reshape(-1))


def test_rank_threshold_matches_oracle():
    """A singular value of Y1 between (M-1) 2^-52 s_1 and N 2^-52 s_1: the
    standard threshold max(N, M-1) 2^-52 s_1 drops it on both sides."""
    N, M = 4000, 9
    rng = np.random.default_rng(11)
    Q1, _ = np.linalg.qr(rng.standard_normal((N, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((M - 1, 3)))
    Y1 = (Q1 * np.array([1.0, 0.5, 1e-14])) @ Q2.T
    D = np.concatenate([Y1, Y1[:, -1:] * 0.9], axis=1)
    ref = odmd.dmd(D, remove_mean=False)
    res = pg.dmd(_dev(D), remove_mean=False, leaf_rows=1000)
    assert ref["r"] == 2
    _compare(res, ref)
