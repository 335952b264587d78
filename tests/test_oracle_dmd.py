"""Pins of the exact-DMD oracle (Sec. 3.2, Algs. 3-5) against facts fixed by
the mathematics, not by the oracle's own formulas:

* data made of K exact oscillations c_k psi_k lambda_k^t (and conjugates):
  the DMD eigenvalues are the lambda_k, each mode times its amplitude is the
  oscillation's own vector c_k psi_k / 2, and the reconstruction of Y1 is
  exact (pins Y2 vs Y1, V S^-1, the 1/mu of the modes, the Vandermonde's
  first power and the amplitude formula together);
* noisy data: the amplitudes equal a brute-force least-squares solve of the
  objective they minimise (pins P, q and the conjugate in P);
* every exact mode is an eigenvector of Y2 Y1^+ (Tu et al.'s defining
  property), checked against an explicit pseudo-inverse;
* a single real decaying mode; invariance under a constant offset with the
  mean removed; the order of modes and conjugate pairs."""
import numpy as np
import pytest

from oracle import dmd as odmd


def _oscillations(N, M, lams, cs, seed, offset=0.0):
    rng = np.random.default_rng(seed)
    t = np.arange(M)
    D = np.full((N, M), offset, dtype=np.float64)
    parts = []
    for lam, c in zip(lams, cs):
        psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        D += np.real(c * psi[:, None] * lam ** t[None, :])
        parts.append(c * psi / 2.0)
    return D, parts


LAMS = [0.97 * np.exp(0.3j), np.exp(0.71j), 1.01 * np.exp(1.4j)]
CS = [2.0, 1.0 + 0.5j, 0.4]


def test_closed_form_oscillations():
    N, M = 80, 40
    D, parts = _oscillations(N, M, LAMS, CS, seed=1)
    out = odmd.dmd(D, remove_mean=False)
    assert out["r"] == 6                            # numerical rank of Y1: 2 per oscillation
    mu, b, Phi = out["mu"], out["b"], out["Phi"]
    for lam, part in zip(LAMS, parts):
        i = int(np.argmin(np.abs(mu - lam)))
        assert abs(mu[i] - lam) <= 1e-11
        j = int(np.argmin(np.abs(mu - np.conj(lam))))
        assert abs(mu[j] - np.conj(lam)) <= 1e-11
        err = np.linalg.norm(Phi[:, i] * b[i] - part) / np.linalg.norm(part)
        assert err <= 1e-9, err
    Vand = odmd.vandermonde(mu, M - 1)
    rec = (Phi * b[None, :]) @ Vand
    assert np.max(np.abs(rec - D[:, :-1])) <= 1e-9 * np.max(np.abs(D))


def test_amplitudes_equal_least_squares():
    import oracle
    rng = np.random.default_rng(2)
    N, M, r = 120, 30, 10
    D, _ = _oscillations(N, M, LAMS, CS, seed=3)
    D += 0.05 * rng.standard_normal((N, M))
    out = odmd.dmd(D, remove_mean=True, r_max=r)
    assert out["r"] == r
    Y = D - D.mean(axis=1, keepdims=True)
    pod = oracle.pod(np.asfortranarray(Y[:, :-1]), remove_mean=False, r_max=r)
    S, VT = pod["S"][:r], pod["VT"][:r]
    lam, W = np.linalg.eig(out["A"])
    W = odmd.normalize_eigvecs(W)
    # brute force: min_b || S V^T - sum_i b_i w_i v_i^T ||_F as a dense complex
    # least-squares problem (v_i = row i of the Vandermonde matrix)
    Vand = odmd.vandermonde(lam, M - 1)
    G = (S[:, None] * VT).astype(np.complex128)
    Amat = np.stack([np.outer(W[:, i], Vand[i]).reshape(-1) for i in range(r)], axis=1)
    b_ls, *_ = np.linalg.lstsq(Amat, G.reshape(-1), rcond=None)
    tol = 1e-8 * np.max(np.abs(b_ls))
    np.testing.assert_allclose(odmd.amplitudes(lam, W, S, VT), b_ls, rtol=0, atol=tol)
    for i, m in enumerate(out["mu"]):           # the sorted output carries the same amplitudes
        k = int(np.argmin(np.abs(lam - m)))
        assert abs(out["b"][i] - b_ls[k]) <= tol


def test_modes_are_eigenvectors_of_y2_y1_pinv():
    rng = np.random.default_rng(4)
    N, M = 50, 16
    D, _ = _oscillations(N, M, LAMS, CS, seed=5)
    D += 0.1 * rng.standard_normal((N, M))
    out = odmd.dmd(D, remove_mean=False)
    r = out["r"]
    assert r == M - 1
    Y1, Y2 = D[:, :-1], D[:, 1:]
    Afull = Y2 @ np.linalg.pinv(Y1)
    for i in range(r):
        phi = out["Phi"][:, i]
        res = np.linalg.norm(Afull @ phi - out["mu"][i] * phi)
        assert res <= 1e-9 * np.linalg.norm(phi) * max(1.0, abs(out["mu"][i])), (i, res)


def test_single_real_decaying_mode():
    rng = np.random.default_rng(6)
    N, M, lam = 40, 12, 0.9
    psi = rng.standard_normal(N)
    D = psi[:, None] * lam ** np.arange(M)[None, :]
    out = odmd.dmd(D, remove_mean=False)
    assert out["r"] == 1
    assert abs(out["mu"][0] - lam) <= 1e-13
    np.testing.assert_allclose(out["Phi"][:, 0] * out["b"][0], psi, rtol=0, atol=1e-12 * np.abs(psi).max())


def test_constant_offset_removed_with_mean():
    rng = np.random.default_rng(7)
    D, _ = _oscillations(60, 25, LAMS, CS, seed=8)
    D += 0.01 * rng.standard_normal(D.shape)
    a = odmd.dmd(D, remove_mean=True, r_max=8)
    bb = odmd.dmd(D + 3.5, remove_mean=True, r_max=8)
    np.testing.assert_allclose(a["mu"], bb["mu"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(a["Phi"] * a["b"][None, :], bb["Phi"] * bb["b"][None, :], rtol=0,
                               atol=1e-9 * np.abs(a["Phi"] * a["b"][None, :]).max())


def test_order_rule():
    rng = np.random.default_rng(9)
    D, _ = _oscillations(70, 30, LAMS, CS, seed=10)
    D += 0.02 * rng.standard_normal(D.shape)
    out = odmd.dmd(D, remove_mean=True, r_max=12)
    mu, b = out["mu"], out["b"]
    r = out["r"]
    key = np.abs(b)
    i = 0
    prev = np.inf
    while i < r:
        if mu[i].imag != 0.0:
            assert mu[i].imag > 0.0 and mu[i + 1] == np.conj(mu[i])   # pair adjacent, Im > 0 first
            k = max(key[i], key[i + 1])
            i += 2
        else:
            k = key[i]
            i += 1
        assert k <= prev
        prev = k


def test_eigvec_normalisation_and_vandermonde():
    W = np.array([[1.0 + 1.0j, 0.1], [-3.0j, 2.0]])
    Wn = odmd.normalize_eigvecs(W)
    np.testing.assert_allclose(np.linalg.norm(Wn, axis=0), 1.0, rtol=1e-15)
    assert Wn[1, 0].imag == 0.0 and Wn[1, 0].real > 0.0
    assert Wn[1, 1].imag == 0.0 and Wn[1, 1].real > 0.0
    V = odmd.vandermonde(np.array([2.0, 1j]), 4)
    np.testing.assert_array_equal(V, np.array([[1, 2, 4, 8], [1, 1j, -1, -1j]]))


@pytest.mark.parametrize("mutation", ["vand_from_one", "no_conj_in_P", "modes_from_y1", "no_inv_mu"])
def test_pins_catch_planted_mistakes(mutation, monkeypatch):
    """A plausible mistake planted in the oracle (on the CPU) fails a pin."""
    if mutation == "vand_from_one":
        orig = odmd.vandermonde
        monkeypatch.setattr(odmd, "vandermonde", lambda mu, n: orig(mu, n + 1)[:, 1:])
    elif mutation == "no_conj_in_P":
        def amp(mu, W, S, VT):
            Vand = odmd.vandermonde(mu, VT.shape[1])
            P = (W.conj().T @ W) * (Vand @ Vand.conj().T)
            q = np.conj(np.diag(Vand @ (S[:, None] * VT).T @ W))
            L = np.linalg.cholesky(P)
            return np.linalg.solve(L.conj().T, np.linalg.solve(L, q))
        monkeypatch.setattr(odmd, "amplitudes", amp)
    elif mutation == "modes_from_y1":
        monkeypatch.setattr(odmd, "shifted_pair", lambda Y: (Y[:, :-1], Y[:, :-1]))
    elif mutation == "no_inv_mu":
        orig = odmd.exact_modes
        monkeypatch.setattr(odmd, "exact_modes", lambda Y2, VT, S, W, mu: orig(Y2, VT, S, W, mu) * mu[None, :])
    failed = 0
    for pin in (test_closed_form_oscillations, test_amplitudes_equal_least_squares,
                test_modes_are_eigenvectors_of_y2_y1_pinv):
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, mutation


def test_rank_threshold_is_the_standard_rule():
    """r is cut to the numerical rank of Y1 with the standard threshold for an
    N x (M-1) matrix, max(N, M-1) * 2^-52 * s_1 (numpy.linalg.matrix_rank's
    default): a singular value between (M-1) 2^-52 s_1 and N 2^-52 s_1 counts
    as zero.  The data are built with that value, so the narrower rule would
    keep one more mode."""
    N, M = 4000, 9
    rng = np.random.default_rng(11)
    Q1, _ = np.linalg.qr(rng.standard_normal((N, 3)))
    Q2, _ = np.linalg.qr(rng.standard_normal((M - 1, 3)))
    s = np.array([1.0, 0.5, 1e-14])              # (M-1) eps = 1.8e-15 < 1e-14 < N eps = 8.9e-13
    Y1 = (Q1 * s) @ Q2.T
    D = np.concatenate([Y1, Y1[:, -1:] * 0.9], axis=1)
    assert np.linalg.matrix_rank(Y1) == 2
    assert np.sum(s > (M - 1) * 2.0 ** -52 * s[0]) == 3
    out = odmd.dmd(D, remove_mean=False)
    assert out["r"] == np.linalg.matrix_rank(Y1) == 2
