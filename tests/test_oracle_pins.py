"""Pins of the FP64 CPU oracle to facts outside itself.

Each test checks the oracle against something the paper or the mathematics
fixes: closed-form spectra, brute force on tiny inputs, invariants of the
SVD/QR (Eqs. svdqr1-svdqr3), special cases, and the cumulative-energy
truncation of Sec. 3.1.  The set is chosen so that a dropped term, a wrong
sign or index, or a transposed operand in the oracle fails at least one.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import closed_forms as cf

EPS = 2.0 ** -52


def _rng(seed):
    return np.random.default_rng(seed)


def _jacobi_eigs_pure_python(G):
    """Two-sided cyclic Jacobi eigenvalues of a small symmetric matrix, pure
    Python (a different algorithm from the oracle's one-sided SVD)."""
    A = [list(map(float, row)) for row in G]
    n = len(A)
    for _ in range(100):
        off = sum(A[i][j] ** 2 for i in range(n) for j in range(n) if i != j)
        if off < 1e-60:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if A[p][q] == 0.0:
                    continue
                theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q])
                t = math.copysign(1.0, theta) / (abs(theta) + math.sqrt(theta * theta + 1.0))
                c = 1.0 / math.sqrt(t * t + 1.0)
                s = t * c
                for k in range(n):
                    akp, akq = A[k][p], A[k][q]
                    A[k][p] = c * akp - s * akq
                    A[k][q] = s * akp + c * akq
                for k in range(n):
                    apk, aqk = A[p][k], A[q][k]
                    A[p][k] = c * apk - s * aqk
                    A[q][k] = s * apk + c * aqk
    return sorted((A[i][i] for i in range(n)), reverse=True)


# ---------------------------------------------------------------------------
# QR (Eq. svdqr1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,M", [(50, 7), (300, 40), (64, 64)])
def test_qr_invariants(N, M):
    A = _rng(10 + M).standard_normal((N, M))
    R, Q = oracle.tsqr(A)
    nA = np.linalg.norm(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    # R^T R = A^T A  (fixes R up to row signs)
    assert np.linalg.norm(R.T @ R - A.T @ A) <= 50 * EPS * nA ** 2
    # Q R = A and Q^T Q = I
    assert np.linalg.norm(Q @ R - A) <= 50 * EPS * nA
    assert np.linalg.norm(Q.T @ Q - np.eye(M)) <= 50 * EPS * math.sqrt(M)
    # |R_ii| agrees with a library QR (row signs are convention)
    Rl = np.linalg.qr(A, mode="r")
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-12, atol=1e-12 * nA)


def test_qr_householder_sign_convention():
    # beta = -sign(alpha) ||x||: R_ii has the opposite sign of the pivot
    A = np.array([[3.0, 1.0], [4.0, 2.0], [0.0, 5.0]])
    packed, tau = oracle.householder_qr(A)
    assert packed[0, 0] == pytest.approx(-5.0, abs=1e-15)
    assert tau[0] == pytest.approx((-5.0 - 3.0) / -5.0, abs=1e-15)
    # v_0 = [1, 4 / (3 + 5), 0]
    assert packed[1, 0] == pytest.approx(0.5, abs=1e-15)
    # a column already in triangular form needs no reflector
    B = np.array([[2.0, 1.0], [0.0, 3.0], [0.0, 0.0]])
    packed, tau = oracle.householder_qr(B)
    assert tau[0] == 0.0 and packed[0, 0] == 2.0


def test_apply_q_is_orthogonal_and_reproduces_A():
    A = _rng(3).standard_normal((40, 6))
    packed, tau = oracle.householder_qr(A)
    R = np.triu(packed[:6, :])
    I = np.zeros((40, 40)); np.fill_diagonal(I, 1.0)
    Qfull = oracle.apply_q(packed, tau, I)
    assert np.linalg.norm(Qfull.T @ Qfull - np.eye(40)) < 1e-13
    RR = np.zeros((40, 6)); RR[:6] = R
    assert np.linalg.norm(Qfull @ RR - A) < 1e-13 * np.linalg.norm(A)


# ---------------------------------------------------------------------------
# SVD (Eq. svdqr2)
# ---------------------------------------------------------------------------

def test_svd_closed_form_spectrum():
    N, M = 2000, 40
    X, _, s = synth.known_spectrum(N, M, weights=False, seeds=(21, 22, 23))
    res = oracle.pod(X, remove_mean=False)
    S = res["S"]
    assert np.max(np.abs(S - s)) <= 1e-13 * s[0]
    big = s >= 1e-2 * s[0]
    assert np.max(np.abs(S[big] - s[big]) / s[big]) <= 1e-12


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 6])
def test_svd_brute_force_tiny(M):
    N = 9
    Y = _rng(100 + M).standard_normal((N, M))
    U, S, V, sw = oracle.svd(Y)
    assert sw > 0
    lam = _jacobi_eigs_pure_python(Y.T @ Y)
    ref = np.sqrt(np.maximum(lam, 0.0))
    assert np.allclose(S, ref, rtol=1e-12, atol=1e-13 * ref[0])
    ref2 = np.sqrt(np.maximum(np.linalg.eigvalsh(Y.T @ Y)[::-1], 0.0))
    assert np.allclose(S, ref2, rtol=1e-12, atol=1e-13 * ref2[0])


def test_svd_2x2_closed_form():
    Y = np.array([[2.0, 1.0], [0.5, -3.0], [1.0, 1.0]])
    G = Y.T @ Y
    l1, l2 = cf.sym2x2_eigs(G[0, 0], G[0, 1], G[1, 1])
    _, S, _, _ = oracle.svd(Y)
    assert S[0] == pytest.approx(math.sqrt(l1), rel=1e-14)
    assert S[1] == pytest.approx(math.sqrt(l2), rel=1e-13)


@pytest.mark.parametrize("N,M,seed", [(200, 16, 1), (120, 33, 2), (64, 64, 3)])
def test_svd_invariants(N, M, seed):
    Y = _rng(seed).standard_normal((N, M)) * np.logspace(0, -5, M)[None, :]
    U, S, V, sw = oracle.svd(Y)
    assert sw > 0
    nY = np.linalg.norm(Y)
    assert np.linalg.norm(Y - (U * S) @ V.T) / nY <= 1e-13
    assert np.linalg.norm(U.T @ U - np.eye(M)) <= 1e-13
    assert np.linalg.norm(V.T @ V - np.eye(M)) <= 1e-13
    assert np.all(np.diff(S) <= 0.0)
    # sign convention: the largest-magnitude entry of each v_i is positive
    for i in range(M):
        k = int(np.argmax(np.abs(V[:, i])))
        assert V[k, i] > 0.0


def test_jacobi_nonconvergence_flag():
    Y = _rng(5).standard_normal((30, 12))
    _, _, _, sw = oracle.jacobi_svd_raw(Y, max_sweeps=1)
    assert sw == -1
    _, _, _, sw = oracle.jacobi_svd_raw(Y, max_sweeps=60)
    assert 1 < sw <= 60


def test_svd_special_cases():
    # rank one: sigma_0 = |u||v|, the rest vanish
    u = _rng(6).standard_normal(50); v = _rng(7).standard_normal(8)
    _, S, V, _ = oracle.svd(np.outer(u, v))
    assert S[0] == pytest.approx(np.linalg.norm(u) * np.linalg.norm(v), rel=1e-14)
    assert np.all(S[1:] <= 1e-14 * S[0])
    assert abs(abs(V[:, 0] @ v) / np.linalg.norm(v) - 1.0) < 1e-14
    # diagonal: singular values are the sorted magnitudes
    d = np.array([0.5, -3.0, 2.0, 0.0, -1.0])
    D = np.zeros((9, 5)); D[np.arange(5), np.arange(5)] = d
    U, S, V, _ = oracle.svd(D)
    assert np.array_equal(S, np.array([3.0, 2.0, 1.0, 0.5, 0.0]))
    assert np.linalg.norm(U.T @ U - np.eye(5)) < 1e-14   # basis completed for sigma = 0
    # zero matrix: all zero, orthonormal U and V
    U, S, V, _ = oracle.svd(np.zeros((7, 4)))
    assert np.all(S == 0.0)
    assert np.linalg.norm(U.T @ U - np.eye(4)) < 1e-14
    assert np.linalg.norm(V.T @ V - np.eye(4)) < 1e-14


# ---------------------------------------------------------------------------
# POD driver (Alg. 2 + Eqs. svdqr1-3), mean, weights, truncation
# ---------------------------------------------------------------------------

def test_pod_waves_closed_form():
    N, M = 4096, 64
    X = synth.waves(N, M, n_waves=8, noise=0.0)
    res = oracle.pod(X, remove_mean=True)
    ref = cf.waves_sigma(N, M, 8)
    S = res["S"]
    assert np.allclose(S[:16], ref, rtol=1e-12)
    assert np.all(S[16:] <= 1e-12 * S[0])
    # mean field 1 + 0.5 cos x is removed exactly
    x = 2 * np.pi * np.arange(N) / N
    assert np.allclose(res["mean"], 1.0 + 0.5 * np.cos(x), atol=1e-13)


def test_pod_mean_constant_rows():
    # integer-valued rows: the mean is exact, so Y is exactly zero
    c = np.round(100 * _rng(8).standard_normal(30))
    X = np.repeat(c[:, None], 5, axis=1)
    res = oracle.pod(X, remove_mean=True)
    assert np.array_equal(res["mean"], c)
    assert np.all(res["S"] == 0.0)
    assert res["r"] == 5
    U = res["U"]
    assert np.linalg.norm(U.T @ U - np.eye(5)) < 1e-14


def test_pod_mean_matches_definition():
    X = _rng(9).standard_normal((100, 13))
    res = oracle.pod(X, remove_mean=True)
    assert np.allclose(res["mean"], X.mean(axis=1), rtol=1e-14, atol=1e-15)
    Y, mean = oracle.center_weight(X, None, True)
    assert np.allclose(Y, X - X.mean(axis=1)[:, None], atol=1e-15)


@pytest.mark.parametrize("remove_mean", [False, True])
def test_pod_invariants_and_parseval(remove_mean):
    N, M = 700, 24
    X = _rng(11).standard_normal((N, M)) + 3.0
    w = synth.log_uniform_weights(N, 12)
    res = oracle.pod(X, w=w, remove_mean=remove_mean)
    Y, _ = oracle.center_weight(X, w, remove_mean)
    U, S, V = res["U"], res["S"], res["VT"].T
    nY = np.linalg.norm(Y)
    assert abs(np.sum(S ** 2) - nY ** 2) <= 1e-13 * nY ** 2          # Parseval
    assert np.linalg.norm(Y - (U * S) @ V.T) / nY <= 1e-13
    assert np.linalg.norm(U.T @ U - np.eye(M)) <= 1e-13
    assert np.all(np.diff(S) <= 0.0)


def test_pod_known_spectrum_with_weights():
    N, M = 3000, 32
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(31, 32, 33))
    res = oracle.pod(X, w=w, remove_mean=False, mode_kind=1)
    S = res["S"]
    assert np.max(np.abs(S - s)) <= 1e-13 * s[0]
    Phi = res["U"]
    # physical modes are orthonormal in the w-weighted inner product (Sec. 2.1)
    G = Phi.T @ (w[:, None] * Phi)
    assert np.linalg.norm(G - np.eye(M)) <= 1e-12


def test_pod_uniform_weight_scaling():
    X = _rng(13).standard_normal((400, 10))
    c = 7.0
    r1 = oracle.pod(X, w=None, remove_mean=True, mode_kind=1)
    r2 = oracle.pod(X, w=np.full(400, c), remove_mean=True, mode_kind=1)
    assert np.allclose(r2["S"], math.sqrt(c) * r1["S"], rtol=1e-13)
    # U_w (the left vectors of sqrt(c) Y) is unchanged up to sign, so the
    # physical modes Phi = U_w / sqrt(c) shrink by sqrt(c) and stay
    # orthonormal in the weighted inner product sum_n c Phi_i Phi_j.
    # (mean removal makes Y rank M-1: the last mode is an arbitrary unit
    # vector orthogonal to the rest and is left out of the alignment check)
    P1, P2 = r1["U"], r2["U"]
    keep = r1["S"] > 1e-10 * r1["S"][0]
    assert keep.sum() == 9
    d = np.abs(np.sum(P1 * P2, axis=0))[keep] * math.sqrt(c)
    assert np.allclose(d, 1.0, atol=1e-12)
    assert np.allclose(c * (P2.T @ P2), np.eye(10), atol=1e-12)


def test_truncation_closed_form():
    M = 256
    s = synth.spectrum(M, 6.0)
    r_cf = cf.truncation_rank(M, 6.0, 0.99)
    assert r_cf == 43
    assert oracle.truncation_rank(s, 0.99, M) == 43
    assert oracle.truncation_rank(s, 0.99, 10) == 10
    assert oracle.truncation_rank(s, 0.0, 17) == 17
    assert oracle.truncation_rank(np.array([3.0, 4.0]), 0.64, 2) == 2   # 9/25 < 0.64
    assert oracle.truncation_rank(np.array([4.0, 3.0]), 0.64, 2) == 1   # 16/25 >= 0.64


def test_pod_truncated_modes_are_leading_vectors():
    N, M = 500, 20
    X, _, s = synth.known_spectrum(N, M, weights=False, seeds=(41, 42, 43))
    full = oracle.pod(X, remove_mean=False)
    tr = oracle.pod(X, remove_mean=False, energy=0.99)
    assert tr["r"] == cf.truncation_rank(M, 6.0, 0.99)
    assert np.allclose(tr["U"], full["U"][:, : tr["r"]], atol=1e-13)


def test_matmul_local_product():
    A = _rng(14).standard_normal((30, 7)); B = _rng(15).standard_normal((30, 5))
    assert np.allclose(oracle.matmul(A, B, transA=True), A.T @ B, rtol=1e-14, atol=1e-13)
    C = _rng(16).standard_normal((7, 30))
    assert np.allclose(oracle.matmul(C, B), C @ B, rtol=1e-14, atol=1e-13)


# ---------------------------------------------------------------------------
# truncated-POD reconstruction loss and its gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("remove_mean,weighted", [(False, True), (True, False), (True, True)])
def test_loss_gradient_matches_central_differences(remove_mean, weighted):
    N, M, r = 40, 6, 2
    s = np.array([4.0, 2.5, 1.0, 0.5, 0.2, 0.1])
    X, w, _ = synth.known_spectrum(N, M, s=s, weights=weighted, seeds=(61, 62, 63))
    X = X + 0.01 * _rng(64).standard_normal((N, M))
    L, G = oracle.pod_loss_grad(X, r, w=w, remove_mean=remove_mean)
    # the loss is the tail energy of the spectrum
    S = oracle.pod(X, w=w, remove_mean=remove_mean)["S"]
    assert L == pytest.approx(np.sum(S[r:] ** 2), rel=1e-12)
    h = 1e-6
    for (n, m) in [(0, 0), (3, 5), (17, 2), (39, 4), (25, 1)]:
        Xp = X.copy(); Xp[n, m] += h
        Xm = X.copy(); Xm[n, m] -= h
        fd = (oracle.pod_loss_grad(Xp, r, w=w, remove_mean=remove_mean, want_grad=False)[0]
              - oracle.pod_loss_grad(Xm, r, w=w, remove_mean=remove_mean, want_grad=False)[0]) / (2 * h)
        assert fd == pytest.approx(G[n, m], rel=1e-6, abs=1e-8 * np.abs(G).max())


def test_loss_gradient_vanishes_for_rank_r():
    # a rank-r snapshot matrix reconstructs exactly: L = 0 and dL/dX = 0
    N, M, r = 50, 5, 2
    X = _rng(70).standard_normal((N, r)) @ _rng(71).standard_normal((r, M))
    L, G = oracle.pod_loss_grad(X, r)
    assert abs(L) < 1e-24 * np.linalg.norm(X) ** 2 + 1e-26
    assert np.abs(G).max() < 1e-12 * np.abs(X).max()


# ---------------------------------------------------------------------------
# complex SVD (per-frequency SVDs of SPOD)
# ---------------------------------------------------------------------------

def test_zqr_reflector_convention():
    # H^H [alpha; x] = [beta; 0] with beta real and opposite in sign to Re(alpha)
    A = np.array([[3.0 + 4.0j], [0.0 + 0.0j], [12.0 + 0.0j]])
    packed, tau = oracle.zhouseholder_qr(A)
    assert packed[0, 0].imag == 0.0
    assert packed[0, 0].real == pytest.approx(-13.0, abs=1e-14)
    assert tau[0] == pytest.approx((-13.0 - (3.0 + 4.0j)) / -13.0, abs=1e-15)


def test_zsvd_closed_form_spectrum():
    N, M = 600, 24
    X, s = synth.complex_known_spectrum(N, M, seeds=(91, 92))
    U, S, V, sw = oracle.zsvd(X)
    assert sw > 0
    assert np.max(np.abs(S - s)) <= 1e-13 * s[0]
    nX = np.linalg.norm(X)
    assert np.linalg.norm(X - (U * S) @ V.conj().T) / nX <= 1e-13
    assert np.linalg.norm(U.conj().T @ U - np.eye(M)) <= 1e-12
    assert np.linalg.norm(V.conj().T @ V - np.eye(M)) <= 1e-12
    # phase rule: the largest |entry| of each v_i is real and positive
    for i in range(M):
        k = int(np.argmax(np.abs(V[:, i])))
        assert abs(V[k, i].imag) <= 1e-15 and V[k, i].real > 0


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_zsvd_brute_force_tiny(M):
    rng = _rng(200 + M)
    X = rng.standard_normal((11, M)) + 1j * rng.standard_normal((11, M))
    _, S, _, _ = oracle.zsvd(X)
    lam = np.linalg.eigvalsh(X.conj().T @ X)[::-1]
    assert np.allclose(S, np.sqrt(np.maximum(lam, 0.0)), rtol=1e-12, atol=1e-13 * np.sqrt(lam[0]))
    if M == 2:
        G = X.conj().T @ X     # Hermitian 2x2: (a + c)/2 +- sqrt(((a - c)/2)^2 + |b|^2)
        l1, l2 = cf.sym2x2_eigs(G[0, 0].real, abs(G[0, 1]), G[1, 1].real)
        assert S[0] == pytest.approx(math.sqrt(l1), rel=1e-13)
        assert S[1] == pytest.approx(math.sqrt(l2), rel=1e-12)


def test_zsvd_of_real_input_matches_real_oracle():
    X = _rng(17).standard_normal((80, 9))
    Uz, Sz, Vz, _ = oracle.zsvd(X.astype(np.complex128))
    Ur, Sr, Vr, _ = oracle.svd(X)
    assert np.allclose(Sz, Sr, rtol=1e-13)
    # same phase rule: for real data the factors coincide
    assert np.allclose(Vz.real, Vr, atol=1e-12) and np.abs(Vz.imag).max() < 1e-12
    assert np.allclose(Uz.real, Ur, atol=1e-12) and np.abs(Uz.imag).max() < 1e-12


def test_zsvd_wave_bin_has_wave_rank():
    # a bin of 4 coherent waves plus 1e-3 noise: 4 singular values stand out
    X = synth.spod_bin(4096, 20, seed=5).astype(np.complex128)
    _, S, _, _ = oracle.zsvd(X)
    assert S[3] > 100 * S[4]
    _, S0, _, _ = oracle.zsvd(synth.spod_bin(4096, 20, seed=5, noise=0.0).astype(np.complex128))
    assert np.all(S0[4:] <= 1e-6 * S0[0])
