"""The algebra the mixed-precision leaf kernel uses to factor a panel
(chunked TSQR, then Householder reconstruction after Ballard et al., 2015),
checked in binary64 numpy on the CPU: from an explicit Q with orthonormal
columns, the LU factorisation without pivoting of Q - [S; 0] with signs
s_j = -sign(pivot) gives V (unit lower trapezoidal), T = -U S V1^-T (upper
triangular, diagonal in [1, 2]) and R = S R_tsqr with (I - V T V^T)[R; 0]
equal to the panel.  This pins the formulas, not the kernel (whose parity
with the oracle the GPU tests check)."""
import numpy as np
import pytest


def _reconstruct(Q):
    m, n = Q.shape
    W = Q.copy()
    s = np.zeros(n)
    for j in range(n):
        s[j] = -1.0 if W[j, j] >= 0 else 1.0
        W[j, j] -= s[j]
        W[j + 1:, j] /= W[j, j]
        W[j + 1:, j + 1:] -= np.outer(W[j + 1:, j], W[j, j + 1:])
    U = np.triu(W[:n])
    V = np.tril(W, -1)
    V[:n] += np.eye(n)
    T = -(U * s[None, :]) @ np.linalg.inv(V[:n]).T
    return V, T, s


def _chunked_q_r(A, rows=16):
    """Explicit Q and R of A by a two-level TSQR (chunk QRs, one QR of the
    stacked chunk R factors), as the kernel's tree computes them."""
    m, n = A.shape
    qs, rs = [], []
    for c in range(0, m, rows):
        q, r = np.linalg.qr(A[c:c + rows], mode="reduced") if A[c:c + rows].shape[0] >= n else (None, None)
        if q is None:   # a short last chunk: pad with zero rows
            blk = np.zeros((n, n))
            blk[:A[c:].shape[0]] = A[c:]
            q, r = np.linalg.qr(blk)
            q = q[:A[c:].shape[0]]
        qs.append(q)
        rs.append(r)
    q2, R = np.linalg.qr(np.vstack(rs))
    Q = np.vstack([qs[i] @ q2[i * n:(i + 1) * n] for i in range(len(qs))])
    return Q, R


@pytest.mark.parametrize("m,n,cond", [(200, 8, 1e2), (333, 12, 1e6), (64, 16, 10.0)])
def test_reconstructed_compact_wy_reproduces_the_panel(m, n, cond):
    rng = np.random.default_rng(m + n)
    U0, _ = np.linalg.qr(rng.standard_normal((m, n)))
    V0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (U0 * np.logspace(0, -np.log10(cond), n)) @ V0.T
    Q, R = _chunked_q_r(A)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)
    V, T, s = _reconstruct(Q)
    assert np.max(np.abs(np.tril(T, -1))) == 0.0                         # upper triangular
    assert np.all(T.diagonal() >= 1.0 - 1e-14) and np.all(T.diagonal() <= 2.0 + 1e-14)
    H = np.eye(m) - V @ T @ V.T
    np.testing.assert_allclose(H.T @ H, np.eye(m), atol=1e-12)           # orthogonal
    np.testing.assert_allclose(H[:, :n] @ (s[:, None] * R), A, atol=1e-12 * np.abs(A).max())
    # the first n columns of H are Q S
    np.testing.assert_allclose(H[:, :n], Q * s[None, :], atol=1e-12)


def test_reconstruction_matches_householder_qr_up_to_signs():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((120, 10))
    Q, R = _chunked_q_r(A)
    V, T, s = _reconstruct(Q)
    R_ref = np.linalg.qr(A, mode="r")
    # R = S R_tsqr agrees with any Householder R up to row signs
    np.testing.assert_allclose(np.abs(s[:, None] * R), np.abs(R_ref), atol=1e-12)
