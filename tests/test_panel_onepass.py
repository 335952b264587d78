"""The algebra of the binary64 leaf kernel's one-pass panel factorisation
(Householder QR of a panel of a row block, Eq. svdqr1), checked in numpy on
the CPU.  The kernel makes one pass over the panel rows per column j: it
scales v_j, applies reflector j to the later columns, and on the rows below
j + 1 sums the products of the updated column j + 1 with every panel column
(d_c).  The next reflector's dot products with column c are then
scale_{j+1} d_c + A[j+1, c] (the reflector's unit entry meets row j + 1),
which serve its norm, its update and its column of the compact-WY factor T
(T[0:j, j] = -tau_j T[0:j, 0:j] V[:, 0:j]^T v_j).  Checked here: those dot
products equal the explicit v^T a at every step, T equals the forward
recurrence on the explicit V, (I - V T V^T)[R; 0] reproduces the panel, Q is
orthogonal, |diag R| equals LAPACK's, and a zero column gives tau = 0.
This pins the formulas, not the kernel (whose parity with the oracle the
GPU tests check)."""
import numpy as np
import pytest


def _one_pass_panel(P, check_dots=None):
    """Factor the h x nbk panel P in place by the one-pass scheme; returns
    (A with beta on the diagonal, v below it and updated columns, tau, T)."""
    A = np.array(P, dtype=np.float64)
    h, nbk = A.shape
    tau = np.zeros(nbk)
    T = np.zeros((nbk, nbk))
    d = A[1:, 0] @ A[1:, :]                          # column 0 against every column, rows below 0
    for j in range(nbk):
        alpha, xx = A[j, j], d[j]
        t, beta, scale = 0.0, alpha, 0.0
        if xx != 0.0:
            nrm = np.sqrt(alpha * alpha + xx)
            beta = -nrm if alpha >= 0.0 else nrm
            t = (beta - alpha) / beta
            scale = 1.0 / (alpha - beta)
        sdot = scale * d + A[j, :]                   # v_j^T a_c through the sums of the previous pass
        sdot[j] = 0.0
        if check_dots is not None:
            check_dots(A, j, scale, sdot)
        tau[j] = t
        for p in range(j):
            T[p, j] = -t * (T[p, p:j] @ sdot[p:j])
        T[j, j] = t
        # the pass over rows j..h-1
        v = np.empty(h - j)
        v[0] = 1.0
        v[1:] = A[j + 1:, j] * scale
        A[j, j] = beta
        A[j + 1:, j] = v[1:]
        if j + 1 < nbk:
            A[j:, j + 1:] -= np.outer(v, t * sdot[j + 1:])
            # sums for column j + 1 over the rows below j + 1: every column,
            # column j read as its reflector
            d = A[j + 2:, j + 1] @ A[j + 2:, :]
    return A, tau, T


def _unpack(A):
    h, nbk = A.shape
    V = np.tril(A, -1)
    V[:nbk] += np.eye(nbk)
    R = np.triu(A[:nbk])
    return V, R


def _panel(h, nbk, seed, graded=True):
    rng = np.random.default_rng(seed)
    P = rng.standard_normal((h, nbk))
    if graded:
        P *= np.logspace(0, -6, nbk)[None, :]
    return P


@pytest.mark.parametrize("h,nbk,seed", [(300, 16, 0), (17, 16, 1), (1000, 7, 2), (16, 16, 3), (40, 1, 4)])
def test_one_pass_panel_is_a_householder_qr(h, nbk, seed):
    P = _panel(h, nbk, seed)

    def check_dots(A, j, scale, sdot):
        # explicit reflector j (before it is written) against every column:
        # rows j.. of an earlier column hold that reflector's entries (v_j is
        # zero above row j), rows j.. of a later column its current values
        v = np.concatenate([[1.0], A[j + 1:, j] * scale])
        for c in range(A.shape[1]):
            if c != j:
                np.testing.assert_allclose(sdot[c], v @ A[j:, c], rtol=1e-12, atol=1e-12 * np.abs(P).max())

    A, tau, T = _one_pass_panel(P, check_dots)
    V, R = _unpack(A)
    Q = np.eye(h) - V @ T @ V.T
    scale = np.linalg.norm(P)
    np.testing.assert_allclose(Q[:, :nbk] @ R, P, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(Q.T @ Q, np.eye(h), rtol=0, atol=1e-13)
    R_ref = np.linalg.qr(P, mode="r")
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(R_ref)), rtol=1e-12)
    # T is the forward recurrence on the explicit reflectors
    T_ref = np.zeros_like(T)
    for j in range(nbk):
        T_ref[:j, j] = -tau[j] * (T_ref[:j, :j] @ (V[:, :j].T @ V[:, j]))
        T_ref[j, j] = tau[j]
    np.testing.assert_allclose(T, T_ref, rtol=1e-12, atol=1e-14)
    assert np.all(np.triu(T) == T)


def test_zero_column_gives_identity_reflector():
    P = _panel(50, 6, 5, graded=False)
    P[:, 2] = 0.0                                     # stays zero under reflectors 0 and 1: x = 0 at step 2
    A, tau, T = _one_pass_panel(P)
    assert tau[2] == 0.0 and T[2, 2] == 0.0
    V, R = _unpack(A)
    assert np.all(V[3:, 2] == 0.0)
    Q = np.eye(50) - V @ T @ V.T
    np.testing.assert_allclose(Q[:, :6] @ R, P, rtol=0, atol=1e-13 * np.linalg.norm(P))


def test_panel_inside_a_leaf_matches_the_blocked_factorisation():
    """Two panels of a 200 x 12 block: the second is factored after the
    first panel's block reflector is applied to it (what the leaf kernel
    does between panels); R equals the unblocked QR's up to row signs."""
    P = _panel(200, 12, 6)
    A1, tau1, T1 = _one_pass_panel(P[:, :6])
    V1, R1 = _unpack(A1)
    C = P[:, 6:] - V1 @ (T1.T @ (V1.T @ P[:, 6:]))   # Q1^T applied to the trailing columns
    A2, tau2, T2 = _one_pass_panel(C[6:])
    V2, R2 = _unpack(A2)
    R = np.zeros((12, 12))
    R[:6, :6] = R1
    R[:6, 6:] = C[:6]
    R[6:, 6:] = R2
    R_ref = np.linalg.qr(P, mode="r")
    sgn = np.sign(np.diag(R)) * np.sign(np.diag(R_ref))
    np.testing.assert_allclose(R, sgn[:, None] * R_ref, rtol=0, atol=1e-12 * np.abs(R_ref).max())
