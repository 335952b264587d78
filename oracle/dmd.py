"""FP64 CPU oracle of the exact DMD with optimal amplitudes (pyLOM, arXiv
2405.15529, Sec. 3.2 and Algs. 3-5).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA library.  Plain numpy in binary64; the SVD
of Y1 is the C oracle's POD (Alg. 2 without mean removal: Householder QR and
one-sided Jacobi), the eigendecomposition of the small operator is a library
step (``numpy.linalg.eig``, LAPACK's dgeev as in Alg. 3), the Cholesky
factor and the triangular solves are library steps (``numpy.linalg``).

Steps, in the order of Alg. 3 (data D: N points x M snapshots):
  optional removal of each point's mean over all M snapshots;
  Y1 = Y[:, :M-1], Y2 = Y[:, 1:];
  Y1 = U S V^T (tsqr_svd), truncated to r (cumulative energy, r_max, and
  the numerical rank, reading below);
  aux = U^T Y2 (Alg. 4's product), A = aux (S^-1 V^T)^T  (r x r);
  A w = w diag(mu)  (eigendecomposition, eigenvectors normalised, below);
  phi = Y2 V S^-1 w diag(mu)^-1  (the exact DMD modes);
  amplitudes b (Alg. 5): V_and[i, t] = mu_i^t (t = 0 .. M-2),
  P = (w^H w) o conj(V_and V_and^H), q = conj(diag(V_and (S V^T)^T w)),
  P = L L^H (Cholesky), b = L^-H L^-1 q;
  modes, eigenvalues and amplitudes ordered by |b| (largest first).
Readings (where Alg. 5 and the sort are terse or at odds with the stated
objective):
  * the amplitudes minimise || S V^T - w diag(b) V_and ||_F, which is the
    paper's || Y1 - phi D_b V_and ||_F for the projected modes U w (the
    inputs of Alg. 5 are mu, w, S and V only); its normal equations carry
    conj(V_and V_and^H) in P, which Alg. 5's formula leaves out, and the
    product "V_and G w" needs G transposed to conform;
  * the Cholesky factor is lower (P = L L^H), b = L^-H (L^-1 q);
  * the sort: a conjugate pair shares the larger |b| of its two members,
    stays adjacent, and the member with positive imaginary part comes first
    (the paper reorders conjugate pairs by the sign of the imaginary part);
  * S^-1 needs s_k > 0: r is cut to the numerical rank of Y1 by the usual
    rule for an N x (M-1) matrix, the count of s_k > max(N, M-1) 2^-52 s_1;
  * eigenvectors: unit Euclidean norm, and the entry of largest modulus
    (the first such entry) made real and positive.
"""
from __future__ import annotations

import numpy as np

import oracle

EPS = 2.0 ** -52


def numerical_rank(S, dim: int) -> int:
    """Count of singular values above dim * 2^-52 * s_1 (S sorted descending)."""
    S = np.asarray(S, dtype=np.float64)
    if S.size == 0 or S[0] <= 0.0:
        return 0
    return int(np.sum(S > dim * EPS * S[0]))


def normalize_eigvecs(W):
    """Unit 2-norm columns with the (first) entry of largest modulus real and positive."""
    W = np.asarray(W, dtype=np.complex128)
    W = W / np.linalg.norm(W, axis=0)[None, :]
    k = np.argmax(np.abs(W), axis=0)
    ph = W[k, np.arange(W.shape[1])]
    return W * (np.conj(ph) / np.abs(ph))[None, :]


def vandermonde(mu, ncols: int):
    """V_and[i, t] = mu_i^t for t = 0 .. ncols-1 (running products)."""
    mu = np.asarray(mu, dtype=np.complex128)
    V = np.empty((mu.shape[0], ncols), dtype=np.complex128)
    if ncols > 0:
        V[:, 0] = 1.0
    for t in range(1, ncols):
        V[:, t] = V[:, t - 1] * mu
    return V


def amplitudes(mu, W, S, VT):
    """Alg. 5: optimal amplitudes of the modes U w (normal equations of the
    least-squares fit of S V^T by w diag(b) V_and, solved by Cholesky)."""
    m1 = VT.shape[1]
    Vand = vandermonde(mu, m1)
    P = (W.conj().T @ W) * np.conj(Vand @ Vand.conj().T)
    G = S[:, None] * VT                      # S V^T, r x (M-1)
    q = np.conj(np.diag(Vand @ G.T @ W))
    L = np.linalg.cholesky(P)                # P = L L^H
    return np.linalg.solve(L.conj().T, np.linalg.solve(L, q))


def shifted_pair(Y):
    """Y1 = snapshots 0 .. M-2, Y2 = snapshots 1 .. M-1 (Eqs. y1, y2)."""
    return Y[:, :-1], Y[:, 1:]


def exact_modes(Y2, VT, S, W, mu):
    """phi = Y2 V S^-1 w diag(mu)^-1 (Alg. 3's mode formula)."""
    return (Y2 @ (VT.T / S[None, :]) @ W) / mu[None, :]


def order(mu, b):
    """Indices by descending |b|; a conjugate pair shares the larger |b| of its
    members, stays adjacent, positive imaginary part first."""
    mu = np.asarray(mu)
    r = mu.shape[0]
    key = np.abs(b).astype(np.float64)
    group = np.arange(r)
    for i in range(r):
        if mu[i].imag != 0.0:
            for j in range(r):
                if j != i and mu[j] == np.conj(mu[i]):
                    key[i] = key[j] = max(abs(b[i]), abs(b[j]))
                    group[i] = group[j] = min(i, j)
    return np.array(sorted(range(r), key=lambda i: (-key[i], group[i], -np.sign(mu[i].imag))))


def dmd(D, energy: float = 0.0, r_max=None, remove_mean: bool = True):
    """Exact DMD of the N x M snapshot matrix D (Alg. 3).  Returns dict with
    mu (r), b (r), Phi (N x r complex), S (M-1 singular values of Y1), r,
    A (r x r), W (r x r, unsorted eigenvectors), mean (N)."""
    D = np.asarray(D, dtype=np.float64)
    N, M = D.shape
    if M < 2:
        raise ValueError("DMD needs at least two snapshots")
    m1 = M - 1
    mean = D.mean(axis=1) if remove_mean else np.zeros(N)
    Y1, Y2 = shifted_pair(D - mean[:, None])
    if r_max is None:
        r_max = m1
    pod = oracle.pod(np.asfortranarray(Y1), remove_mean=False, energy=energy, r_max=r_max)
    S_all = pod["S"]
    r = min(pod["r"], numerical_rank(S_all, max(N, m1)))
    U, S, VT = pod["U"][:, :r], S_all[:r], pod["VT"][:r, :]
    if r == 0:
        z = np.zeros(0, dtype=np.complex128)
        return dict(mu=z, b=z, Phi=np.zeros((N, 0), dtype=np.complex128), S=S_all, r=0,
                    A=np.zeros((0, 0)), W=np.zeros((0, 0), dtype=np.complex128), mean=mean)
    aux = oracle.matmul(U, Y2, transA=True)              # U^T Y2 (Alg. 4)
    A = aux @ (VT / S[:, None]).T                        # aux (S^-1 V^T)^T
    mu, W = np.linalg.eig(A)
    W = normalize_eigvecs(W)
    Phi = exact_modes(Y2, VT, S, W, mu)
    b = amplitudes(mu, W, S, VT)
    idx = order(mu, b)
    return dict(mu=mu[idx], b=b[idx], Phi=Phi[:, idx], S=S_all, r=r, A=A, W=W, mean=mean)
