"""Seeded synthetic snapshot matrices shared by the tests, the smoke check and
the benchmark.

This module holds input construction only: none of the POD method's
arithmetic (no mean removal, no QR of the snapshot matrix, no SVD) lives
here.  Library primitives (numpy/torch GEMM, and a library QR used only to
draw random orthonormal factors) build the inputs.  The CUDA library and the
oracle both consume what it returns; neither is imported here.

Workloads (N gridpoints x M snapshots, column-major / Fortran order):

* ``waves``: a wake-like field of traveling waves
  ``f0(x) + sum_j a_j sin(k_j x - w_j t) + noise`` on ``x_n = 2 pi n / N``,
  ``t_m = m dt`` with ``w_j = 2 pi q_j / (M dt)``, so that with distinct
  integer ``k_j < N/2`` and ``q_j < M/2`` the sampled sines and cosines are
  orthogonal and, noise-free, each wave contributes the singular value
  ``a_j sqrt(N M) / 2`` twice (a closed form the tests use).
* ``known_spectrum``: ``X = diag(w)^(-1/2) Q1 diag(s) Q2^T`` with seeded
  random orthonormal ``Q1`` (N x M) and Haar ``Q2`` (M x M), so the weighted
  snapshot matrix ``diag(sqrt w) X`` has singular values ``s`` exactly (up
  to construction rounding).
"""
from __future__ import annotations

import math

import numpy as np

# ----------------------------------------------------------------------------
# wave parameters of the two wave workloads
# ----------------------------------------------------------------------------

def wave_params(n_waves: int, amp: str = "geometric"):
    """(a_j, k_j, q_j) for the wave workloads.

    geometric: a_j = 2^-j (16384 x 64 workload, 8 waves)
    powerlaw:  a_j = (1 + j)^(-5/6) (10^7 x 1808 workload, 64 waves)
    """
    j = np.arange(n_waves, dtype=np.float64)
    if amp == "geometric":
        a = 2.0 ** (-j)
        k = 1 + 2 * np.arange(n_waves)
        q = 1 + 3 * np.arange(n_waves)
    elif amp == "powerlaw":
        a = (1.0 + j) ** (-5.0 / 6.0)
        k = 1 + 2 * np.arange(n_waves)
        q = 1 + 7 * np.arange(n_waves)
    else:
        raise ValueError(amp)
    return a, k.astype(np.int64), q.astype(np.int64)


def waves(N: int, M: int, n_waves: int = 8, amp: str = "geometric", noise: float = 1e-3,
          seed: int = 1, dt: float = 0.2, dtype=np.float64) -> np.ndarray:
    """Traveling-wave snapshot matrix (numpy, Fortran order)."""
    a, k, q = wave_params(n_waves, amp)
    x = 2.0 * np.pi * np.arange(N, dtype=np.float64) / N
    t = dt * np.arange(M, dtype=np.float64)
    omega = 2.0 * np.pi * q / (M * dt)
    # sin(kx - wt) = sin(kx) cos(wt) - cos(kx) sin(wt): a rank-2J product
    Fx = np.concatenate([np.sin(np.outer(x, k)), -np.cos(np.outer(x, k))], axis=1)  # N x 2J
    Gt = np.concatenate([np.cos(np.outer(omega, t)), np.sin(np.outer(omega, t))], axis=0)  # 2J x M
    Gt = Gt * np.concatenate([a, a])[:, None]
    X = Fx @ Gt
    X += (1.0 + 0.5 * np.cos(x))[:, None]
    if noise > 0.0:
        rng = np.random.default_rng(seed)
        X += noise * rng.standard_normal((N, M))
    return np.asfortranarray(X.astype(dtype))


def waves_torch(N: int, M: int, n_waves: int, amp: str, noise: float, seed: int, device,
                dtype=None, dt: float = 0.2, row_chunk: int = 1 << 22):
    """Device-side version of :func:`waves` for large N (column-major result:
    a torch tensor of shape (M, N) whose transpose view is the N x M matrix)."""
    import torch
    dtype = dtype or torch.float64
    a, k, q = wave_params(n_waves, amp)
    omega = 2.0 * np.pi * q / (M * dt)
    t = dt * np.arange(M, dtype=np.float64)
    Gt = np.concatenate([np.cos(np.outer(omega, t)), np.sin(np.outer(omega, t))], axis=0)
    Gt = torch.tensor(Gt * np.concatenate([a, a])[:, None], dtype=torch.float64, device=device)
    kk = torch.tensor(k, dtype=torch.float64, device=device)
    XT = torch.empty((M, N), dtype=dtype, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    for r0 in range(0, N, row_chunk):
        r1 = min(N, r0 + row_chunk)
        x = 2.0 * math.pi * torch.arange(r0, r1, dtype=torch.float64, device=device) / N
        kx = torch.outer(x, kk)
        Fx = torch.cat([torch.sin(kx), -torch.cos(kx)], dim=1)
        blk = Fx @ Gt + (1.0 + 0.5 * torch.cos(x))[:, None]
        if noise > 0.0:
            blk += noise * torch.randn(blk.shape, dtype=torch.float64, device=device, generator=gen)
        XT[:, r0:r1] = blk.T.to(dtype)
    return XT


# ----------------------------------------------------------------------------
# known-spectrum workload
# ----------------------------------------------------------------------------

def spectrum(M: int, decades: float = 6.0) -> np.ndarray:
    """s_i = 10^(-decades * i / (M - 1)), i = 0..M-1."""
    i = np.arange(M, dtype=np.float64)
    return 10.0 ** (-decades * i / max(M - 1, 1))


def log_uniform_weights(N: int, seed: int, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return 10.0 ** rng.uniform(math.log10(lo), math.log10(hi), size=N)


def haar_orthogonal(M: int, seed: int) -> np.ndarray:
    """Haar-distributed M x M orthogonal matrix (library QR of a Gaussian with
    the signs of R's diagonal moved into Q)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((M, M))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def orthonormal_columns(N: int, M: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, M))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def known_spectrum(N: int, M: int, s=None, weights: bool = True, seeds=(2, 3, 4),
                   dtype=np.float64):
    """X = diag(w)^(-1/2) Q1 diag(s) Q2^T; returns (X, w or None, s)."""
    if s is None:
        s = spectrum(M)
    Q1 = orthonormal_columns(N, M, seeds[0])
    Q2 = haar_orthogonal(M, seeds[1])
    Y = (Q1 * s[None, :]) @ Q2.T
    w = log_uniform_weights(N, seeds[2]) if weights else None
    X = Y / np.sqrt(w)[:, None] if weights else Y
    return np.asfortranarray(X.astype(dtype)), w, np.asarray(s, dtype=np.float64)


def known_spectrum_torch(N: int, M: int, device, s=None, weights: bool = True, seeds=(2, 3, 4),
                         dtype=None):
    """Device-side :func:`known_spectrum` for large N.  Returns (XT, w, s) with
    XT of shape (M, N) (so XT.T is the column-major N x M matrix).  Q1 is a
    different seeded orthonormal factor than the host version's (same
    distribution up to the orthonormalisation route)."""
    import torch
    dtype = dtype or torch.float64
    if s is None:
        s = spectrum(M)
    gen = torch.Generator(device=device)
    gen.manual_seed(seeds[0])
    Q1 = torch.randn((N, M), dtype=torch.float64, device=device, generator=gen)
    # orthonormalise the Gaussian by two Cholesky-QR passes: Gram matrix on
    # the device, its M x M Cholesky factor inverted on the host (no device
    # linear-algebra library needed), one product per pass
    for _ in range(2):
        gram = (Q1.T @ Q1).cpu()
        L = torch.linalg.cholesky(gram)
        Linv_t = torch.linalg.inv(L).T.contiguous().to(device)
        Q1 = Q1 @ Linv_t
    Q2 = torch.tensor(haar_orthogonal(M, seeds[1]), dtype=torch.float64, device=device)
    st = torch.tensor(s, dtype=torch.float64, device=device)
    Y = (Q1 * st[None, :]) @ Q2.T
    del Q1
    if weights:
        w = torch.tensor(log_uniform_weights(N, seeds[2]), dtype=torch.float64, device=device)
        Y /= torch.sqrt(w)[:, None]
    else:
        w = None
    XT = Y.T.contiguous().to(dtype)
    del Y
    return XT, w, np.asarray(s, dtype=np.float64)


# ----------------------------------------------------------------------------
# complex per-frequency matrices (SPOD bins)
# ----------------------------------------------------------------------------

def unitary_columns(N: int, M: int, seed: int) -> np.ndarray:
    """Seeded N x M matrix with orthonormal complex columns (library QR of a
    complex Gaussian, phases of R's diagonal moved into Q)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((N, M)) + 1j * rng.standard_normal((N, M))
    Q, R = np.linalg.qr(G)
    d = np.diag(R)
    return Q * (d / np.abs(d))[None, :]


def complex_known_spectrum(N: int, M: int, s=None, seeds=(81, 82), dtype=np.complex128):
    """X = Q1 diag(s) Q2^H with seeded orthonormal complex Q1 (N x M) and
    unitary Q2 (M x M): singular values s exactly."""
    if s is None:
        s = spectrum(M)
    Q1 = unitary_columns(N, M, seeds[0])
    Q2 = unitary_columns(M, M, seeds[1])
    X = (Q1 * np.asarray(s)[None, :]) @ Q2.conj().T
    return np.asfortranarray(X.astype(dtype)), np.asarray(s, dtype=np.float64)


def spod_bin_sizes(n_bins: int, seed: int, n_lo: int = 1 << 16, n_hi: int = 1 << 20,
                   nb_lo: int = 16, nb_hi: int = 128):
    """Per-bin sizes of the batched SPOD workload: N_f log-uniform in
    [n_lo, n_hi], Nb_f uniform integers in [nb_lo, nb_hi]."""
    rng = np.random.default_rng(seed)
    N = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=n_bins))).astype(np.int64)
    Nb = rng.integers(nb_lo, nb_hi + 1, size=n_bins).astype(np.int64)
    return N, Nb


def window_sizes(n_windows: int, seed: int, n_lo: int = 1 << 16, n_hi: int = 1 << 20,
                 m_lo: int = 16, m_hi: int = 128):
    """Sizes of a batch of real snapshot windows: N_i log-uniform in
    [n_lo, n_hi], M_i uniform integers in [m_lo, m_hi]."""
    return spod_bin_sizes(n_windows, seed, n_lo, n_hi, m_lo, m_hi)


def spod_bin(N: int, Nb: int, seed: int, n_waves: int = 4, noise: float = 1e-3, dtype=np.complex64):
    """One frequency bin's matrix of block Fourier coefficients of a
    traveling-wave field (numpy, Fortran order): a traveling wave
    a sin(k x - w t) seen through windowed blocks contributes, at its own
    frequency, a spatial complex exponential exp(i k x) whose coefficient in
    block b carries the phase of that block's start time, so the bin is
    sum_j a_j exp(i k_j x) exp(i phi_jb) + complex noise, scaled by
    1/sqrt(Nb) like the SPOD matrix.  Phases and noise are seeded."""
    rng = np.random.default_rng(seed)
    x = 2.0 * np.pi * np.arange(N, dtype=np.float64) / N
    k = 1 + rng.permutation(min(N // 2 - 1, 4096))[:n_waves]
    a = 2.0 ** (-np.arange(n_waves, dtype=np.float64))
    Fx = np.exp(1j * np.outer(x, k))                       # N x J
    Ph = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=(n_waves, Nb))) * a[:, None]
    X = Fx @ Ph
    X += noise * (rng.standard_normal((N, Nb)) + 1j * rng.standard_normal((N, Nb))) / math.sqrt(2.0)
    X /= math.sqrt(Nb)
    return np.asfortranarray(X.astype(dtype))


def spod_bin_torch(N: int, Nb: int, seed: int, device, n_waves: int = 4, noise: float = 1e-3):
    """Device-side :func:`spod_bin` (complex64); returns XT of shape (Nb, N)
    so that XT.T is the column-major N x Nb matrix."""
    import torch
    rng = np.random.default_rng(seed)
    k = 1 + rng.permutation(min(N // 2 - 1, 4096))[:n_waves]
    a = 2.0 ** (-np.arange(n_waves, dtype=np.float64))
    Ph = np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=(n_waves, Nb))) * a[:, None]
    x = 2.0 * math.pi * torch.arange(N, dtype=torch.float64, device=device) / N
    kk = torch.tensor(k, dtype=torch.float64, device=device)
    Fx = torch.exp(1j * torch.outer(x, kk))
    X = Fx @ torch.tensor(Ph, dtype=torch.complex128, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    X += noise * torch.complex(torch.randn((N, Nb), dtype=torch.float64, device=device, generator=gen),
                               torch.randn((N, Nb), dtype=torch.float64, device=device, generator=gen)) / math.sqrt(2.0)
    X /= math.sqrt(Nb)
    return X.T.contiguous().to(torch.complex64)


# ----------------------------------------------------------------------------
# oscillation workload (DMD)
# ----------------------------------------------------------------------------

def oscillation_params(K: int, seed: int = 0, rho_lo: float = 0.985, rho_hi: float = 1.0):
    """K eigenvalues lambda_k = rho_k exp(i theta_k) with theta_k spread over
    (0.05, 3.0) and rho_k in [rho_lo, rho_hi], and amplitudes a_k with
    distinct moduli 1 + k / K (phases random)."""
    rng = np.random.default_rng(seed)
    theta = np.linspace(0.05, 3.0, K)
    rho = rho_lo + (rho_hi - rho_lo) * rng.random(K)
    lam = rho * np.exp(1j * theta)
    amp = (1.0 + np.arange(K) / K) * np.exp(2j * np.pi * rng.random(K))
    return lam, amp


def oscillations(N: int, M: int, lams, amps, seed: int = 0, noise: float = 0.0, offset: float = 0.0):
    """D[:, t] = offset + sum_k Re(a_k psi_k lambda_k^t) + noise (numpy,
    Fortran order), psi_k with independent standard normal real and
    imaginary parts.  Noise-free, D has rank 2K and its DMD is known in
    closed form: eigenvalues lambda_k and conj(lambda_k), and each mode
    times its amplitude equals a_k psi_k / 2 (or its conjugate).  Returns
    (D, parts) with parts[k] = a_k psi_k / 2."""
    rng = np.random.default_rng(seed)
    t = np.arange(M)
    D = np.full((N, M), float(offset), dtype=np.float64, order="F")
    parts = []
    for lam, a in zip(lams, amps):
        psi = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        D += np.real(a * psi[:, None] * np.asarray(lam) ** t[None, :])
        parts.append(a * psi / 2.0)
    if noise > 0.0:
        D += noise * rng.standard_normal((N, M))
    return np.asfortranarray(D), parts


def oscillations_torch(N: int, M: int, lams, amps, seed: int, device, noise: float = 0.0, dtype=None,
                       row_chunk: int = 1 << 21):
    """Device-side :func:`oscillations` for large N: XT of shape (M, N)
    (transpose view = the N x M matrix), built as Re(Psi C) with C[k, t] =
    a_k lambda_k^t by library GEMMs.  Returns (XT, Psi_fn) where Psi_fn(rows)
    regenerates psi for a row range (seeded per chunk) for closed-form checks."""
    import torch
    dtype = dtype or torch.float64
    K = len(lams)
    t = np.arange(M)
    C = np.asarray(amps)[:, None] * np.asarray(lams)[:, None] ** t[None, :]
    Cr = torch.tensor(C.real, dtype=torch.float64, device=device)
    Ci = torch.tensor(C.imag, dtype=torch.float64, device=device)
    XT = torch.empty((M, N), dtype=dtype, device=device)

    def psi_chunk(r0, r1):
        gen = torch.Generator(device=device)
        gen.manual_seed(seed * 1000003 + r0)
        pr = torch.randn((r1 - r0, K), dtype=torch.float64, device=device, generator=gen)
        pi = torch.randn((r1 - r0, K), dtype=torch.float64, device=device, generator=gen)
        nz = torch.randn((r1 - r0, M), dtype=torch.float64, device=device, generator=gen) if noise > 0 else None
        return pr, pi, nz

    for r0 in range(0, N, row_chunk):
        r1 = min(N, r0 + row_chunk)
        pr, pi, nz = psi_chunk(r0, r1)
        blk = pr @ Cr - pi @ Ci
        if nz is not None:
            blk += noise * nz
        XT[:, r0:r1] = blk.T.to(dtype)
    return XT, psi_chunk
