"""FP64 CPU oracle of the SPOD front end and of the whole SPOD (pyLOM, arXiv
2405.15529, Sec. 2.3 and Alg. 6).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.
It shares no code with the CUDA library.  Plain numpy in binary64; the
per-block Fourier transform is a library step (``numpy.fft.rfft``), the
per-frequency SVDs are the C oracle's complex one-sided Jacobi.

Steps, in the order of Alg. 6 (data D: N points x T snapshots):
  nBlks = floor((T - nolap) / (npwin - nolap));
  window_j = 0.54 - 0.46 cos(2 pi j / (npwin - 1)), j = 0 .. npwin - 1 (Hamming);
  optional removal of each point's temporal mean;
  block b starts at snapshot i0 = b (npwin - nolap); every point's npwin
  samples are multiplied by the window, transformed, and divided by
  mean(window) npwin; the one-sided spectrum keeps frequencies
  k = 0 .. ceil(npwin / 2) (for even npwin: 0 .. npwin / 2) and doubles all
  but its first and last entries;
  Q_f (N x nBlks) gathers frequency k of every block, scaled by 1/sqrt(nBlks);
  per frequency (1/sqrt(nBlks)) Q_f = U_f S_f V_f^H; energies L_f = S_f^2;
  frequencies f_k = k / (dt npwin); bins ordered by their leading energy.
Readings (where Alg. 6 is garbled): [0:1:npwin] is read as j = 0 .. npwin-1;
the frequency axis "(ceil(npwin/2)+1)/(dt npwin)" is read as the count
ceil(npwin/2) + 1 of one-sided frequencies k / (dt npwin); the modes are
returned complex (real(U) is post-processing).
"""
from __future__ import annotations

import math

import numpy as np


def spod_shape(T: int, npwin: int, nolap: int):
    """(nBlks, nfreq) for T snapshots, blocks of npwin overlapping by nolap."""
    if not (npwin >= 2 and 0 <= nolap < npwin and T >= npwin):
        raise ValueError("need npwin >= 2, 0 <= nolap < npwin, T >= npwin")
    nblks = (T - nolap) // (npwin - nolap)
    nfreq = npwin // 2 + 1
    return nblks, nfreq


def hamming(npwin: int) -> np.ndarray:
    j = np.arange(npwin, dtype=np.float64)
    return 0.54 - 0.46 * np.cos(2.0 * np.pi * j / (npwin - 1))


def spod_blocks(D, npwin: int, nolap: int, remove_mean: bool = True) -> np.ndarray:
    """Q (nfreq, N, nBlks) complex128: Q[k] = Q_f of frequency k / sqrt(nBlks)."""
    D = np.asarray(D, dtype=np.float64)
    N, T = D.shape
    nblks, nfreq = spod_shape(T, npwin, nolap)
    Y = D - D.mean(axis=1, keepdims=True) if remove_mean else D
    win = hamming(npwin)
    norm = win.mean() * npwin
    Q = np.empty((nfreq, N, nblks), dtype=np.complex128)
    for b in range(nblks):
        i0 = b * (npwin - nolap)
        q = np.fft.rfft(Y[:, i0:i0 + npwin] * win[None, :], axis=1) / norm   # N x nfreq
        q[:, 1:-1] *= 2.0
        Q[:, :, b] = q.T
    return Q / math.sqrt(nblks)


def spod(D, dt: float, npwin: int, nolap: int, remove_mean: bool = True, kmodes: int = 8):
    """Whole SPOD: per frequency (in bin order 0..nfreq-1) the singular values
    S (nBlks), the energies L = S^2, the first kmodes left vectors (complex,
    phase rule of the complex SVD), the frequency axis, and the order of the
    bins by their leading energy (largest first; ties by index)."""
    from oracle import zsvd
    Q = spod_blocks(D, npwin, nolap, remove_mean)
    nfreq = Q.shape[0]
    S, U = [], []
    for k in range(nfreq):
        Uk, Sk, _, _ = zsvd(np.asfortranarray(Q[k]), k=min(kmodes, Q.shape[2]))
        S.append(Sk)
        U.append(Uk)
    S = np.array(S)
    L = S ** 2
    f = np.arange(nfreq, dtype=np.float64) / (dt * npwin)
    order = sorted(range(nfreq), key=lambda k: (-L[k, 0], k))
    return {"Q": Q, "S": S, "L": L, "U": U, "f": f, "order": np.array(order)}
