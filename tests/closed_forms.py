"""Closed forms the tests pin the oracle (and the CUDA path) against.

Each is derived from the mathematics of the synthetic inputs, not from any
implementation of the method.
"""
from __future__ import annotations

import math

import numpy as np

from synth import wave_params


def waves_sigma(N: int, M: int, n_waves: int, amp: str = "geometric") -> np.ndarray:
    """Noise-free singular values of the mean-removed traveling-wave field.

    With x_n = 2 pi n / N, t_m = m dt and w_j = 2 pi q_j / (M dt), the sampled
    sin(k x), cos(k x) (distinct integers 0 < k < N/2) are mutually orthogonal
    with squared norm N/2, and likewise cos(w t), sin(w t) over the M
    snapshots with squared norm M/2.  a sin(kx - wt) = a [sin kx cos wt -
    cos kx sin wt] is then an orthogonal rank-2 term with both singular values
    a sqrt(N/2) sqrt(M/2) = a sqrt(N M) / 2, and the time-constant mean field
    is removed exactly by the temporal mean."""
    a, k, q = wave_params(n_waves, amp)
    if np.any(k >= N // 2) or np.any(q >= M // 2):
        raise ValueError("wave numbers must stay below N/2 and M/2 for the closed form")
    s = np.repeat(a * math.sqrt(N * M) / 2.0, 2)
    return np.sort(s)[::-1]


def truncation_rank(M: int, decades: float, energy: float) -> int:
    """r for s_i = 10^(-decades i / (M-1)): s_i^2 = q^i with
    q = 10^(-2 decades / (M-1)), so the cumulative energy of the first r values
    is (1 - q^r) / (1 - q^M) (geometric series); r is the first that reaches
    ``energy``."""
    q = 10.0 ** (-2.0 * decades / (M - 1))
    for r in range(1, M + 1):
        if (1.0 - q ** r) / (1.0 - q ** M) >= energy:
            return r
    return M


def truncation_rank_of(s, energy: float) -> int:
    """First r whose leading singular values s[:r] hold >= `energy` of
    sum(s^2) (the cumulative-energy rule of Sec. 3.1, in plain FP64)."""
    e = np.cumsum(np.asarray(s, dtype=np.float64) ** 2)
    return int(np.argmax(e >= energy * e[-1])) + 1


def sym2x2_eigs(a: float, b: float, c: float):
    """Eigenvalues of [[a, b], [b, c]] (quadratic formula)."""
    mid = 0.5 * (a + c)
    rad = math.hypot(0.5 * (a - c), b)
    return mid + rad, mid - rad
