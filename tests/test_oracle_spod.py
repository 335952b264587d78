"""Pins of the SPOD front-end oracle (Sec. 2.3, Alg. 6) against facts fixed
by the paper and by the mathematics: the transform of an impulse (block
placement, window index, sign convention, scaling and one-sided doubling in
one closed form), Parseval's identity per block (normalisation, and which
bins are doubled), the constant signal, the Hamming window's values, the
block count of Alg. 6, the energy of each frequency's SVD, and the order of
the bins."""
import math

import numpy as np
import pytest

from oracle import spod as osp


def test_block_count_and_frequency_count():
    # nBlks = floor((T - nolap) / (npwin - nolap)); one-sided frequencies 0..npwin/2
    assert osp.spod_shape(4128, 64, 32) == (128, 33)
    assert osp.spod_shape(100, 60, 30) == (2, 31)
    assert osp.spod_shape(64, 64, 0) == (1, 33)
    assert osp.spod_shape(61, 60, 30) == (1, 31)


def test_hamming_window_values():
    w = osp.hamming(60)
    assert w[0] == pytest.approx(0.08, abs=1e-15) and w[-1] == pytest.approx(0.08, abs=1e-15)
    np.testing.assert_allclose(w, w[::-1], atol=1e-15)          # symmetric, j = 0 .. npwin - 1
    w7 = osp.hamming(7)
    assert w7[3] == pytest.approx(1.0, abs=1e-15)                # 0.54 + 0.46 at the centre
    assert w7[1] == pytest.approx(0.54 - 0.46 * math.cos(2 * math.pi / 6), abs=1e-15)


@pytest.mark.parametrize("npwin,nolap,t0", [(8, 4, 9), (8, 0, 3), (10, 5, 12), (7, 3, 5)])
def test_impulse_closed_form(npwin, nolap, t0):
    # D[p, t] = delta(t - t0): block b holds the impulse iff i0 <= t0 < i0 + npwin,
    # with i0 = b (npwin - nolap); there the transform at frequency k is
    # w[t0 - i0] exp(-2 pi i k (t0 - i0) / npwin) / (mean(w) npwin), doubled
    # for 0 < k < last, and every Q_f carries 1 / sqrt(nBlks)
    T = 3 * npwin
    D = np.zeros((2, T))
    D[:, t0] = 1.0
    Q = osp.spod_blocks(D, npwin, nolap, remove_mean=False)
    nblks, nfreq = osp.spod_shape(T, npwin, nolap)
    w = osp.hamming(npwin)
    for b in range(nblks):
        i0 = b * (npwin - nolap)
        for k in range(nfreq):
            if i0 <= t0 < i0 + npwin:
                j = t0 - i0
                ref = w[j] * np.exp(-2j * np.pi * k * j / npwin) / (w.mean() * npwin)
                if 0 < k < nfreq - 1:
                    ref *= 2.0
            else:
                ref = 0.0
            ref /= math.sqrt(nblks)
            assert abs(Q[k, 0, b] - ref) <= 1e-14, (b, k, Q[k, 0, b], ref)


def test_constant_signal():
    D = np.full((3, 200), 2.5)
    Q = osp.spod_blocks(D, 32, 16, remove_mean=False)
    nblks = Q.shape[2]
    # bin 0 of every block is the (window-weighted) mean of the block: 2.5
    np.testing.assert_allclose(Q[0], 2.5 / math.sqrt(nblks), atol=1e-13)
    # the temporal mean removes it entirely
    Q0 = osp.spod_blocks(D, 32, 16, remove_mean=True)
    assert np.max(np.abs(Q0)) <= 1e-13


@pytest.mark.parametrize("npwin", [16, 15])
def test_parseval_per_block(npwin):
    # for one block y_j = x_j w_j: sum_j y_j^2 = (1/n) sum over all n DFT
    # terms |Y_k|^2.  The one-sided q_k = c_k Y_k / (mean(w) n) keeps
    # k = 0 .. floor(n/2) and, as Alg. 6 writes it, doubles all but the first
    # and last kept entries: c = 1 at k = 0 and at the last k, 2 in between.
    # The last kept bin is the Nyquist term for even n (weight 1) but an
    # ordinary frequency with a mirror image for odd n (weight 2, undoubled).
    rng = np.random.default_rng(npwin)
    D = rng.standard_normal((4, npwin))
    Q = osp.spod_blocks(D, npwin, 0, remove_mean=False)[:, :, 0]   # nfreq x N, nBlks = 1
    w = osp.hamming(npwin)
    m, n = w.mean(), npwin
    lhs = np.sum((D * w[None, :]) ** 2, axis=1)
    weights = np.full(Q.shape[0], 0.5)     # |Y_k|^2 + |Y_{n-k}|^2 = 2 |Y_k|^2 = (m n)^2 |q_k|^2 / 2
    weights[0] = 1.0
    weights[-1] = 1.0 if n % 2 == 0 else 2.0
    rhs = (m * n) ** 2 / n * np.sum(weights[:, None] * np.abs(Q) ** 2, axis=0)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-13)


def test_energy_per_frequency_and_order():
    rng = np.random.default_rng(3)
    N, T, npwin, nolap = 30, 160, 32, 16
    x = np.linspace(0, 2 * np.pi, N, endpoint=False)
    t = np.arange(T)
    # two traveling waves at exact bins 3 and 10 of a 32-sample window, plus
    # noise (the Hamming window leaks about 0.43 of a wave into each
    # neighbouring bin, below the weaker wave's own 1.5)
    D = (2.0 * np.cos(3 * x[:, None] - 2 * np.pi * 3 * t[None, :] / npwin)
         + 1.5 * np.cos(5 * x[:, None] - 2 * np.pi * 10 * t[None, :] / npwin)
         + 1e-3 * rng.standard_normal((N, T)))
    out = osp.spod(D, 0.1, npwin, nolap, remove_mean=True, kmodes=3)
    for k in range(out["Q"].shape[0]):
        # the SVD of Q_f keeps its Frobenius energy
        assert np.sum(out["L"][k]) == pytest.approx(np.sum(np.abs(out["Q"][k]) ** 2), rel=1e-12)
    lead = out["L"][:, 0]
    order = out["order"]
    assert np.all(np.diff(lead[order]) <= 0.0)
    # the two waves' bins carry the two largest leading energies, the stronger first
    assert list(order[:2]) == [3, 10]
    np.testing.assert_allclose(out["f"], np.arange(npwin // 2 + 1) / (0.1 * npwin))
