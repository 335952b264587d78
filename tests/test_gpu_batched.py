"""GPU parity of the batched complex SVDs (per-frequency SVDs of SPOD):
every bin against the complex128 oracle, the complex64 ("mixed") batched
path against single-bin binary64 runs, graph replay, Parseval per bin, and
non-finite input."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")

MIXED_SIGMA = 2e-6      # |dS| <= 2e-6 S_max for the complex64 leaves
FP64_SIGMA = 1e-12


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda").t()


def _bins():
    """Small bins of mixed shapes: wave bins and known complex spectra,
    ragged leaf counts, Nb from 1 to 40."""
    out = []
    for i, (N, Nb) in enumerate([(3000, 24), (777, 7), (5000, 40), (300, 1), (2048, 16), (1500, 33)]):
        if i % 2 == 0:
            X = synth.spod_bin(N, Nb, seed=100 + i)
        else:
            X, _ = synth.complex_known_spectrum(N, Nb, seeds=(110 + i, 120 + i), dtype=np.complex64)
        out.append(np.asfortranarray(X.astype(np.complex64)))
    return out


# The complex64 leaves perturb R by about 2^-24 S_max, so a mode's angle
# error is about 2^-24 S_max / gap; the 1 - 1e-6 overlap bound is met where
# the mode's singular value is at least 1e-3 S_max.
MIXED_MODE_FLOOR = 1e-3


def _check_modes(U, U_ref, S_ref, k, tol=1e-6, gap=1e-3, floor=0.0):
    from tests import parity
    for grp in parity.clusters(S_ref, gap):
        grp = [i for i in grp if i < k and S_ref[i] >= floor * S_ref[0]]
        if not grp:
            continue
        G = U[:, grp].conj().T @ U_ref[:, grp]
        v = abs(G[0, 0]) if len(grp) == 1 else np.linalg.svd(G, compute_uv=False).min()
        assert v >= 1 - tol, (grp, v)


@pytest.mark.parametrize("prec,stol", [(pg.PREC_FP64, FP64_SIGMA), (pg.PREC_MIXED_3XTF32, MIXED_SIGMA)])
def test_batched_matches_oracle(prec, stol):
    bins = _bins()
    Q = [_dev(X) for X in bins]
    b = pg.BatchedSVD(Q, kmodes=8, prec=prec, leaf_rows=[512, 64, 700, 0, 128, 300])
    b.run()
    assert b.status() == pg.OK
    for f, X in enumerate(bins):
        U_ref, S_ref, V_ref, _ = oracle.zsvd(X.astype(np.complex128))
        S = b.S[f].cpu().numpy()
        assert np.max(np.abs(S - S_ref)) <= stol * S_ref[0], (f, np.max(np.abs(S - S_ref)) / S_ref[0])
        assert np.all(np.diff(S) <= 0)
        k = b.k[f]
        U = b.modes[f].cpu().numpy().astype(np.complex128)
        floor = 0.0 if prec == pg.PREC_FP64 else MIXED_MODE_FLOOR
        _check_modes(U, U_ref, S_ref, k, floor=floor)
        # same phase rule as the oracle: isolated modes agree as vectors.  With
        # |<u, u_ref>| >= 1 - 1e-6 and a consistent phase, |u - u_ref| <= 1.5e-3;
        # a phase-rule mismatch would be O(1).
        from tests import parity
        vtol = 1e-5 if prec == pg.PREC_FP64 else 2e-3
        for grp in parity.clusters(S_ref):
            if len(grp) == 1 and grp[0] < k and S_ref[grp[0]] >= floor * S_ref[0]:
                i = grp[0]
                assert np.linalg.norm(U[:, i] - U_ref[:, i]) <= vtol, (f, i)


def test_batched_mixed_equals_single_bin_fp64_runs():
    bins = _bins()
    Q = [_dev(X) for X in bins]
    mixed = pg.BatchedSVD(Q, kmodes=4, prec=pg.PREC_MIXED_3XTF32)
    mixed.run()
    assert mixed.status() == pg.OK
    for f, q in enumerate(Q):
        single = pg.BatchedSVD([q], kmodes=4, prec=pg.PREC_FP64)
        single.run()
        assert single.status() == pg.OK
        S1, Sm = single.S[0].cpu().numpy(), mixed.S[f].cpu().numpy()
        assert np.max(np.abs(Sm - S1)) <= MIXED_SIGMA * S1[0]
        _check_modes(mixed.modes[f].cpu().numpy().astype(np.complex128),
                     single.modes[0].cpu().numpy().astype(np.complex128), S1, mixed.k[f],
                     floor=MIXED_MODE_FLOOR)


def test_batched_graph_replay_and_parseval():
    bins = _bins()
    Q = [_dev(X) for X in bins]
    b = pg.BatchedSVD(Q, kmodes=8, prec=pg.PREC_MIXED_3XTF32)
    b.run()
    torch.cuda.synchronize()
    S0 = b.S_all.clone()
    U0 = [m.clone() for m in b.modes]
    b.capture()
    b.S_all.zero_()
    for _ in range(2):
        b.replay()
    torch.cuda.synchronize()
    assert b.status() == pg.OK
    assert torch.equal(b.S_all, S0)
    for u, u0 in zip(b.modes, U0):
        assert torch.equal(u, u0)
    for f, X in enumerate(bins):
        e = float(np.sum(np.abs(X.astype(np.complex128)) ** 2))
        assert float(torch.sum(b.S[f] ** 2)) == pytest.approx(e, rel=1e-5)


def test_batched_reports_nonfinite():
    X = synth.spod_bin(1000, 10, seed=3)
    X[5, 2] = np.nan
    b = pg.BatchedSVD([_dev(X)], kmodes=2, prec=pg.PREC_MIXED_3XTF32)
    b.run()
    assert b.status() == pg.ERR_NONFINITE


def test_batched_rejects_bad_plans():
    with pytest.raises(pg.PylomError):
        pg.BatchedSVD([_dev(synth.spod_bin(200, 129, seed=1))], kmodes=2)     # Nb > 128
    with pytest.raises(pg.PylomError):
        pg.BatchedSVD([_dev(synth.spod_bin(500, 10, seed=1))], kmodes=33)     # kmodes > 32


# Bins at the sizes the 256-bin workload runs: Nb up to the 128-column limit,
# leaves at the 1024-row cap of complex64 leaves (512 for complex128), bins
# split into several capped leaves, and up to 32 returned modes.  The
# known-spectrum bins (geometric decay over six decades) keep all 32 leading
# modes separated, so every mode is compared as a vector.
_BIG_SPECS = [  # N, Nb, leaf-height hint
    (4096, 128, 1024),   # 4 leaves of exactly 1024 rows (complex64)
    (5000, 96, 1024),    # hint 1024 -> 4 leaves of 1250 rows, split to 5 of 1000
    (3001, 127, 0),      # built-in height, ragged leaves, odd Nb
    (2048, 64, 1024),
    (1100, 128, 0),      # split into two leaves of 550 rows
]
_BIG_CACHE = {}


def _big_bins():
    if not _BIG_CACHE:
        for i, (N, Nb, _) in enumerate(_BIG_SPECS):
            if i % 2 == 0:
                X, _ = synth.complex_known_spectrum(N, Nb, seeds=(210 + i, 220 + i), dtype=np.complex64)
            else:
                X = synth.spod_bin(N, Nb, seed=200 + i)
            X = np.asfortranarray(X.astype(np.complex64))
            U_ref, S_ref, _, _ = oracle.zsvd(X.astype(np.complex128))
            _BIG_CACHE[i] = (X, U_ref, S_ref)
    return [_BIG_CACHE[i] for i in range(len(_BIG_SPECS))]


@pytest.mark.parametrize("kmodes", [8, 32])
@pytest.mark.parametrize("prec,stol", [(pg.PREC_FP64, FP64_SIGMA), (pg.PREC_MIXED_3XTF32, MIXED_SIGMA)])
def test_batched_full_size_bins_match_oracle(prec, stol, kmodes):
    from tests import parity
    bins = _big_bins()
    b = pg.BatchedSVD([_dev(X) for X, _, _ in bins], kmodes=kmodes, prec=prec,
                      leaf_rows=[h for _, _, h in _BIG_SPECS])
    b.run()
    assert b.status() == pg.OK
    hmax = pg.batched_max_leaf_rows(prec)
    for f, ((X, U_ref, S_ref), (N, Nb, hint)) in enumerate(zip(bins, _BIG_SPECS)):
        # the leaf partition: the hint (or the cap), split so no leaf exceeds the cap
        h = hint if hint > 0 else min(hmax, N)
        P = max(N // h, -(-N // hmax), 1)
        assert b.info(f, 1) == P, (f, b.info(f, 1), P)
        assert -(-N // P) <= hmax
        S = b.S[f].cpu().numpy()
        assert np.max(np.abs(S - S_ref)) <= stol * S_ref[0], (f, np.max(np.abs(S - S_ref)) / S_ref[0])
        assert np.all(np.diff(S) <= 0)
        k = b.k[f]
        assert k == min(kmodes, Nb)
        U = b.modes[f].cpu().numpy().astype(np.complex128)
        floor = 0.0 if prec == pg.PREC_FP64 else MIXED_MODE_FLOOR
        _check_modes(U, U_ref, S_ref, k, floor=floor)
        vtol = 1e-5 if prec == pg.PREC_FP64 else 2e-3
        for grp in parity.clusters(S_ref):
            if len(grp) == 1 and grp[0] < k and S_ref[grp[0]] >= floor * S_ref[0]:
                i = grp[0]
                assert np.linalg.norm(U[:, i] - U_ref[:, i]) <= vtol, (f, i)
        # orthonormal returned modes (complex64 storage)
        G = U[:, :k].conj().T @ U[:, :k]
        assert np.linalg.norm(G - np.eye(k), 2) <= 1e-5
