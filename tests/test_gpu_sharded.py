"""GPU parity of the row-sharded POD (Sec. 3.1, Alg. 1 with the row blocks
as shards): each shard factors its rows (pylom_pod_shard_factor), the G
factors R_g are stacked by plain device copies (standing in for the
all-gather between devices), the replicated top runs once
(pylom_pod_rstack), and each shard forms its modes (pylom_pod_shard_modes).
The stacked result is compared element by element with the FP64 oracle's
POD of the whole matrix, at the oracle tolerances (binary64 path) or the
mixed-precision ones."""
import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")
from paper_2405_15529_gb300 import sharded  # noqa: E402


def _dev(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda", dtype).t()


def _run_shards(X, w, bounds, remove_mean, energy, r_max, leaf_rows, prec, mode_kind, xdtype=torch.float64):
    states = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        Xg = _dev(X[a:b], xdtype)
        wg = None if w is None else torch.from_numpy(w[a:b]).cuda()
        states.append((sharded.shard_factor(Xg, wg, remove_mean, leaf_rows, r_max, prec), wg))
    # the exchange: R_g into slot g of the stack on "every shard"
    Rstack = torch.stack([st.R.t().contiguous() for st, _ in states])
    top = sharded.rstack(Rstack, energy, r_max)
    Us = []
    for g, (st, wg) in enumerate(states):
        Us.append(sharded.shard_modes(st, top.B[g], top.r_dev, wg, mode_kind))
    torch.cuda.synchronize()
    for st, _ in states:
        assert pg.workspace_status(st.ws)[0] == pg.OK
    status, r, sweeps = pg.workspace_status(top.ws)
    assert status == pg.OK
    U = torch.cat([u[:, :r] for u in Us]).cpu().numpy()
    mean = torch.cat([st.mean for st, _ in states]).cpu().numpy()
    return U, top.S.cpu().numpy(), top.VT.cpu().numpy(), r, mean


CASES = [
    # N, M, shard row counts (fractions), leaf_rows, weights, mean, energy, r_max
    (6000, 48, [0.5, 0.5], 700, False, True, 0.0, 48),
    (9001, 40, [0.2, 0.5, 0.3], 0, True, True, 0.99, 40),
    (7000, 33, [0.1, 0.3, 0.2, 0.25, 0.15], 500, True, False, 0.0, 20),
    (5000, 400, [0.3, 0.3, 0.4], 0, False, True, 0.0, 64),     # M >= 384: cooperative trees
]


def _bounds(N, fr):
    cuts = np.round(np.cumsum([0.0] + list(fr)) * N).astype(int)
    cuts[-1] = N
    return [int(c) for c in cuts]


@pytest.mark.parametrize("case", CASES)
def test_sharded_fp64_matches_oracle(case):
    N, M, fr, b, weighted, rm, energy, r_max = case
    X = synth.waves(N, M, n_waves=min(8, M // 4), noise=1e-3, seed=31 + M)
    w = synth.log_uniform_weights(N, seed=32) if weighted else None
    bounds = _bounds(N, fr)
    U, S, VT, r, mean = _run_shards(X, w, bounds, rm, energy, r_max, b, pg.PREC_FP64, pg.MODES_ORTHONORMAL)
    ref = oracle.pod(X, w=w, remove_mean=rm, energy=energy, r_max=r_max)
    assert r == ref["r"]
    parity.check_sigma(S, ref["S"])
    parity.check_vectors(U, ref["U"], ref["S"], ncols=r)
    parity.check_vectors(VT[:r].T, ref["VT"][:r].T, ref["S"], ncols=r)
    np.testing.assert_allclose(mean, ref["mean"], rtol=0, atol=1e-13 * max(1.0, np.abs(X).max()))
    # orthonormal to rounding: about r epsilon-sized entries per column, each
    # from a few hundred reflector applications (leaf, shard tree, top tree)
    assert parity.orthonormality(U) <= r * 1e-13


def test_sharded_physical_modes_and_single_shard():
    N, M = 4000, 24
    X = synth.waves(N, M, n_waves=4, noise=1e-3, seed=41)
    w = synth.log_uniform_weights(N, seed=42)
    ref = oracle.pod(X, w=w, remove_mean=True, mode_kind=pg.MODES_PHYSICAL)
    for bounds in ([0, N], [0, 1500, N]):
        U, S, VT, r, _ = _run_shards(X, w, bounds, True, 0.0, M, 0, pg.PREC_FP64, pg.MODES_PHYSICAL)
        parity.check_sigma(S, ref["S"])
        parity.check_vectors(U, ref["U"], ref["S"], ncols=r, weight=w)


def test_sharded_mixed_matches_fp64_oracle():
    N, M = 8192, 64
    XT, w, s = synth.known_spectrum_torch(N, M, device="cuda", dtype=torch.float32, seeds=(52, 53, 54))
    X = XT.t().cpu().numpy().astype(np.float64)
    wn = w.cpu().numpy()
    bounds = [0, 3000, 5000, N]
    U, S, VT, r, _ = _run_shards(X, wn, bounds, False, 0.0, M, 0, pg.PREC_MIXED_3XTF32, pg.MODES_ORTHONORMAL,
                                 xdtype=torch.float32)
    ref = oracle.pod(X, w=wn, remove_mean=False)
    assert np.max(np.abs(S - ref["S"])) <= 2e-6 * ref["S"][0]
    keep = [i for i in range(r) if ref["S"][i] >= 1e-3 * ref["S"][0]]
    parity.check_vectors(U[:, keep], ref["U"][:, keep], ref["S"][keep], ncols=len(keep))


def test_sharded_rejects_bad_shapes():
    X = torch.zeros((100, 200), dtype=torch.float64, device="cuda")     # N_g < M
    with pytest.raises(pg.PylomError):
        sharded.shard_factor(X)
    with pytest.raises(pg.PylomError):
        sharded.rstack(torch.zeros((2, 8, 8), dtype=torch.float64, device="cuda"), r_max=9)
