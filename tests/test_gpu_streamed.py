"""GPU parity of the out-of-core POD (snapshot matrix in host memory,
streamed through the device in chunks of whole leaves): it runs the same
kernels on the same leaves as the in-core call, so its results must equal
those of pylom_pod with the same leaf partition bit for bit -- for the
last-arriver tree (M < 384 and fewer than 64 leaves), whose merges span chunk launches, and for the
cooperative tree (M >= 384 or 64 leaves), launched once after the last chunk -- and the
FP64 oracle's within the parity tolerances."""
import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")


def _host(X, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to(dtype).t()


@pytest.mark.parametrize("N,M,b,chunk,dtype,weighted,mode_kind,energy", [
    (20000, 40, 1000, 3000, torch.float64, False, 0, 0.0),   # climb tree, 7 chunks, P = 20
    (20011, 33, 900, 2500, torch.float32, True, 1, 0.0),     # ragged leaves, F32 input, physical modes
    (40000, 400, 4000, 9000, torch.float64, False, 0, 0.0),  # cooperative tree, 5 chunks
    (40000, 400, 4000, 1 << 30, torch.float64, True, 0, 0.0),  # cooperative tree, one chunk
    (30000, 64, 1024, 4000, torch.float64, False, 0, 1e-6),  # energy truncation
    (400000, 32, 0, 1 << 18, torch.float32, False, 0, 0.0),  # automatic leaves: 304 per chunk, 2 chunks
])
def test_streamed_equals_in_core(N, M, b, chunk, dtype, weighted, mode_kind, energy):
    X = synth.waves(N, M, n_waves=min(8, M // 4), noise=1e-3, seed=N + M)
    w = synth.log_uniform_weights(N, seed=3) if weighted else None
    Xh = _host(X, dtype)
    wd = None if w is None else torch.from_numpy(w).cuda()
    b_eff = pg.pod_streamed_leaf_rows(N, M, b, chunk)
    assert b_eff == (b if b > 0 else max(M, 1024, chunk // 304))
    ref = pg.pod(Xh.cuda(), w=wd, energy=energy, mode_kind=mode_kind, leaf_rows=b_eff)
    res = pg.pod_streamed(Xh, w=w, energy=energy, mode_kind=mode_kind, leaf_rows=b, chunk_rows=chunk)
    assert res.r == ref.r
    assert torch.equal(res.S, ref.S)
    assert torch.equal(res.VT, ref.VT)
    assert torch.equal(res.U, ref.U.cpu())
    assert torch.equal(res.mean, ref.mean.cpu())


def test_streamed_matches_oracle():
    N, M, b = 9001, 24, 700
    X = synth.waves(N, M, n_waves=6, noise=1e-3, seed=5)
    w = synth.log_uniform_weights(N, seed=8)
    ref = oracle.pod(X, w=w, remove_mean=True, mode_kind=1)
    res = pg.pod_streamed(_host(X), w=w, mode_kind=1, leaf_rows=b, chunk_rows=2000)
    S_ref = ref["S"]
    parity.check_sigma(res.S.cpu().numpy(), S_ref, abs_tol=parity.SIGMA_ABS)
    assert res.r == ref["r"]
    parity.check_vectors(res.U.numpy(), ref["U"], S_ref, ncols=res.r, weight=w)
    np.testing.assert_allclose(res.mean.numpy(), ref["mean"], rtol=0, atol=1e-14 * np.abs(X).max())


def test_streamed_rejects_bad_arguments():
    X = torch.zeros((1000, 20), dtype=torch.float64)
    with pytest.raises(pg.PylomError):
        pg.pod_streamed(X, leaf_rows=10)          # leaves shorter than M
    with pytest.raises(pg.PylomError):
        pg.pod_streamed(X, chunk_rows=0)
    with pytest.raises(ValueError):
        pg.pod_streamed(X.cuda())                 # the streamed path takes host memory
