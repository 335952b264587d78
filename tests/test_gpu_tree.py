"""GPU parity of the three forms of the tree reduction (Sec. 3.1, the reduce
loop of Alg. 1): last-arriver merges inside the leaf kernels, the
cooperative kernel that spreads every merge over all blocks, and the
column-block pipeline with one block per merge (chosen with the PYLOM_TREE
environment variable), each against the FP64 oracle, against each other, and
through the top-down pass, the mixed path and the adjoint, which read the
node reflectors all three forms leave behind."""
import functools
import math

import numpy as np
import pytest

import oracle
import synth
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

pg = pytest.importorskip("paper_2405_15529_gb300")

TREES = ["climb", "coop", "pipe"]


def _dev(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to("cuda").t()


@functools.lru_cache(maxsize=None)
def _case(N, M, remove_mean):
    X = synth.waves(N, M, n_waves=min(16, max(1, M // 4)), noise=1e-3, seed=N + M)
    return X, oracle.pod(X, remove_mean=remove_mean)


SHAPES = [
    (3001, 37, 128, True),       # P = 23, last panel short
    (5000, 10, 500, False),      # M below one panel
    (20000, 100, 1000, True),    # P = 20, seven panels
    (1 << 20, 48, 0, True),      # automatic P = 304: nine levels, odd counts; the pipeline by default
    (40000, 520, 2500, False),   # P = 16, 33 panels; the cooperative tree by default
]


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("N,M,b,remove_mean", SHAPES)
def test_pod_both_trees_match_oracle(monkeypatch, tree, N, M, b, remove_mean):
    monkeypatch.setenv("PYLOM_TREE", tree)
    X, ref = _case(N, M, remove_mean)
    res = pg.pod(_dev(X), remove_mean=remove_mean, leaf_rows=b)
    parity.check_sigma(res.S.cpu().numpy(), ref["S"])
    assert res.r == ref["r"]
    parity.check_vectors(res.U.cpu().numpy(), ref["U"], ref["S"], ncols=res.r)
    parity.check_vectors(res.VT.cpu().numpy().T, ref["VT"].T, ref["S"], ncols=res.r)


def test_coop_tree_repeatable_and_agrees_with_climb(monkeypatch):
    X, _ = _case(1 << 20, 48, True)
    Xd = _dev(X)
    monkeypatch.setenv("PYLOM_TREE", "coop")
    a = pg.pod(Xd, leaf_rows=0)
    b = pg.pod(Xd, leaf_rows=0)
    assert torch.equal(a.S, b.S) and torch.equal(a.U, b.U) and torch.equal(a.VT, b.VT)
    monkeypatch.setenv("PYLOM_TREE", "climb")
    c = pg.pod(Xd, leaf_rows=0)
    S = a.S.cpu().numpy()
    assert np.max(np.abs(S - c.S.cpu().numpy())) <= 1e-13 * S[0]


def test_pipe_tree_repeatable_and_agrees_with_coop(monkeypatch):
    X, _ = _case(1 << 20, 48, True)
    Xd = _dev(X)
    monkeypatch.setenv("PYLOM_TREE", "pipe")
    a = pg.pod(Xd, leaf_rows=0)
    b = pg.pod(Xd, leaf_rows=0)
    assert torch.equal(a.S, b.S) and torch.equal(a.U, b.U) and torch.equal(a.VT, b.VT)
    monkeypatch.setenv("PYLOM_TREE", "coop")
    c = pg.pod(Xd, leaf_rows=0)
    S = a.S.cpu().numpy()
    assert np.max(np.abs(S - c.S.cpu().numpy())) <= 1e-13 * S[0]
    parity.check_vectors(a.U.cpu().numpy(), c.U.cpu().numpy(), S, ncols=a.r)


@pytest.mark.parametrize("P", [2, 3, 64, 65, 127, 300])
def test_pipe_tree_leaf_counts(monkeypatch, P):
    """Uneven trees: a missing partner passes R up, so a merge's bottom child
    can be a leaf or a merge several levels down."""
    monkeypatch.setenv("PYLOM_TREE", "pipe")
    N, M = 40 * P + 17, 33
    A = np.asfortranarray(np.random.default_rng(P).standard_normal((N, M)))
    R, Q = pg.tsqr(_dev(A), leaf_rows=N // P)
    R, Q = R.cpu().numpy(), Q.cpu().numpy()
    nA = np.linalg.norm(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(R.T @ R - A.T @ A) <= 1e-13 * nA ** 2
    assert np.linalg.norm(Q.T @ Q - np.eye(M)) <= 1e-13 * math.sqrt(M)
    assert np.linalg.norm(Q @ R - A) <= 1e-13 * nA


@pytest.mark.parametrize("tree", ["coop", "pipe"])
@pytest.mark.parametrize("N,M,b", [(3001, 37, 128), (1 << 18, 40, 0), (30000, 400, 3000)])
def test_tsqr_coop_tree(monkeypatch, tree, N, M, b):
    monkeypatch.setenv("PYLOM_TREE", tree)
    A = np.asfortranarray(np.random.default_rng(N + M).standard_normal((N, M)))
    R, Q = pg.tsqr(_dev(A), leaf_rows=b)
    R, Q = R.cpu().numpy(), Q.cpu().numpy()
    nA = np.linalg.norm(A)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.linalg.norm(R.T @ R - A.T @ A) <= 1e-13 * nA ** 2
    assert np.linalg.norm(Q.T @ Q - np.eye(M)) <= 1e-13 * math.sqrt(M)
    assert np.linalg.norm(Q @ R - A) <= 1e-13 * nA


@pytest.mark.parametrize("tree", ["coop", "pipe"])
@pytest.mark.parametrize("N,M,b", [(3001, 37, 128), (40000, 520, 2500)])
def test_mixed_path_coop_tree(monkeypatch, tree, N, M, b):
    monkeypatch.setenv("PYLOM_TREE", tree)
    X, ref = _case(N, M, False)
    res = pg.pod(_dev(X.astype(np.float32)), remove_mean=False, leaf_rows=b, prec=pg.PREC_MIXED_3XTF32)
    S, S_ref = res.S.cpu().numpy(), ref["S"]
    # the oracle factors the float64 matrix; float32 storage moves sigma by ~2^-24 S_max
    assert np.max(np.abs(S - S_ref)) <= 2e-6 * S_ref[0]


@pytest.mark.parametrize("tree", ["coop", "pipe"])
def test_adjoint_through_coop_tree(monkeypatch, tree):
    monkeypatch.setenv("PYLOM_TREE", tree)
    N, M, r = 512, 16, 4
    X, w, s = synth.known_spectrum(N, M, weights=True, seeds=(7, 8, 9))
    Xd = _dev(X).requires_grad_(True)
    wd = torch.from_numpy(w).cuda()
    U, S, VT = pg.pod_autograd(Xd, r, w=wd, remove_mean=False, leaf_rows=64)
    Yw = Xd * torch.sqrt(wd)[:, None]
    L = torch.sum((Yw - U @ (U.T @ Yw)) ** 2)
    L.backward()
    _, G_ref = oracle.pod_loss_grad(X, r, w=w, remove_mean=False)
    G = Xd.grad.cpu().numpy()
    assert np.linalg.norm(G - G_ref) / np.linalg.norm(G_ref) <= 1e-6
