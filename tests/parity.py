"""Comparison helpers for GPU-vs-oracle parity (tolerances from the POD
accuracy targets: FP64 path |dS| <= 1e-12 S_max, relative 1e-12 where
S >= 1e-2 S_max; modes up to sign with |<u, u_ref>| >= 1 - 1e-6 where the
singular value is separated by >= 1e-3 relatively, else a subspace check)."""
from __future__ import annotations

import numpy as np

SIGMA_ABS = 1e-12
SIGMA_REL = 1e-12
MODE_TOL = 1e-6
GAP = 1e-3
NULL_REL = 1e-10


def check_sigma(S, S_ref, abs_tol=SIGMA_ABS, rel_tol=SIGMA_REL):
    S = np.asarray(S); S_ref = np.asarray(S_ref)
    smax = max(S_ref[0], 1e-300)
    err = np.abs(S - S_ref)
    assert np.all(err <= abs_tol * smax), f"max |dS|/S_max = {err.max() / smax:.3e}"
    big = S_ref >= 1e-2 * smax
    if big.any():
        rel = err[big] / S_ref[big]
        assert np.all(rel <= rel_tol), f"max relative dS = {rel.max():.3e}"
    assert np.all(np.diff(S) <= 0.0), "singular values not sorted descending"


def clusters(S, gap=GAP, null_rel=NULL_REL):
    """Groups of consecutive indices whose singular values are closer than
    `gap` relatively; values below null_rel * S_max are left out."""
    S = np.asarray(S)
    keep = np.nonzero(S > null_rel * S[0])[0]
    groups, cur = [], []
    for i in keep:
        if cur and (S[cur[-1]] - S[i]) > gap * S[cur[-1]]:
            groups.append(cur); cur = []
        cur.append(int(i))
    if cur:
        groups.append(cur)
    return groups


def check_vectors(U, U_ref, S_ref, ncols=None, tol=MODE_TOL, gap=GAP, weight=None):
    """Columns of U against U_ref up to sign (separated values) or as
    subspaces (clusters).  weight: optional inner-product weights."""
    U = np.asarray(U); U_ref = np.asarray(U_ref)
    n = U.shape[1] if ncols is None else ncols
    worst = 1.0
    for grp in clusters(S_ref, gap):
        grp = [i for i in grp if i < n]
        if not grp:
            continue
        A = U[:, grp]; B = U_ref[:, grp]
        G = A.T @ (B * weight[:, None]) if weight is not None else A.T @ B
        if len(grp) == 1:
            v = abs(G[0, 0])
        else:
            v = np.linalg.svd(G, compute_uv=False).min()
        worst = min(worst, v)
        assert v >= 1.0 - tol, f"modes {grp}: overlap {v:.9f}"
    return worst


def orthonormality(U, weight=None):
    U = np.asarray(U)
    G = U.T @ (U * weight[:, None]) if weight is not None else U.T @ U
    return np.linalg.norm(G - np.eye(U.shape[1]))
