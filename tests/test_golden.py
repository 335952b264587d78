"""Stored fixtures (tests/golden/): values the paper prints for its SPOD
validation case, and the oracle's POD of a small seeded field written by
tests/golden/make_golden.py (which calls only the oracle).  The CPU tests
check the oracle and the library's host-side SPOD shape against them; the
GPU test holds the CUDA path to the stored oracle values at the parity
tolerances."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import spod as ospod
from tests import parity
from tests.golden import make_golden as mg

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _spod_case():
    g = mg.read_fixture(os.path.join(HERE, "spod_cylinder_re100.txt"))
    T, npwin = int(g["snapshots"]), int(g["npwin"])
    nolap = int(round(g["overlap_fraction"] * npwin))
    return g, T, npwin, nolap


def test_spod_frequency_axis_holds_the_papers_frequencies():
    """Sec. 2.3 / Alg. 6: one-sided frequencies k / (dt npwin).  With the
    cylinder case's dt = 0.2 and 60-snapshot windows the grid step is 1/12,
    and the two frequencies the paper reports (0.166, 0.333, truncated to
    three decimals) are bins 2 and 4."""
    g, T, npwin, nolap = _spod_case()
    nblks, nfreq = ospod.spod_shape(T, npwin, nolap)
    f = np.arange(nfreq) / (g["dt"] * npwin)
    for _, printed in g["freq"]:
        k = int(np.argmin(np.abs(f - printed)))
        assert 0.0 <= f[k] - printed < 1e-3            # truncated, not rounded
        assert math.isclose(f[k] * g["dt"] * npwin, round(f[k] * g["dt"] * npwin), abs_tol=1e-9)
    assert [int(np.argmin(np.abs(f - p))) for _, p in g["freq"]] == [2, 4]
    # 151 snapshots in windows of 60 overlapping by 30: 4 whole blocks
    assert (nblks, nfreq) == (4, 31)
    assert (nblks - 1) * (npwin - nolap) + npwin <= T < nblks * (npwin - nolap) + npwin


def test_library_spod_shape_matches_the_case():
    import ctypes
    import paper_2405_15529_gb300 as pg
    from paper_2405_15529_gb300 import _build
    _build.build()
    lib = pg.load_library()
    _, T, npwin, nolap = _spod_case()
    nb, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.pylom_spod_shape(T, npwin, nolap, ctypes.byref(nb), ctypes.byref(nf)) == 0
    assert (nb.value, nf.value) == ospod.spod_shape(T, npwin, nolap)


def _pod_fixture():
    g = mg.read_fixture(mg.POD_FILE)
    S = np.array([v for _, v in sorted(g["S"])])
    mean = dict(g["mean"])
    return int(g["r"]), S, mean


def test_oracle_reproduces_its_stored_pod():
    """A change to the oracle's arithmetic shows here; regenerating the
    fixture is then a deliberate step (make_golden.py)."""
    r, S, mean = _pod_fixture()
    X, w = mg.pod_case_inputs()
    res = oracle.pod(X, w=w, remove_mean=True, energy=mg.POD_CASE["energy"])
    assert res["r"] == r
    np.testing.assert_allclose(res["S"], S, rtol=0, atol=1e-13 * S[0])
    for n, v in mean.items():
        assert abs(res["mean"][n] - v) <= 1e-15 * abs(v) * 8


@pytest.mark.gpu
def test_cuda_pod_matches_the_stored_oracle_values():
    torch = pytest.importorskip("torch")
    import paper_2405_15529_gb300 as pg
    r, S, mean = _pod_fixture()
    X, w = mg.pod_case_inputs()
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to("cuda").t()
    res = pg.pod(Xd, w=torch.from_numpy(w).cuda(), remove_mean=True, energy=mg.POD_CASE["energy"])
    parity.check_sigma(res.S.cpu().numpy(), S)
    assert res.r == r
    m = res.mean.cpu().numpy()
    for n, v in mean.items():
        assert abs(m[n] - v) <= 1e-14 * abs(v)
