"""Failure detection of the bounded device waits, without a GPU fault.

Every cooperative kernel of the library waits on other thread blocks only
through its grid barrier, and the mixed-precision leaves wait on their
tcgen05 commits through an mbarrier; both poll the GPU's global timer and give
up after a limit.  pylom_wait_selftest makes each form wait for something
that never comes, with a limit of a few milliseconds: the wait must give up,
record PYLOM_ERR_TIMEOUT, let its kernel end, and leave the context usable
for the next call on the same stream."""
import ctypes
import time

import numpy as np
import pytest

import paper_2405_15529_gb300 as pg


@pytest.fixture(scope="module")
def lib():
    from paper_2405_15529_gb300 import _build
    _build.build()
    return pg.load_library()


def test_selftest_host_validation(lib):
    # rejected on the host before anything is launched (no GPU needed)
    fake = ctypes.c_void_p(0x100000)
    assert lib.pylom_wait_selftest(2, 4, 2.0, None, fake, 512, None) == pg.ERR_ARG
    assert lib.pylom_wait_selftest(0, 0, 2.0, None, fake, 512, None) == pg.ERR_ARG
    assert lib.pylom_wait_selftest(0, 4, 0.0, None, fake, 512, None) == pg.ERR_ARG
    assert lib.pylom_wait_selftest(0, 4, 2500.0, None, fake, 512, None) == pg.ERR_ARG
    assert lib.pylom_wait_selftest(0, 4, 2.0, None, ctypes.c_void_p(0x100010), 512, None) == pg.ERR_WORKSPACE
    assert lib.pylom_wait_selftest(0, 4, 2.0, None, fake, 100, None) == pg.ERR_WORKSPACE
    assert lib.pylom_wait_selftest_workspace_size() == 512


@pytest.mark.gpu
@pytest.mark.parametrize("kind,blocks", [("grid", 1), ("grid", 64), ("grid", 608), ("mbarrier", 1)])
def test_bounded_wait_gives_up_and_context_survives(lib, kind, blocks):
    torch = pytest.importorskip("torch")
    t0 = time.perf_counter()
    st, gave = pg.wait_selftest(kind, blocks=blocks, limit_ms=3.0)
    dt = time.perf_counter() - t0
    assert st == pg.ERR_TIMEOUT
    assert gave == blocks          # every waiting block gave up and returned
    assert dt < 10.0
    # a normal call on the same stream afterwards succeeds
    rng = np.random.default_rng(7)
    R = np.triu(rng.standard_normal((24, 24)))
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda().t()
    U, S, VT, sweeps = pg.svd_small(Rd)
    S_ref = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(S.cpu().numpy() - S_ref)) <= 1e-12 * S_ref[0]
