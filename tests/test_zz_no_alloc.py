"""pylom_svd_small_noalloc: the small SVD for callers that cannot give the
library device memory (a host solver that owns every device buffer, or a loop
that may not allocate once running).  Its scratch is a fixed array inside the
library, so it is checked here against the workspace entry point
pylom_svd_small, through the C ABI, on two calls in a row (the second call
finds the first call's leftovers in the shared array).  This file is
collected last so that a stop-at-first-failure run has already run every
other test."""
import ctypes

import numpy as np
import pytest

import paper_2405_15529_gb300 as pg
from tests import parity


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2405_15529_gb300 import _build
    _build.build()
    lib = pg.load_library()
    fake = ctypes.c_void_p(0x100000)  # never dereferenced: the size check comes first
    st = lib.pylom_svd_small_noalloc(fake, 257, 257, fake, 257, fake, fake, 257, 60, None, None)
    assert st == pg.ERR_SHAPE
    assert b"256" in lib.pylom_last_error()
    st = lib.pylom_svd_small_noalloc(fake, 0, 1, fake, 1, fake, fake, 1, 60, None, None)
    assert st == pg.ERR_SHAPE


@pytest.mark.gpu
@pytest.mark.parametrize("M", [256, 37])
def test_noalloc_matches_workspace_entry_point(M):
    torch = pytest.importorskip("torch")
    R = np.random.default_rng(1000 + M).standard_normal((M, M)) * np.logspace(0, -4, M)[None, :]
    R = np.asfortranarray(np.triu(R))
    Rd = torch.from_numpy(np.ascontiguousarray(R.T)).cuda().t()
    U1, S1, VT1, sw1 = pg.svd_small(Rd)
    S1n = S1.cpu().numpy()
    for call in range(2):
        U2, S2, VT2, status, sweeps = pg.svd_small_noalloc(Rd)
        assert status == pg.OK, f"call {call}: device status {status}"
        assert 1 <= sweeps <= 60
        parity.check_sigma(S2.cpu().numpy(), S1n)
        parity.check_vectors(U2.cpu().numpy(), U1.cpu().numpy(), S1n)
        parity.check_vectors(VT2.cpu().numpy().T, VT1.cpu().numpy().T, S1n)
