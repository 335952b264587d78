"""The autotuner of the batched SVD's leaf heights (paper_2405_15529_gb300.tune):
candidate lists, cache keys and the cache round trip on the CPU; on the GPU,
that the chosen height is the fastest one timed and that BatchedSVD runs the
chosen heights."""
import json

import numpy as np
import pytest

import paper_2405_15529_gb300 as pg
from paper_2405_15529_gb300 import tune


@pytest.fixture(scope="module")
def lib():
    from paper_2405_15529_gb300 import _build
    _build.build()
    return pg.load_library()


def test_max_leaf_rows_query(lib):
    assert pg.batched_max_leaf_rows(pg.PREC_MIXED_3XTF32) == 1024
    assert pg.batched_max_leaf_rows(pg.PREC_FP64) == 512
    assert lib.pylom_svd_batched_max_leaf_rows(7) == -1


def test_candidates_respect_bin_and_library_limits():
    assert tune.candidates(1 << 20, 16, 1024) == [256, 384, 512, 768, 1024]
    # complex128 leaves stop at 512 rows: taller hints would be split again
    assert tune.candidates(1 << 20, 16, 512) == [256, 384, 512]
    # never fewer rows than columns, never more rows than the bin has
    assert tune.candidates(1 << 20, 300, 1024) == [300, 384, 512, 768, 1024]
    assert tune.candidates(600, 64, 1024) == [256, 384, 512]
    assert tune.candidates(100, 64, 1024) == []
    for N, Nb, hmax in [(70000, 128, 1024), (5000, 40, 512)]:
        c = tune.candidates(N, Nb, hmax)
        assert c == sorted(set(c)) and all(Nb <= h <= min(N, hmax) for h in c)


def test_classes_and_keys():
    assert tune._classes(65536, 16) == (16, 16)
    assert tune._classes(1048575, 17) == (32, 19)
    assert tune._classes(300000, 128) == (128, 18)
    assert tune._key("NVIDIA GB300", 1, 128, 18) == "NVIDIA GB300|prec1|nb128|n2^18"


def test_cache_round_trip(tmp_path, monkeypatch):
    path = str(tmp_path / "cache.json")
    monkeypatch.setattr(tune, "CACHE", path)
    monkeypatch.setattr(tune, "gpu_name", lambda: "cpu")
    assert tune._load() == {}
    d = {"cpu|prec1|nb32|n2^16": 512, "cpu|prec1|nb128|n2^19": 1024}
    tune._save(d)
    assert json.load(open(path)) == d
    assert tune._load() == d
    # cached classes are read without tuning; a missing class gives 0 (the
    # library's built-in choice); never fewer rows than the bin's columns
    out = tune.leaf_rows_for([70000, 600000, 70000], [20, 100, 500], pg.PREC_MIXED_3XTF32, tune=False)
    assert out == [512, 1024, 0]


@pytest.mark.gpu
def test_tuned_height_is_fastest_and_is_run(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    import synth
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    prec = pg.PREC_MIXED_3XTF32
    best, times = tune.tune_class(1 << 14, 32, prec)
    assert set(times) == set(tune.candidates(1 << 14, 32, 1024))
    assert times[best] == min(times.values())
    Ns, Nbs = [20000, 17000], [30, 25]          # both in class (nb 32, n 2^14)
    heights = tune.leaf_rows_for(Ns, Nbs, prec, tune=True)
    assert heights[0] == heights[1] and heights[0] in times
    Q = [synth.spod_bin_torch(N, Nb, 40 + i, device="cuda").t() for i, (N, Nb) in enumerate(zip(Ns, Nbs))]
    b = pg.BatchedSVD(Q, kmodes=4, prec=prec, leaf_rows=heights)
    hmax = pg.batched_max_leaf_rows(prec)
    for f, N in enumerate(Ns):
        assert b.info(f, 0) == heights[f]                       # the height the plan runs
        # and its leaf count: floor(N / h) leaves, more if the longest would exceed the cap
        assert b.info(f, 1) == max(1, N // heights[f], -(-N // hmax))
    b.run()
    assert b.status() == pg.OK


def test_pod_candidates_are_whole_waves():
    # 4,194,304 x 256: 152, 304, 456, 608 leaves (FP64), 152 and 304 (mixed)
    c = tune.pod_candidates(1 << 22, 256, pg.PREC_FP64, sms=152)
    assert c == [(1 << 22) // (k * 152) for k in (1, 2, 3, 4)]
    assert tune.pod_candidates(1 << 22, 256, pg.PREC_MIXED_3XTF32, sms=152) == c[:2]
    # leaves never below max(M, 1024) rows
    assert all(b >= 1808 for b in tune.pod_candidates(10_000_000, 1808, pg.PREC_FP64, sms=152))
    assert tune.pod_candidates(100_000, 256, pg.PREC_FP64, sms=152) == []


def test_pod_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "c.json"))
    monkeypatch.setattr(tune, "gpu_name", lambda: "cpu")
    assert tune.pod_leaf_rows_for(1 << 22, 256, pg.PREC_FP64, tune=False) == 0
    tune._save({"cpu|pod|prec0|N4194304|M256": 13797})
    assert tune.pod_leaf_rows_for(1 << 22, 256, pg.PREC_FP64, tune=False) == 13797


@pytest.mark.gpu
def test_pod_tuner_picks_fastest_and_result_holds(tmp_path, monkeypatch):
    torch = pytest.importorskip("torch")
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    N, M = 1 << 19, 64
    best, times = tune.tune_pod(N, M, pg.PREC_FP64)
    assert times and times[best] == min(times.values())
    assert tune.pod_leaf_rows_for(N, M, pg.PREC_FP64, tune=True) in times
    assert pg.leaf_count(N, M, best) == N // best


@pytest.mark.gpu
def test_batched_workload_tuner_picks_fastest_policy():
    torch = pytest.importorskip("torch")
    import synth
    Ns, Nbs = [30000, 9000, 70000], [40, 100, 17]
    Q = [synth.spod_bin_torch(N, Nb, 60 + i, device="cuda").t() for i, (N, Nb) in enumerate(zip(Ns, Nbs))]
    heights, times = tune.tune_batched_workload(Q, 4, pg.PREC_MIXED_3XTF32)
    assert "built-in" in times and len(times) >= 2
    best = min(times, key=times.get)
    expect = [0] * 3 if best == "built-in" else [max(int(best.split()[1]), nb) for nb in Nbs]
    assert heights == expect
    b = pg.BatchedSVD(Q, kmodes=4, prec=pg.PREC_MIXED_3XTF32, leaf_rows=heights)
    b.run()
    assert b.status() == pg.OK
