"""Autotuner of the TSQR leaf heights.

Batched complex SVD (SPOD bins and windows): the leaf height trades the leaf
QR's memory traffic (a taller leaf streams its trailing columns from HBM once
per reflector) against the binary64 tree (P - 1 merges of (8/3) Nb^3 real
flops each).  For every (Nb class, N class) the tuner times a small batch of
seeded sample bins with each candidate height through the library's own
batched launch and keeps the fastest.  Those per-class heights are tuned
on a few bins at a time; inside a full launch of hundreds of bins the device
is already busy and shorter leaves mostly add tree merges (on the 256-bin
SPOD workload the per-class heights ran 2.80 s against 2.00 s for the
built-in choice), so `tune_batched_workload` chooses among whole-batch
policies timed on the batch itself, and the benchmark uses it.

POD (pylom_pod): the leaf count P trades the leaves' parallelism (one or two
thread blocks per SM) and their panel latency against the tree's (P - 1)
(2/3) M^3 binary64 flops.  For an (N, M, precision) the tuner times the POD
of a seeded known-spectrum matrix of that shape at each candidate leaf count
(whole multiples of the SM count, so every wave of leaves fills the GPU)
and keeps the fastest leaf height.

Results are cached in JSON, keyed by GPU name, precision and class; the cache
file is a runtime artifact (PYLOM_TUNE_CACHE overrides its path).
"""
from __future__ import annotations

import json
import math
import os
import time

import paper_2405_15529_gb300 as pg

_HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("PYLOM_TUNE_CACHE", os.path.join(_HERE, "tune_cache.json"))


def _classes(N: int, Nb: int):
    nb_c = 1 << max(0, math.ceil(math.log2(max(Nb, 1))))
    n_c = int(math.floor(math.log2(max(N, 1))))
    return nb_c, n_c


def _key(gpu: str, prec: int, nb_c: int, n_c: int) -> str:
    return f"{gpu}|prec{prec}|nb{nb_c}|n2^{n_c}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(d):
    tmp = CACHE + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def set_cache_path(path: str) -> None:
    """Where the cache lives (default: tune_cache.json beside this file, or
    $PYLOM_TUNE_CACHE)."""
    global CACHE
    CACHE = path


CANDIDATE_ROWS = (256, 384, 512, 768, 1024)


def candidates(N: int, Nb: int, max_leaf_rows: int):
    """Distinct leaf heights worth timing for an N x Nb bin: at least Nb
    rows, at most N, and at most the longest leaf the library runs at this
    precision (it splits taller hints into more leaves, which would time an
    already listed configuration again)."""
    c = sorted({max(Nb, h) for h in CANDIDATE_ROWS})
    return [h for h in c if h <= N and h <= max_leaf_rows]


def time_leaf_rows(N: int, Nb: int, prec: int, h: int, nbins: int = 4, reps: int = 3, seed: int = 0) -> float:
    """Median seconds of one batched run over `nbins` seeded N x Nb bins."""
    import torch
    import synth
    Q = [synth.spod_bin_torch(N, Nb, seed + i, device="cuda").t() for i in range(nbins)]
    b = pg.BatchedSVD(Q, kmodes=min(8, Nb), prec=prec, leaf_rows=[h] * nbins)
    b.run()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.run()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    st = b.status()
    if st != pg.OK:
        raise pg.PylomError(st, "autotuner sample run")
    ts.sort()
    return ts[len(ts) // 2]


def tune_class(N: int, Nb: int, prec: int):
    """Times every candidate height on sample bins of this class; returns
    (fastest height, {height: median seconds})."""
    times = {}
    for h in candidates(N, Nb, pg.batched_max_leaf_rows(prec)):
        times[h] = time_leaf_rows(N, Nb, prec, h)
    best = min(times, key=lambda h: (times[h], h))
    return best, times


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"


def leaf_rows_for(Ns, Nbs, prec: int, tune: bool = False):
    """Leaf heights for a batch (from the cache; missing classes are tuned
    when `tune`, else left to the library's built-in choice, 0)."""
    gpu = gpu_name()
    cache = _load()
    out = []
    dirty = False
    for N, Nb in zip(Ns, Nbs):
        nb_c, n_c = _classes(int(N), int(Nb))
        k = _key(gpu, prec, nb_c, n_c)
        if k not in cache and tune:
            cache[k] = tune_class(1 << n_c, nb_c, prec)[0]
            dirty = True
        h = int(cache.get(k, 0))
        out.append(max(h, int(Nb)) if h else 0)
    if dirty:
        _save(cache)
    return out


def tune_batched_workload(Q, kmodes: int, prec: int, heights=(512, 768, 1024), reps: int = 1):
    """Leaf heights for a whole batch, chosen on the batch itself.

    A height that wins for a few bins of one size class can lose inside the
    full persistent launch: with hundreds of bins the device is already
    full, and shorter leaves only add binary64 tree merges.  So the policies
    are timed on the actual bins, one launch each: the library's built-in
    choice and one height for every bin (each of `heights`, at least the
    bin's columns, at most the longest leaf of the precision).  Returns
    (per-bin heights of the fastest policy, 0 = built-in; {policy: seconds})."""
    import torch
    hmax = pg.batched_max_leaf_rows(prec)
    Nbs = [int(q.shape[1]) for q in Q]
    policies = {"built-in": [0] * len(Q)}
    for h in heights:
        if h <= hmax:
            policies[f"all {h}"] = [max(h, nb) for nb in Nbs]
    times = {}
    for name, lr in policies.items():
        b = pg.BatchedSVD(Q, kmodes=kmodes, prec=prec, leaf_rows=lr)
        b.run()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            b.run()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        st = b.status()
        if st != pg.OK:
            raise pg.PylomError(st, f"autotuner batch run ({name})")
        times[name] = min(ts)
        del b
        torch.cuda.empty_cache()
    best = min(times, key=times.get)
    return policies[best], times


# ---------------------------------------------------------------------------
# POD leaf heights
# ---------------------------------------------------------------------------

def pod_candidates(N: int, M: int, prec: int, sms: int = 152):
    """Leaf heights whose leaf counts are 1, 2, 3 or 4 thread blocks per SM
    (the mixed path holds one block per SM at a time, so its counts stay
    whole waves of one block per SM), keeping >= max(M, 1024) rows a leaf."""
    per = (1, 2, 3, 4) if prec == pg.PREC_FP64 else (1, 2)
    out = []
    for k in per:
        P = k * sms
        b = N // P
        if b >= max(M, 1024) and b not in out:
            out.append(b)
    return out


def time_pod(N: int, M: int, prec: int, leaf_rows: int, reps: int = 3, seed: int = 0) -> float:
    """Median seconds of pylom_pod on a seeded N x M known-spectrum matrix."""
    import torch
    import synth
    dt = torch.float64 if prec == pg.PREC_FP64 else torch.float32
    XT, w, _ = synth.known_spectrum_torch(N, M, device="cuda", dtype=dt, seeds=(2 + seed, 3, 4))
    X = XT.t()
    ws = torch.empty(pg.pod_workspace_size(N, M, leaf_rows, M, pg.F64 if dt == torch.float64 else pg.F32, prec),
                     dtype=torch.uint8, device="cuda")
    res = pg.pod(X, w=w, remove_mean=False, energy=0.99, leaf_rows=leaf_rows, prec=prec, workspace=ws)
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        pg.pod(X, w=w, remove_mean=False, energy=0.99, leaf_rows=leaf_rows, prec=prec, workspace=ws, check=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    st, _, _ = pg.workspace_status(ws)
    if st != pg.OK:
        raise pg.PylomError(st, "autotuner POD run")
    del X, XT, ws, res
    torch.cuda.empty_cache()
    ts.sort()
    return ts[len(ts) // 2]


def tune_pod(N: int, M: int, prec: int, sms: int = None):
    """Times every candidate leaf height; returns (fastest height, {height: s})."""
    import torch
    if sms is None:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    times = {b: time_pod(N, M, prec, b) for b in pod_candidates(N, M, prec, sms)}
    if not times:
        return 0, times      # too few rows for a full wave of leaves: the automatic choice
    best = min(times, key=lambda b: (times[b], b))
    return best, times


def pod_leaf_rows_for(N: int, M: int, prec: int, tune: bool = False) -> int:
    """The cached leaf height for this (N, M, precision) -- tuned first when
    `tune` and not cached -- or 0 (the library's automatic choice)."""
    key = f"{gpu_name()}|pod|prec{prec}|N{N}|M{M}"
    cache = _load()
    if key not in cache and tune:
        cache[key] = tune_pod(N, M, prec)[0]
        _save(cache)
    return int(cache.get(key, 0))
