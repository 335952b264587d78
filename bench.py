#!/usr/bin/env python
"""Benchmark of the POD hot path: GB/s of the snapshot matrix X processed.

Workload (default): the 4,194,304 x 256 binary64 known-spectrum snapshot
matrix X = diag(w)^(-1/2) Q1 diag(s) Q2^T with s_i = 10^(-6 i / 255) and
log-uniform cell volumes w in [1e-3, 1]; POD without mean removal, weights
on, truncated at 99 % cumulative energy (r = 43).  One step = one full
pylom_pod call (leaf QR + tree + small SVD + top-down pass + modes).

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "POD GB/s of X processed"
# DRAM bytes (read + write) of one leaf_qr_kernel launch on the 4,194,304 x 256
# workload (304 leaves), from a one-pass ncu capture of that launch inside
# this benchmark (dram__bytes_read.sum + dram__bytes_write.sum); see the
# profile summary of the FP64 path.
LEAF_FP64_TRAFFIC_BYTES = 345.47e9 + 153.50e9
LEAF_FP64_TRAFFIC_SOURCE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum -k regex:leaf_qr_kernel, "
                            "full-size launch (1 pass), profiles/pod_fp64_known_spectrum_4194304x256.md")
N_FULL, M_FULL, ENERGY = 1 << 22, 256, 0.99
WORKLOAD = "known_spectrum_4194304x256_f64_weighted_energy0.99"


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


_PROBE = None


def probe_peak(kind: str) -> float:
    """Measured TFLOP/s of this GPU from the benchmark's own probes
    (bench_probe.cu): 'mma' binary64 mma.sync.m8n8k4, 'fma' binary64 FMA,
    'ffma' binary32 FMA."""
    import ctypes
    import torch
    global _PROBE
    if _PROBE is None:
        from paper_2405_15529_gb300 import _build
        lib = ctypes.CDLL(_build.build_probe())
        lib.bench_probe_scratch_bytes.restype = ctypes.c_size_t
        lib.bench_probe_peak.restype = ctypes.c_int
        lib.bench_probe_peak.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p]
        _PROBE = lib
    scratch = torch.empty(_PROBE.bench_probe_scratch_bytes(), dtype=torch.uint8, device="cuda")
    out = ctypes.c_double(0.0)
    rc = _PROBE.bench_probe_peak({"mma": 0, "fma": 1, "ffma": 2}[kind], ctypes.c_void_p(scratch.data_ptr()),
                                 ctypes.byref(out), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError(f"bench_probe_peak({kind}) failed with code {rc}")
    return float(out.value)


def rank_max(value: float, device=None) -> float:
    """Max of a per-rank time over the job's ranks (the slowest rank sets the
    step time); the value itself on a single process."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbs(bytes_per_rank: float, ms: float, world: int) -> float:
    """Whole-job throughput: every rank processes its own bytes_per_rank in ms."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def cpu_baseline(n_rows: int, M: int, seed_shift: int = 0, X=None, w=None):
    """The FP64 oracle, as it stands, on the workload: on the given host
    matrix X (N x M, with weights w) when passed -- the full workload -- else
    on a freshly generated row sample of it.
    Returns (GB/s of X, seconds, threads, sample description)."""
    import numpy as np
    import oracle
    import synth
    if X is None:
        X, w, s = synth.known_spectrum(n_rows, M, weights=True, seeds=(2 + seed_shift, 3, 4))
        what = f"a {n_rows} x {M} row sample of the workload (same spectrum, weights, energy {ENERGY})"
    else:
        n_rows = X.shape[0]
        what = f"the full {n_rows} x {M} workload (the same X and weights the GPU step reads, energy {ENERGY})"
    t0 = time.perf_counter()
    res = oracle.pod(X, w=w, remove_mean=False, energy=ENERGY)
    dt = time.perf_counter() - t0
    gbs = n_rows * M * 8 / dt / 1e9
    desc = f"oracle.pod on {what}; r={res['r']}; one run"
    return gbs, dt, oracle.num_threads(), desc


def fp64_matmul_tflops(dev, n=4096, reps=3):
    """TFLOP/s of the library's binary64 product (pylom_matmul, the FP64
    tensor pipe) on an n x n x n problem whose flops are known (2 n^3): a
    cross-check of the probe's FP64 peak by a kernel doing real work."""
    import torch
    import paper_2405_15529_gb300 as pg
    g = torch.Generator(device=dev).manual_seed(9)
    A = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    B = torch.randn((n, n), dtype=torch.float64, device=dev, generator=g)
    pg.matmul(A, B)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        C = pg.matmul(A, B)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del A, B, C
    torch.cuda.empty_cache()
    return best


def h2d_sweep(Xh, dev, sizes_mb=(64, 512, 2048), chunk_mb=256):
    """Host-to-device copy rate from the page-locked buffer Xh at several
    sizes, as one copy and as a train of chunk_mb copies on a side stream
    (diagnostics of the end-to-end upload; not part of any timed step)."""
    import torch
    flat = Xh.view(-1).view(torch.uint8)
    total = flat.numel()
    dst = torch.empty(total, dtype=torch.uint8, device=dev)
    out = {}
    side = torch.cuda.Stream(device=dev)

    def rate(nbytes, chunked):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(side):
            ev0.record(side)
            if chunked:
                step = chunk_mb << 20
                for o in range(0, nbytes, step):
                    e = min(nbytes, o + step)
                    dst[o:e].copy_(flat[o:e], non_blocking=True)
            else:
                dst[:nbytes].copy_(flat[:nbytes], non_blocking=True)
            ev1.record(side)
        ev1.synchronize()
        return nbytes / (ev0.elapsed_time(ev1) * 1e-3) / 1e9

    for mb in list(sizes_mb) + [total >> 20]:
        nb = min(total, mb << 20)
        rate(nb, False)                     # warm
        out[f"{nb >> 20}MB_one_copy_gbs"] = rate(nb, False)
        out[f"{nb >> 20}MB_{chunk_mb}MB_chunks_gbs"] = rate(nb, True)
    # the library's chunked upload on the current stream, as the timed step issues it
    import paper_2405_15529_gb300 as pg
    for rep in range(2):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        pg.upload(dst, flat)
        ev1.record()
        ev1.synchronize()
        out[f"pg_upload_current_stream_gbs_{rep}"] = total / (ev0.elapsed_time(ev1) * 1e-3) / 1e9
    del dst
    torch.cuda.empty_cache()
    return out


def gpu_numa_info(local_rank):
    """Where the GPU and this process sit (sysfs), recorded beside the
    end-to-end number."""
    info = {}
    try:
        import torch
        p = torch.cuda.get_device_properties(local_rank)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        info["pci"] = bus
        for key in ("numa_node", "local_cpulist"):
            try:
                with open(f"/sys/bus/pci/devices/{bus}/{key}") as f:
                    info[key] = f.read().strip()
            except OSError:
                pass
    except Exception as exc:  # noqa: BLE001 - diagnostics only
        info["error"] = str(exc)[:200]
    try:
        info["process_cpus"] = len(os.sched_getaffinity(0))
    except OSError:
        pass
    return info


def bench_adjoint(args, dev):
    """Forward + hand-written backward of the truncated-POD reconstruction
    loss on the 4,194,304 x 256 float32 known-spectrum matrix, r = 20: timed
    on the mixed-precision path (FP32 modes, 3xTF32 products on tcgen05,
    binary64 tree passes and square SVD adjoint) and, for comparison, on the
    binary64 path."""
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, M, r = N_FULL, M_FULL, 20
    XT, w, s = synth.known_spectrum_torch(N, M, device=dev, dtype=torch.float32)
    X = XT.t()

    def loss(Xg, U):
        Yw = Xg.double() * torch.sqrt(w)[:, None]
        Ud = U.double()
        return torch.sum((Yw - Ud @ (Ud.T @ Yw)) ** 2)

    def run(prec, steps, warmup):
        def step():
            Xg = X.detach().requires_grad_(True)
            U, S, VT = pg.pod_autograd(Xg, r, w=w, prec=prec)
            loss(Xg, U).backward()
            return Xg.grad, U

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            G, U = step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        with torch.no_grad():
            Ud = U.double()
            Yw = X.double() * torch.sqrt(w)[:, None]
            Gc = 2.0 * torch.sqrt(w)[:, None] * (Yw - Ud @ (Ud.T @ Yw))
            rel = (torch.linalg.norm(G.double() - Gc) / torch.linalg.norm(Gc)).item()
        del G, U, Ud, Yw, Gc
        torch.cuda.empty_cache()
        return ms, rel

    ms, rel = run(pg.PREC_MIXED_3XTF32, args.adj_steps, max(1, args.warmup - 2))
    ms64, rel64 = run(pg.PREC_FP64, 1, 1)
    out = {"workload": "known_spectrum_4194304x256_f32_weighted_r20_loss_grad", "ms_per_step": ms,
           "value": N * M * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s of X (forward + backward)",
           "steps": args.adj_steps, "precision": "mixed (3xTF32 tcgen05; binary64 tree and square SVD adjoint)",
           "grad_rel_err_vs_closed_form": rel,
           "fp64_path_ms_same_x": ms64, "fp64_path_grad_rel_err_vs_closed_form": rel64,
           "speedup_vs_fp64_path": ms64 / ms,
           "note": "step = pylom_pod forward (check) + torch loss + pylom_pod_backward"}
    del X, XT, w
    torch.cuda.empty_cache()
    return out


def bench_mixed(args, dev):
    """The 4,194,304 x 256 float32 known-spectrum matrix through the mixed
    path (FP32 leaves, 3xTF32 block reflectors on tcgen05, FP64 tree and
    SVD) and, once, through the FP64 path on the same X."""
    import numpy as np
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, M = args.rows, M_FULL
    XT, w, s = synth.known_spectrum_torch(N, M, device=dev, dtype=torch.float32)
    X = XT.t()
    prec = pg.PREC_MIXED_3XTF32
    leaf = 0
    if args.tune:
        from paper_2405_15529_gb300 import tune
        leaf = tune.pod_leaf_rows_for(N, M, prec, tune=True)
    ws = torch.empty(pg.pod_workspace_size(N, M, leaf, M, pg.F32, prec), dtype=torch.uint8, device=dev)
    U = pg.empty_colmajor(N, M, torch.float32, dev)
    S = torch.empty(M, dtype=torch.float64, device=dev)
    VT = pg.empty_colmajor(M, M, torch.float64, dev)
    r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    out = (U, S, VT, None, r_dev)

    def step():
        pg.pod(X, w=w, remove_mean=False, energy=ENERGY, r_max=M, prec=prec, leaf_rows=leaf, workspace=ws, out=out,
               check=False)

    for _ in range(args.warmup):
        step()
    st, r, sweeps = pg.workspace_status(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pg.profile_begin(args.steps)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    phases, n = pg.profile_end()
    ms = e0.elapsed_time(e1) / args.steps
    S_mix = S.cpu().numpy()
    ref = pg.pod(X, w=w, remove_mean=False, energy=ENERGY)
    t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    ref = pg.pod(X, w=w, remove_mean=False, energy=ENERGY)
    t1.record()
    torch.cuda.synchronize()
    ms64 = t0.elapsed_time(t1)
    S64 = ref.S.cpu().numpy()
    leaf_ms = phases["leaf_qr"] / max(n, 1)
    out = {"workload": f"known_spectrum_{N}x{M}_f32_weighted_energy0.99", "status": st, "r": r,
           "leaf_rows": leaf, "leaves": pg.leaf_count(N, M, leaf) if leaf else min(152, pg.leaf_count(N, M, 0)),
           "ms_per_step": ms, "value": N * M * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s of X (float32)",
           "phases_ms_per_step": {k: v / max(n, 1) for k, v in phases.items()},
           "fp64_path_ms_same_x": ms64, "speedup_vs_fp64_path": ms64 / ms,
           "sigma_max_abs_diff_vs_fp64_path_over_smax": float(np.max(np.abs(S_mix - S64)) / S64[0]),
           "sigma_max_abs_err_vs_closed_form_over_smax": float(np.max(np.abs(S_mix - s)) / s[0]),
           "leaf_kernel": {"kernel": "leaf_qr_mixed_kernel (FP32 panels + 3xTF32 tcgen05 trailing updates)",
                           "ms_per_launch": leaf_ms,
                           "useful_tflops": 2.0 * N * M * M / (leaf_ms * 1e-3) / 1e12}}
    del X, XT, w, ws, U, S, VT, r_dev, ref
    torch.cuda.empty_cache()
    return out


def bench_spod_end_to_end(args, dev):
    """The whole SPOD of one snapshot matrix (Sec. 2.3, Alg. 6) as one CUDA
    graph: 2^20 points x 4128 instants (float32, 17.3 GB; wave field),
    windows of 64 instants overlapping by 32 (128 blocks, 33 frequencies),
    the front end, the 33 complex64 SVDs (1,048,576 x 128 each) in one
    persistent launch, and the order of the frequencies."""
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, T, npwin, nolap = 1 << 20, 4128, 64, 32
    XT = synth.waves_torch(N, T, 8, "geometric", 1e-3, 12, dev, dtype=torch.float32, row_chunk=1 << 18)
    D = XT.t()
    sp = pg.SPOD(D, 0.2, npwin, nolap, remove_mean=True, kmodes=8)
    sp.capture()
    for _ in range(max(1, args.warmup - 2)):
        sp.replay()
    torch.cuda.synchronize()
    steps = args.spod_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        sp.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = sp.status()
    # the front end alone (its own launches, same buffers)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(steps):
        pg.spod_blocks(D, npwin, nolap, True, Q=sp.Q, workspace=sp.ws)
    f1.record()
    torch.cuda.synchronize()
    fms = f0.elapsed_time(f1) / steps
    hbm = 6800.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            hbm = json.load(fh).get("hbm_gbs", hbm)
    except (OSError, ValueError):
        pass
    front_bytes = N * T * 4 + sp.nfreq * sp.nblks * N * 8       # read D once, write every Q_f
    order = sp.order[:4].cpu().tolist()
    out = {"workload": f"spod_waves8_{N}x{T}_f32_npwin{npwin}_nolap{nolap}", "ms_per_step": ms, "steps": steps,
           "value": N * T * 4 / (ms * 1e-3) / 1e9, "unit": "GB/s of snapshots (front end + SVDs + order)",
           "graph": "captured (front end + batched SVD launch + order)", "status": st,
           "blocks": sp.nblks, "frequencies": sp.nfreq, "leading_frequencies": order,
           "front_end": {"ms": fms, "algorithmic_bytes": front_bytes,
                         "achieved_gbs": front_bytes / (fms * 1e-3) / 1e9, "hbm_peak_gbs": hbm,
                         "frac": front_bytes / (fms * 1e-3) / 1e9 / hbm,
                         "kernel": "spod_dft_tc_kernel<float> (window and scaling folded into a 64 x 80 DFT matrix; 3xTF32 on tcgen05)"}}
    del sp, D, XT
    torch.cuda.empty_cache()
    return out


def bench_dmd(args, dev):
    """Exact DMD (Sec. 3.2, Algs. 3-5) of a 4,194,304 x 256 float64 field of
    24 damped / neutral oscillations (rank 48, |lambda| in [0.985, 1]) plus
    1e-5 noise (8.6 GB), r_max = 48, no mean removal (the field is a pure
    Krylov sequence, so its DMD has a closed form).  Timed with CUDA events;
    the eigenvalues are checked against the construction's lambda_k and the
    products mode x amplitude against a_k psi_k / 2 on the first rows."""
    import numpy as np
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, M, K = args.rows, M_FULL, 24
    lam, amp = synth.oscillation_params(K, seed=21)
    XT, psi_chunk = synth.oscillations_torch(N, M, lam, amp, seed=22, device=dev, noise=1e-5)
    X = XT.t()
    r_max = 2 * K
    res = pg.dmd(X, remove_mean=False, r_max=r_max)
    ws = res.workspace
    mu = torch.empty(2 * r_max, dtype=torch.float64, device=dev)
    b = torch.empty_like(mu)
    Phi = pg.empty_colmajor(N, r_max, torch.float64, dev)
    S = torch.empty(M - 1, dtype=torch.float64, device=dev)
    mean = torch.empty(N, dtype=torch.float64, device=dev)
    r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    out = (mu, b, Phi, S, mean, r_dev)
    for _ in range(max(1, args.warmup - 1)):
        pg.dmd(X, remove_mean=False, r_max=r_max, workspace=ws, out=out, check=False)
    torch.cuda.synchronize()
    steps = args.dmd_steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        pg.dmd(X, remove_mean=False, r_max=r_max, workspace=ws, out=out, check=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st, r, _ = pg.workspace_status(ws)
    res = pg.DmdResult(mu=torch.view_as_complex(mu.view(-1, 2))[:r], b=torch.view_as_complex(b.view(-1, 2))[:r],
                       Phi_packed=Phi[:, :r], S=S, mean=mean, r=r, workspace=ws)
    muc = res.mu.cpu().numpy()
    lam_all = np.concatenate([lam, np.conj(lam)])
    mu_err = float(max(np.min(np.abs(muc - l)) for l in lam_all)) if r == r_max else None
    # mode x amplitude on the first 4096 rows vs a_k psi_k / 2
    rows = 4096
    pr, pi, _ = psi_chunk(0, min(N, 1 << 21))
    psi = (pr[:rows] + 1j * pi[:rows]).cpu().numpy()
    pb = (res.Phi[:rows] * res.b[None, :]).cpu().numpy()
    pb_err = 0.0
    for k in range(K):
        i = int(np.argmin(np.abs(muc - lam[k])))
        part = amp[k] * psi[:, k] / 2.0
        pb_err = max(pb_err, float(np.linalg.norm(pb[:, i] - part) / np.linalg.norm(part)))
    out_d = {"workload": f"dmd_oscillations24_{N}x{M}_f64_noise1e-5", "ms_per_step": ms, "steps": steps,
             "value": N * M * 8 / (ms * 1e-3) / 1e9, "unit": "GB/s of snapshots", "status": st, "r": r,
             "max_abs_eig_err_vs_construction": mu_err,
             "max_rel_mode_times_amplitude_err_first_4096_rows": pb_err,
             "path": "one TSQR of Y (leaf QR + tree), SVD of R[:M-1,:M-1], small DMD kernels "
                     "(Hessenberg + Francis QR, Cholesky amplitudes), modes = Q [B; 0]"}
    del X, XT, ws, Phi, res, out
    torch.cuda.empty_cache()
    return out_d


def bench_streamed(args, dev):
    """The out-of-core POD: the 4,194,304 x 256 known-spectrum matrix (float64,
    8.6 GB) held in page-locked HOST memory and streamed through the device in
    chunks of 304 leaves (about --stream-chunk rows); the modes return to host
    memory.  Timed end to end (host to host) beside the in-core call with the
    same leaf partition on a device-resident copy; the results must agree bit
    for bit."""
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, M, chunk = args.rows, M_FULL, args.stream_chunk
    XT, w, s = synth.known_spectrum_torch(N, M, device=dev)
    b = pg.pod_streamed_leaf_rows(N, M, 0, chunk)
    Xh = torch.empty((M, N), dtype=torch.float64, pin_memory=True)
    Xh.copy_(XT)
    Xh = Xh.t()
    wh = w.cpu().reshape(-1, 1).pin_memory()      # N x 1: used in place (no per-call copy)
    ref = pg.pod(XT.t(), w=w, remove_mean=False, energy=ENERGY, leaf_rows=b)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.stream_steps):
        ref = pg.pod(XT.t(), w=w, remove_mean=False, energy=ENERGY, leaf_rows=b, workspace=ref.workspace)
    torch.cuda.synchronize()
    ms_in = (time.perf_counter() - t0) * 1e3 / args.stream_steps
    S_ref, U_ref, r_ref = ref.S.clone(), ref.U.cpu(), ref.r
    del ref, XT
    torch.cuda.empty_cache()
    Yh = torch.empty(N * M, dtype=torch.float64, pin_memory=True)
    Uh = torch.empty((M, N), dtype=torch.float64, pin_memory=True).t()
    res = pg.pod_streamed(Xh, w=wh, remove_mean=False, energy=ENERGY, leaf_rows=0, chunk_rows=chunk,
                          host_scratch=Yh, out=Uh)
    ws = res.workspace
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.stream_steps):
        res = pg.pod_streamed(Xh, w=wh, remove_mean=False, energy=ENERGY, leaf_rows=0, chunk_rows=chunk,
                              workspace=ws, host_scratch=Yh, out=Uh)
    ms = (time.perf_counter() - t0) * 1e3 / args.stream_steps
    equal = bool(res.r == r_ref and torch.equal(res.S, S_ref) and torch.equal(res.U, U_ref))
    # the host link alone: one 2 GiB page-locked copy each way
    hb = torch.empty(1 << 28, dtype=torch.float64, pin_memory=True)
    db = torch.empty(1 << 28, dtype=torch.float64, device=dev)
    link_gbs = {}
    for name, dst, src in (("h2d", db, hb), ("d2h", hb, db)):
        dst.copy_(src, non_blocking=True)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record()
        dst.copy_(src, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        link_gbs[name] = hb.numel() * 8 / (c0.elapsed_time(c1) * 1e-3) / 1e9
    del hb, db
    P = pg.leaf_count(N, M, b)
    link = N * M * 8 * 3 + N * res.r * 8 + N * 8     # X up, reflectors down and up, modes down, weights
    out = {"workload": f"pod_known_spectrum_{N}x{M}_f64_host_resident", "ms_per_step": ms,
           "steps": args.stream_steps, "value": N * M * 8 / (ms * 1e-3) / 1e9,
           "unit": "GB/s of snapshots, host to host", "leaf_rows": b, "leaves": P,
           "leaves_per_chunk": 304, "chunks": -(-P // 304), "device_workspace_gb": ws.numel() / 1e9,
           "host_link_bytes_per_step": link, "host_link_gbs": link / (ms * 1e-3) / 1e9,
           "link_copy_gbs_measured": link_gbs,
           "bound_ms": max(ms_in, (N * M * 8 * 2 + N * res.r * 8) / (link_gbs["d2h"] * 1e9) * 1e3,
                           N * M * 8 * 2 / (link_gbs["h2d"] * 1e9) * 1e3),
           "in_core_same_partition_ms": ms_in, "streamed_over_in_core": ms / ms_in,
           "r": res.r, "bitwise_equal_to_in_core": equal}
    del res, ws, Xh, wh, Yh, Uh
    torch.cuda.empty_cache()
    return out


C3_N, C3_M, C3_RMAX = 10_000_000, 1808, 128


def c3_cpu_baseline(N, M, rmax, rows=(8192, 16384)):
    """The FP64 oracle on row samples of the 1808-column wave field, as it
    stands: the POD of each sample is timed whole, its time fitted as
    a + b * rows (the QR and modes grow with the rows, the Jacobi SVD of the
    1808 x 1808 R does not) and extrapolated to N rows.  Minutes of CPU."""
    import oracle
    import synth
    ts = []
    for n in rows:
        X = synth.waves(n, M, n_waves=64, amp="powerlaw", noise=1e-4, seed=5)
        t0 = time.perf_counter()
        oracle.pod(X, remove_mean=True, energy=ENERGY, r_max=rmax)
        ts.append(time.perf_counter() - t0)
    b = (ts[1] - ts[0]) / (rows[1] - rows[0])
    a = ts[0] - b * rows[0]
    t_full = a + b * N
    return {"value": N * M * 4 / t_full / 1e9, "unit": "GB/s of X (float32)", "cores": oracle.num_threads(),
            "kind": "oracle", "extrapolated": True, "seconds_full_size": t_full,
            "sample": f"oracle.pod on {rows[0]} and {rows[1]} x {M} samples of the wave field "
                      f"({ts[0]:.1f} s, {ts[1]:.1f} s), fitted as a + b*rows and extrapolated linearly in "
                      f"rows to {N}"}


def bench_waves_1808(args, dev):
    """The 10,000,000 x 1808 float32 wake-like field (64 traveling waves,
    power-law amplitudes, noise 1e-4; 72.3 GB) through the mixed path, timed,
    and once through the FP64 path on the same X (the reference its accuracy
    and speed are stated against).  99 % energy, at most 128 modes."""
    import numpy as np
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    N, M, rmax = args.c3_rows, C3_M, C3_RMAX
    XT = synth.waves_torch(N, M, 64, "powerlaw", 1e-4, 5, dev, dtype=torch.float32, row_chunk=1 << 18)
    X = XT.t()
    a, _, _ = synth.wave_params(64, "powerlaw")
    s_cf = np.repeat(a * math.sqrt(N * M) / 2.0, 2)          # noise-free closed form (pairs)
    noise_bound = 1e-4 * (math.sqrt(N) + math.sqrt(M))       # ~ ||noise||_2 (Weyl)

    def run(prec, steps, warmup):
        ws = torch.empty(pg.pod_workspace_size(N, M, 0, rmax, pg.F32, prec), dtype=torch.uint8, device=dev)
        U = pg.empty_colmajor(N, rmax, torch.float32 if prec == pg.PREC_MIXED_3XTF32 else torch.float64, dev)
        S = torch.empty(M, dtype=torch.float64, device=dev)
        VT = pg.empty_colmajor(M, M, torch.float64, dev)
        mean = torch.empty(N, dtype=torch.float64, device=dev)
        r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
        out = (U, S, VT, mean, r_dev)
        for _ in range(warmup):
            pg.pod(X, remove_mean=True, energy=ENERGY, r_max=rmax, prec=prec, workspace=ws, out=out, check=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pg.profile_begin(steps)
        e0.record()
        for _ in range(steps):
            pg.pod(X, remove_mean=True, energy=ENERGY, r_max=rmax, prec=prec, workspace=ws, out=out, check=False)
        e1.record()
        torch.cuda.synchronize()
        phases, n = pg.profile_end()
        st, r, sweeps = pg.workspace_status(ws)
        res = {"ms": e0.elapsed_time(e1) / steps, "status": st, "r": r, "sweeps": sweeps,
               "phases_ms": {k: v / max(n, 1) for k, v in phases.items()}, "S": S.cpu().numpy()}
        del ws, VT, mean, r_dev, S
        torch.cuda.empty_cache()
        return res, U

    mix, Umix = run(pg.PREC_MIXED_3XTF32, args.c3_steps, 1)
    f64, U64 = run(pg.PREC_FP64, 1, 0)
    r = min(mix["r"], f64["r"])
    G = torch.zeros((r, r), dtype=torch.float64, device=dev)
    for r0 in range(0, N, 1 << 20):
        G += Umix[r0:r0 + (1 << 20), :r].double().T @ U64[r0:r0 + (1 << 20), :r]
    Gm = torch.zeros((r, r), dtype=torch.float64, device=dev)
    for r0 in range(0, N, 1 << 20):
        blk = Umix[r0:r0 + (1 << 20), :r].double()
        Gm += blk.T @ blk
    orth_mix = torch.linalg.norm(Gm - torch.eye(r, dtype=torch.float64, device=dev)).item()
    # overlap of each mixed mode (pair subspace where the pair is unresolved) with the FP64 path's
    Sm, S64 = mix["S"], f64["S"]
    Gn = G.cpu().numpy()
    worst = 1.0
    i = 0
    while i < r:
        j = i + 1
        while j < r and (S64[j - 1] - S64[j]) <= 1e-3 * S64[j - 1]:
            j += 1
        blk = Gn[i:j, i:j]
        v = abs(blk[0, 0]) if j - i == 1 else float(np.linalg.svd(blk, compute_uv=False).min())
        if S64[i] >= 1e-3 * S64[0]:
            worst = min(worst, v)
        i = j
    del Umix, U64, G, Gm, X, XT
    torch.cuda.empty_cache()
    bytes_x = N * M * 4
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    tf32_3x = peaks.get("bf16_tflops", 1900.0) * 0.5 / 3.0     # nominal tf32/bf16 = 1/2; three MMAs per product
    t_roof = max(bytes_x / (hbm * 1e9), 2.0 * N * M * M / (tf32_3x * 1e12))
    leaf_ms = mix["phases_ms"]["leaf_qr"]
    tree_ms = mix["phases_ms"]["tree"]
    # dominant kernel of the mixed step: the leaves (FP32 panels + 3xTF32
    # trailing updates, 2NM^2 - (2/3)PM^3 flops as three TF32 products); the
    # binary64 cooperative tree that follows is reported beside it
    P = pg.leaf_count(N, M, 0)
    P = min(P, 152) if P > 152 else P
    leaf_flops = 2.0 * N * M * M - (2.0 / 3.0) * P * M ** 3
    tree_flops = (P - 1) * (2.0 / 3.0) * M ** 3
    fp64_peak = probe_peak("mma")
    leaf_bytes = N * M * 4 + N * M * 4      # read X (FP32), write the FP32 reflectors
    t_leaf_roof = max(leaf_flops / (tf32_3x * 1e12), leaf_bytes / (hbm * 1e9))
    roofline = {"bound": "tensor", "achieved": leaf_flops / (leaf_ms * 1e-3) / 1e12, "peak": tf32_3x,
                "unit": "TFLOP/s", "frac": t_leaf_roof / (leaf_ms * 1e-3), "traffic": None,
                "kernel": "leaf_qr_mixed_kernel",
                "peak_source": "3xTF32 = measured bf16 burst x nominal tf32/bf16 (1/2) / 3",
                "algorithmic_flops_per_launch": leaf_flops, "algorithmic_bytes_per_launch": leaf_bytes,
                "ms_per_launch": leaf_ms, "leaves": P,
                "tree": {"kernel": "tree_coop_kernel (binary64)", "ms_per_launch": tree_ms,
                         "algorithmic_flops_per_launch": tree_flops, "peak_fp64_tflops": fp64_peak,
                         "frac": tree_flops / (fp64_peak * 1e12) / (tree_ms * 1e-3) if tree_ms > 0 else None}}
    cpu = {"skipped": "the oracle's unblocked QR and cyclic Jacobi at 1808 columns take minutes even on a "
                      "row sample; run bench.py --c3-cpu for the extrapolated figure"}
    if args.c3_cpu:
        cpu = c3_cpu_baseline(N, M, rmax)
    return {"workload": f"waves64_powerlaw_{N}x{M}_f32_mean_removed_energy0.99_rmax{rmax}",
            "status": [mix["status"], f64["status"]], "r": [mix["r"], f64["r"]],
            "ms_per_step": mix["ms"], "steps": args.c3_steps, "warmup": 1, "roofline": roofline,
            "cpu_baseline": cpu,
            "value": bytes_x / (mix["ms"] * 1e-3) / 1e9, "unit": "GB/s of X (float32)",
            "phases_ms_per_step": mix["phases_ms"], "jacobi_sweeps": mix["sweeps"],
            "fp64_path_ms_same_x": f64["ms"], "fp64_path_phases_ms": f64["phases_ms"],
            "speedup_vs_fp64_path": f64["ms"] / mix["ms"],
            "sigma_max_abs_diff_vs_fp64_path_over_smax": float(np.max(np.abs(Sm - S64)) / S64[0]),
            "sigma_wave_pairs_max_abs_err_vs_noise_free_closed_form_over_smax":
                float(np.max(np.abs(Sm[:128] - s_cf)) / s_cf[0]),
            "noise_weyl_bound_over_smax": noise_bound / s_cf[0],
            "min_mode_overlap_vs_fp64_path": worst, "mixed_U_orthonormality_fro": orth_mix,
            "pct_roofline": {"value": t_roof / (mix["ms"] * 1e-3),
                             "formula": "max(bytes_X/HBM_peak, 2NM^2/(tf32_peak/3)) / step time",
                             "tf32_peak_tflops": peaks.get("bf16_tflops", 1900.0) * 0.5,
                             "hbm_peak_gbs": hbm},
            "leaf_kernel": {"kernel": "leaf_qr_mixed_kernel", "ms_per_step": leaf_ms,
                            "useful_tflops": 2.0 * N * M * M / (leaf_ms * 1e-3) / 1e12}}


def bench_spod(args, dev):
    """All 256 SPOD bins (complex64, N_f log-uniform in [2^16, 2^20], Nb_f in
    [16, 128]) in one persistent launch captured in a CUDA graph."""
    import numpy as np
    import torch
    import paper_2405_15529_gb300 as pg
    from paper_2405_15529_gb300 import tune
    import synth
    Ns, Nbs = synth.spod_bin_sizes(args.spod_bins, seed=6)
    Q = [synth.spod_bin_torch(int(n), int(nb), seed=1000 + f, device=dev).t()
         for f, (n, nb) in enumerate(zip(Ns, Nbs))]
    torch.cuda.synchronize()
    prec = pg.PREC_MIXED_3XTF32
    t_tune = time.perf_counter()
    tune_times = None
    if args.tune:
        leaf_rows, tune_times = tune.tune_batched_workload(Q, 8, prec)
    else:
        leaf_rows = [0] * len(Q)
    t_tune = time.perf_counter() - t_tune
    b = pg.BatchedSVD(Q, kmodes=8, prec=prec, leaf_rows=leaf_rows)
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    st = b.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.spod_steps):
        b.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.spod_steps
    in_bytes = float(sum(int(n) * int(nb) * 8 for n, nb in zip(Ns, Nbs)))
    out_bytes = float(sum(int(n) * min(8, int(nb)) * 8 for n, nb in zip(Ns, Nbs)))
    flops = float(sum(8.0 * int(n) * int(nb) ** 2 for n, nb in zip(Ns, Nbs)))
    peak_ffma = probe_peak("ffma")
    # the ALU roofline's denominator from unit counts and clocks: 128 binary32
    # FMA lanes per SM per clock x 152 SMs x 2 flops x the maximum SM clock
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_alu = 128 * sms * 2 * 2.07e9 / 1e12
    # accuracy check on the two smallest bins: LAPACK's complex128 singular
    # values of the same complex64 data (element-wise parity is the tests')
    small = np.argsort(Ns * Nbs ** 2)[:2]
    errs = []
    for f in small:
        Xf = Q[f].cpu().numpy().astype(np.complex128)
        S_ref = np.linalg.svd(Xf, compute_uv=False)
        errs.append(float(np.max(np.abs(b.S[f].cpu().numpy() - S_ref)) / S_ref[0]))
    out = {"workload": f"spod_{args.spod_bins}bins_c64_N2^16..2^20_Nb16..128_k8", "ms_per_step": ms,
           "value": in_bytes / (ms * 1e-3) / 1e9, "unit": "GB/s of bins processed", "steps": args.spod_steps,
           "status": st, "input_bytes": in_bytes, "graph": "captured (memsets + one cooperative kernel)",
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak_alu,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / peak_alu,
                        "kernel": "svd_batched_kernel<float>",
                        "algorithmic_flops_per_launch": flops,
                        "peak_source": "derived: 128 FP32 FMA lanes/clk/SM x %d SMs x 2 flops x 2070 MHz "
                                       "(the live FMA probe reaches %.1f TFLOP/s)" % (sms, peak_ffma),
                        "hbm_gbs_of_algorithmic_bytes": (in_bytes + out_bytes) / (ms * 1e-3) / 1e9},
           "sigma_err_vs_lapack_smallest_bins": errs,
           "leaf_rows_tuned": bool(args.tune), "tune_seconds_untimed": t_tune,
           "tuned_policy_seconds": tune_times,
           "leaf_rows_histogram": {str(h): leaf_rows.count(h) for h in sorted(set(leaf_rows))}}
    del Q, b
    torch.cuda.empty_cache()
    return out


def bench_batched_pod(args, dev):
    """Multi-window PODs: 32 real float32 snapshot windows of uneven size (N_i
    log-uniform in [2^16, 2^20], M_i uniform in [16, 128]; traveling waves
    plus noise), each with its own temporal mean removal and cell volumes
    (Alg. 2 per window), in one persistent launch captured in a CUDA graph
    (binary32 leaves, binary64 R / tree / Jacobi, 8 modes per window)."""
    import numpy as np
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    Ns, Ms = synth.window_sizes(args.win_count, seed=17)
    X, W = [], []
    for i, (n, m) in enumerate(zip(Ns, Ms)):
        X.append(synth.waves_torch(int(n), int(m), min(6, int(m) // 3), "geometric", 1e-3, 500 + i, dev,
                                   dtype=torch.float32).t())
        W.append(torch.from_numpy(synth.log_uniform_weights(int(n), seed=600 + i)).to(dev))
    torch.cuda.synchronize()
    bp = pg.BatchedPOD(X, weights=W, remove_mean=True, kmodes=8, prec=pg.PREC_MIXED_3XTF32)
    bp.capture()
    bp.replay()
    torch.cuda.synchronize()
    st = bp.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.win_steps):
        bp.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.win_steps
    in_bytes = float(sum(int(n) * int(m) * 4 for n, m in zip(Ns, Ms)))
    flops = float(sum(2.0 * int(n) * int(m) ** 2 for n, m in zip(Ns, Ms)))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_alu = 128 * sms * 2 * 2.07e9 / 1e12
    # accuracy on the two smallest windows: LAPACK's singular values of the
    # same float32 data, centred and weighted in binary64
    small = np.argsort(Ns * Ms ** 2)[:2]
    errs = []
    for i in small:
        Xi = X[i].double().cpu().numpy()
        wi = W[i].cpu().numpy()
        Y = np.sqrt(wi)[:, None] * (Xi - Xi.mean(axis=1, keepdims=True))
        S_ref = np.linalg.svd(Y, compute_uv=False)
        errs.append(float(np.max(np.abs(bp.S[i].cpu().numpy() - S_ref)) / S_ref[0]))
    out = {"workload": f"pod_windows_{len(Ns)}_f32_N2^16..2^20_M16..128_k8", "ms_per_step": ms,
           "value": in_bytes / (ms * 1e-3) / 1e9, "unit": "GB/s of windows processed", "steps": args.win_steps,
           "status": st, "input_bytes": in_bytes, "graph": "captured (memsets + one cooperative kernel)",
           "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peak_alu,
                        "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / 1e12 / peak_alu,
                        "kernel": "svd_batched_kernel<float> (real windows through the complex leaves)",
                        "algorithmic_flops_per_launch": flops,
                        "flops_note": "2 sum N_i M_i^2 (real Householder QR); the leaves run the real "
                                      "windows with the complex arithmetic of the SPOD bins",
                        "peak_source": "derived: 128 FP32 FMA lanes/clk/SM x %d SMs x 2 flops x 2070 MHz" % sms},
           "sigma_err_vs_lapack_smallest_windows": errs}
    del X, W, bp
    torch.cuda.empty_cache()
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    n_rows = args.ref_rows
    steps = []
    for i in range(args.warmup + args.steps):
        gbs, dt, thr, desc = cpu_baseline(n_rows, M_FULL)
        if i >= args.warmup:
            steps.append(dt)
    t = statistics.median(steps)
    value = n_rows * M_FULL * 8 / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_FULL, "M": M_FULL, "sample_rows": n_rows},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": thr, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2405_15529_gb300 as pg
    import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    N, M = args.rows, M_FULL
    # page-locked host buffers of the end-to-end measurement, allocated first
    # (before the process's other host allocations)
    host = None
    if not args.no_e2e:
        host = {"X": torch.empty((M, N), dtype=torch.float64, pin_memory=True),
                "U": torch.empty((M, N), dtype=torch.float64, pin_memory=True)}
    XT, w, s = synth.known_spectrum_torch(N, M, device=dev)
    X = XT.t()
    torch.cuda.synchronize()
    # leaf height: given, or the autotuner's (timed outside the timed region, cached)
    tuned_leaf = None
    if args.leaf_rows == 0 and args.tune:
        from paper_2405_15529_gb300 import tune
        t_tune = time.perf_counter()
        tuned_leaf = tune.pod_leaf_rows_for(N, M, pg.PREC_FP64, tune=True)
        t_tune = time.perf_counter() - t_tune
        args.leaf_rows = tuned_leaf
    P = pg.leaf_count(N, M, args.leaf_rows)
    ws_bytes = pg.pod_workspace_size(N, M, args.leaf_rows, M, pg.F64, pg.PREC_FP64)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    U = pg.empty_colmajor(N, M, torch.float64, dev)
    S = torch.empty(M, dtype=torch.float64, device=dev)
    VT = pg.empty_colmajor(M, M, torch.float64, dev)
    r_dev = torch.zeros(1, dtype=torch.int64, device=dev)
    out = (U, S, VT, None, r_dev)

    def step():
        pg.pod(X, w=w, remove_mean=False, energy=ENERGY, r_max=M, leaf_rows=args.leaf_rows,
               workspace=ws, out=out, check=False)

    for _ in range(args.warmup):
        step()
    st, r, sweeps = pg.workspace_status(ws)
    if st != pg.OK:
        raise RuntimeError(f"pylom_pod failed during warm-up: status {st}")
    S_np = S.cpu().numpy()
    sig_err = float(np.max(np.abs(S_np - s)) / s[0])

    # FP64 roofline denominators, measured on this GPU
    peak_mma = probe_peak("mma")
    peak_fma = probe_peak("fma")
    mm_tflops = fp64_matmul_tflops(dev)
    torch.cuda.synchronize()

    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    pg.profile_begin(args.steps)
    # an event between consecutive steps as well, for the median step
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps - 1)]
    e0.record(stream)
    for i in range(args.steps):
        step()
        if i + 1 < args.steps:
            evs[i].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    phases, ncalls = pg.profile_end()
    clk = clocks.stop()
    ms = rank_max(e0.elapsed_time(e1) / args.steps, dev)
    marks = [e0] + evs + [e1]
    step_ms = sorted(marks[i].elapsed_time(marks[i + 1]) for i in range(args.steps))
    median_ms = step_ms[len(step_ms) // 2] if len(step_ms) % 2 else 0.5 * (
        step_ms[len(step_ms) // 2 - 1] + step_ms[len(step_ms) // 2])

    # the same call captured in a CUDA graph and replayed (outside the timed region)
    graph_ms = None
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            step()
        gs.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            step()
        graph.replay()
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        for _ in range(args.steps):
            graph.replay()
        g1.record()
        torch.cuda.synchronize()
        graph_ms = g0.elapsed_time(g1) / args.steps
        del graph
    except RuntimeError as exc:     # reported, not fatal: the eager number above is the result
        graph_ms = f"capture failed: {exc}"
    bytes_x = N * M * 8
    value = job_gbs(bytes_x, ms, world)

    # dominant kernel: the leaf QR kernel (one launch per step).  When the
    # tree runs as its own cooperative kernel (from 64 leaves) the leaf
    # kernel's work is the leaves' 2NM^2 - (2/3)PM^3; when the leaves merge
    # as they finish, the tree's (P - 1)(2/3)M^3 is in the same launch.
    leaf_ms = phases["leaf_qr"] / max(ncalls, 1)
    tree_ms = phases["tree"] / max(ncalls, 1)
    coop_tree = tree_ms > 0.0
    flops_tree = (P - 1) * (2.0 / 3.0) * M ** 3
    flops_leaf = 2.0 * N * M * M - (2.0 / 3.0) * P * M ** 3 + (0.0 if coop_tree else flops_tree)
    achieved = flops_leaf / (leaf_ms * 1e-3) / 1e12
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    hbm_peak = hbm_peak or 6800.0
    t_roof = max(bytes_x / (hbm_peak * 1e9), 2.0 * N * M * M / (peak_mma * 1e12))
    pct_roof = t_roof / (ms * 1e-3)

    # end to end through the public API from pinned host memory: pylom_pod
    # reads X where it lies (page-locked host memory, mapped into the
    # device's address space) -- the leaf kernel's prologue loads cross the
    # host link, so the transfer is part of the POD launch and overlaps its
    # compute; the modes, S, VT and r come back by copies
    e2e = None
    if not args.no_e2e:
        Xh = host["X"]
        Xh.copy_(XT)
        XhT = Xh.t()                          # column-major N x M view of the host buffer
        wh = w.cpu().pin_memory()
        wd = torch.empty_like(w)
        Uh = host["U"]
        Sh = torch.empty(M, dtype=torch.float64, pin_memory=True)
        VTh = torch.empty((M, M), dtype=torch.float64, pin_memory=True)
        rh = torch.empty(1, dtype=torch.int64, pin_memory=True)
        d2h = 0

        split = {"w_h2d": 0.0, "pod_reading_host_x": 0.0, "d2h": 0.0}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

        def fetch_results():
            nonlocal d2h
            rh.copy_(r_dev, non_blocking=True)
            Sh.copy_(S, non_blocking=True)
            VTh.copy_(VT.t(), non_blocking=True)
            torch.cuda.current_stream().synchronize()
            rr = int(rh.item())
            Uh[:rr].copy_(U.t()[:rr], non_blocking=True)
            d2h = 8 + M * 8 + M * M * 8 + rr * N * 8

        def e2e_step(record=False):
            if record:
                ev[0].record()
            wd.copy_(wh, non_blocking=True)
            if record:
                ev[1].record()
            pg.pod(XhT, w=wd, remove_mean=False, energy=ENERGY, r_max=M, leaf_rows=args.leaf_rows,
                   workspace=ws, out=out, check=False)
            if record:
                ev[2].record()
            fetch_results()
            if record:
                ev[3].record()
                ev[3].synchronize()
                split["w_h2d"] += ev[0].elapsed_time(ev[1])
                split["pod_reading_host_x"] += ev[1].elapsed_time(ev[2])
                split["d2h"] += ev[2].elapsed_time(ev[3])
        e2e_step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(args.steps):
            e2e_step()
        f1.record()
        torch.cuda.synchronize()
        ems = rank_max(f0.elapsed_time(f1) / args.steps, dev)
        # one more step with events between its parts (outside the timed region)
        e2e_step(record=True)
        torch.cuda.synchronize()
        S_e2e = Sh.clone()
        # the other route, outside the timed region: copy X with the copy
        # engines (256 MB pieces), then the POD of the device copy
        Xd = torch.empty_like(XT)
        c = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        copy_route = []
        for _ in range(3):
            c[0].record()
            pg.upload(Xd, Xh)
            wd.copy_(wh, non_blocking=True)
            c[1].record()
            pg.pod(Xd.t(), w=wd, remove_mean=False, energy=ENERGY, r_max=M, leaf_rows=args.leaf_rows,
                   workspace=ws, out=out, check=False)
            fetch_results()
            c[2].record()
            c[2].synchronize()
            copy_route.append({"ms": c[0].elapsed_time(c[2]),
                               "h2d_gbs": (N * M * 8 + N * 8) / (c[0].elapsed_time(c[1]) * 1e-3) / 1e9})
        del Xd
        e2e = {"value": job_gbs(bytes_x, ems, world), "unit": "GB/s", "ms_per_step": ems,
               "h2d_bytes_per_step": N * M * 8 + N * 8, "d2h_bytes_per_step": d2h,
               "route": "pylom_pod on the page-locked host X (read by the leaf kernel across the host link) "
                        "+ 33.6 MB copy of w; U[:, :r], S, VT, r copied back",
               "split_ms_one_step": split, "host_buffers_pinned": bool(Xh.is_pinned() and Uh.is_pinned()),
               "host_x_read_gbs_one_step": N * M * 8 / ((split["pod_reading_host_x"] - ms) * 1e-3) / 1e9
               if split["pod_reading_host_x"] > ms else None,
               "same_result_as_device_x": bool(torch.equal(S_e2e, S.cpu())),
               "copy_engine_route_outside_timed_region": copy_route}
        if not args.no_h2d_sweep:
            e2e["h2d_sweep_outside_timed_region"] = h2d_sweep(Xh, dev)
        e2e["placement"] = gpu_numa_info(local_rank)
        del Xh, XhT, Uh, host

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        if args.cpu_rows >= N:
            Xc = XT.cpu().numpy().T          # the same X (column-major N x M) on the host
            gbs, dt, thr, desc = cpu_baseline(N, M, X=Xc, w=w.cpu().numpy())
            del Xc
        else:
            gbs, dt, thr, desc = cpu_baseline(args.cpu_rows, M)
        cpu = {"value": gbs, "unit": "GB/s", "cores": thr, "kind": "oracle", "sample": desc,
               "seconds": dt}

    # free the POD buffers before the extra workloads
    del XT, X, ws, U, S, VT, r_dev, out
    torch.cuda.empty_cache()
    extra = {}
    if world == 1 and not args.no_mixed:
        extra["mixed_3xtf32"] = bench_mixed(args, dev)
    if world == 1 and not args.no_adjoint:
        extra["adjoint"] = bench_adjoint(args, dev)
    if world == 1 and not args.no_spod:
        extra["spod_batched"] = bench_spod(args, dev)
    if world == 1 and not args.no_spod:
        extra["spod_end_to_end"] = bench_spod_end_to_end(args, dev)
    if world == 1 and not args.no_win:
        try:
            extra["batched_pod_windows"] = bench_batched_pod(args, dev)
        except Exception as exc:          # recorded; the headline line still prints
            extra["batched_pod_windows"] = {"error": f"{type(exc).__name__}: {exc}"}
    if world == 1 and not args.no_dmd:
        extra["dmd_oscillations"] = bench_dmd(args, dev)
    if world == 1 and not args.no_stream:
        extra["streamed_host_resident"] = bench_streamed(args, dev)
    if world == 1 and not args.no_c3:
        extra["mixed_waves_1808"] = bench_waves_1808(args, dev)

    tree_env = os.environ.get("PYLOM_TREE", "")
    tree_kernel = ("tree_coop_kernel (level by level, merges spread over all blocks)"
                   if tree_env == "coop" or (tree_env != "pipe" and M >= 384)
                   else "tree_pipe_kernel (column-block pipeline, one block per merge)")
    levels = max(0, math.ceil(math.log2(P))) if P > 1 else 0
    # per POD call (counted in the ncu launch list of this command): leaf kernel, tree kernel
    # (pipelined or cooperative; none when the leaves merge as they finish), the small SVD
    # (binary32 preconditioning from M = 256: init, sweeps, widen, 2 Newton-Schulz steps of two
    # products each + A = R^T V; else one init) + binary64 sweeps + finalize, the root block,
    # one top-down launch per tree level, the modes
    svd_launches = (3 + 5 + 2 if M >= 256 else 1) + 2
    launches_per_step = 1 + (1 if P >= 64 or M >= 384 else 0) + svd_launches + 1 + levels + 1
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "M": M, "leaves": P, "r": r,
                       "leaf_rows": args.leaf_rows,
                       "leaf_rows_source": ("autotuned (tune.pod_leaf_rows_for, %.0f s outside the timed region)"
                                            % t_tune) if tuned_leaf else (
                           "given" if args.leaf_rows else "automatic"),
                       "l2": "inputs (8.6 GB per rank) larger than L2 (129 MB); no flush",
                       "parallelism": f"independent problems x{world}"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak_mma, "unit": "TFLOP/s",
                         "frac": achieved / peak_mma, "traffic": LEAF_FP64_TRAFFIC_BYTES if (
                             N == N_FULL and M == M_FULL and P == 304) else None,
                         "traffic_source": LEAF_FP64_TRAFFIC_SOURCE,
                         "algorithmic_bytes_per_launch": (8 + 8) * N * M,
                         "kernel": "leaf_qr_kernel (leaf Householder QR%s)" % (
                             "; the tree is its own kernel" if coop_tree else " + tree merges"),
                         "peak_source": "measured live: FP64 mma.sync.m8n8k4 throughput probe with "
                                        "independent chains (bench_probe.cu; MEASURED_PEAKS.json has no "
                                        "FP64 figure); cross-checked by the FP64 4096^3 product",
                         "algorithmic_flops_per_launch": flops_leaf, "ms_per_launch": leaf_ms,
                         "tree": {"kernel": tree_kernel, "ms_per_launch": tree_ms,
                                  "algorithmic_flops_per_launch": flops_tree,
                                  "achieved_tflops": flops_tree / (tree_ms * 1e-3) / 1e12 if coop_tree else None}},
            "pct_roofline_pod": {"value": pct_roof,
                                 "formula": "max(bytes_X/HBM_peak, 2NM^2/FP64_mma_peak) / step time",
                                 "hbm_peak_gbs": hbm_peak, "fp64_mma_tflops": peak_mma,
                                 "fp64_fma_tflops": peak_fma,
                                 "fp64_matmul_4096cubed_tflops": mm_tflops},
            "phases_ms_per_step": {k: v / max(ncalls, 1) for k, v in phases.items()},
            "step_timing": {"mean_ms": ms, "median_ms": median_ms, "min_ms": step_ms[0], "max_ms": step_ms[-1],
                            "graph_replay_ms": graph_ms,
                            "graph_note": "one pylom_pod call captured in a CUDA graph, replayed "
                                          "args.steps times after the timed region"},
            "accuracy": {"sigma_max_abs_err_over_smax_vs_closed_form": sig_err, "r": r,
                         "jacobi_sweeps": sweeps},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
            "clocks": clk, "extra": extra,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_case(name: str) -> int:
    """Fixed workloads for kernel captures (no JSON line):
    spod16        the batched-SVD section on the first 16 SPOD bins, one replay;
    mixed1808     two mixed-precision POD calls on the 2,000,000 x 1808 wave field
                  (64 waves, power-law amplitudes, noise 1e-4, mean removed, 99 %, r <= 128),
                  phases printed;
    mixedwave512  two mixed-precision POD calls on a 1,048,576 x 512 wave field (same recipe);
    fp64ks        two binary64 POD calls on the 262,144 x 256 known-spectrum matrix (weights, 99 %,
                  256 leaves), the small case of the benchmark workload's leaf and modes kernels;
    spodfront     two SPOD front-end calls on a 262,144 x 4128 float32 wave field (windows of 64
                  instants overlapping by 32: 128 blocks, 33 frequencies), then three timed calls
                  with and three without the mean removal."""
    import torch
    import paper_2405_15529_gb300 as pg
    import synth
    dev = torch.device("cuda", 0)
    if name == "spod16":
        out = bench_spod(argparse.Namespace(spod_bins=16, spod_steps=1, tune=False, warmup=1), dev)
        print("ms", round(out["ms_per_step"], 1), out["status"])
        return 0
    if name == "spodfront":
        N, T, npwin, nolap = 1 << 18, 4128, 64, 32
        XT = synth.waves_torch(N, T, 8, "geometric", 1e-3, 12, dev, dtype=torch.float32, row_chunk=1 << 18)
        D = XT.t()
        Q = None
        for _ in range(2):
            Q = pg.spod_blocks(D, npwin, nolap, True, Q=Q)
        torch.cuda.synchronize()
        out = {"case": name, "N": N, "T": T, "npwin": npwin, "nolap": nolap}
        for rm in (True, False):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                pg.spod_blocks(D, npwin, nolap, rm, Q=Q)
            e1.record()
            torch.cuda.synchronize()
            out["ms_remove_mean" if rm else "ms_no_mean"] = e0.elapsed_time(e1) / 3
        print(json.dumps(out))
        return 0
    if name == "fp64ks":
        N, M = 1 << 18, M_FULL
        XT, w, _ = synth.known_spectrum_torch(N, M, device=dev)
        X = XT.t()
        for _ in range(2):
            res = pg.pod(X, w=w, remove_mean=False, energy=ENERGY, r_max=M)
        st, r, sw = pg.workspace_status(res.workspace)
        print(json.dumps({"case": name, "N": N, "M": M, "leaves": pg.leaf_count(N, M, 0), "r": r, "status": st}))
        return 0
    N, M = {"mixed1808": (2_000_000, 1808), "mixedwave512": (1 << 20, 512)}[name]
    XT = synth.waves_torch(N, M, 64, "powerlaw", 1e-4, 5, dev, dtype=torch.float32, row_chunk=1 << 18)
    X = XT.t()
    res = pg.pod(X, remove_mean=True, energy=0.99, r_max=128, prec=pg.PREC_MIXED_3XTF32)
    torch.cuda.synchronize()
    pg.profile_begin(1)
    res = pg.pod(X, remove_mean=True, energy=0.99, r_max=128, prec=pg.PREC_MIXED_3XTF32, check=False)
    torch.cuda.synchronize()
    ph, n = pg.profile_end()
    st, r, sw = pg.workspace_status(res.workspace)
    print(json.dumps({k: round(v / max(n, 1), 2) for k, v in ph.items()} | {"r": r, "sweeps": sw, "status": st,
                                                                           "N": N, "M": M}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rows", type=int, default=N_FULL)
    ap.add_argument("--leaf-rows", type=int, default=0)
    ap.add_argument("--cpu-rows", type=int, default=N_FULL,
                    help="rows of the oracle's CPU baseline (>= --rows: the full workload)")
    ap.add_argument("--ref-rows", type=int, default=1 << 16)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-h2d-sweep", action="store_true", help="skip the upload-rate diagnostics")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-spod", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the 10,000,000 x 1808 mixed-vs-FP64 section")
    ap.add_argument("--no-stream", action="store_true", help="skip the host-resident (streamed) POD section")
    ap.add_argument("--no-dmd", action="store_true", help="skip the exact-DMD section")
    ap.add_argument("--no-win", action="store_true", help="skip the multi-window batched POD section")
    ap.add_argument("--win-count", type=int, default=32)
    ap.add_argument("--win-steps", type=int, default=3)
    ap.add_argument("--dmd-steps", type=int, default=3)
    ap.add_argument("--stream-chunk", type=int, default=1 << 20)
    ap.add_argument("--stream-steps", type=int, default=2)
    ap.add_argument("--c3-rows", type=int, default=C3_N)
    ap.add_argument("--c3-steps", type=int, default=3)
    ap.add_argument("--c3-cpu", action="store_true",
                    help="time the oracle on row samples of the 10,000,000 x 1808 workload (minutes)")
    ap.add_argument("--adj-steps", type=int, default=3)
    ap.add_argument("--spod-steps", type=int, default=3)
    ap.add_argument("--spod-bins", type=int, default=256)
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="run the SPOD bins with the built-in leaf heights instead of the autotuned ones")
    ap.add_argument("--case", choices=["spod16", "mixed1808", "mixedwave512", "fp64ks", "spodfront"], default=None,
                    help="run one fixed workload for a kernel capture instead of the benchmark")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
