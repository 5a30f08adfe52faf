#!/usr/bin/env python
"""Throughput benchmark of the hybrid Fourier / real-space galaxy renderer.

Workload (one step): render the fixed-size batch of 100,000 synthetic
galaxies at 64 x 64 (50/50 exponential / de Vaucouleurs mixtures, r_e
log-uniform 0.3-20 px, |e| <= 0.6, flux 1-1e4, sub-pixel offsets, one shared
two-Gaussian PSF) with one call of the library's batched render.  Inputs are
resident in HBM when the timed region starts.

Prints one JSON line (rank 0).  Under torchrun each rank renders its own copy
of the batch on its own GPU (replicas: no collective on the data path; the
barrier and the max over ranks of the elapsed time are control only).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the plain reference of the
method) on the host cores on bounded samples of the same workload.
"""

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

G_DEFAULT = 100_000
N_PATCH = 64
METRIC = "galaxy patches rendered/s at 64x64 (100k-galaxy fixed-size batch)"
UNIT = "patches/s"
PARAM_BYTES = 7 * 4 + 3 * 4 + 8      # float params, int ids, int64 offset
SFU_PER_CLK_SM = 32                  # MUFU ex2 per SM per clock (measured live: "pipe_rates" in the line)
FP32_FLOP_PER_CLK_SM = 256           # 128 FMA lanes x 2 (measured live: "pipe_rates")
KERNEL_SOURCES = ("paper_2012_15797_gb300/csrc/render_fwd.cu", "paper_2012_15797_gb300/csrc/common.cuh")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "render_fwd_64_100k.md")
KERNELS_PER_RENDER = 5   # the planner's three kernels, the record prologue, the size kernel


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--galaxies", type=int, default=G_DEFAULT)
    ap.add_argument("--size", type=int, default=0, choices=(0, 32, 64, 128, 256),
                    help="with --only fwd/grad: the galaxies of that patch side out of a mixed-size draw of "
                         "--galaxies (16 PSFs) instead of the 64x64 fixed-size batch")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extra", action="store_true", help="skip the mixed-size / gradient / per-galaxy lines")
    ap.add_argument("--extra-steps", type=int, default=20)
    ap.add_argument("--only", choices=("fwd", "grad", "mixed", "serving", "lanczos", "eigen", "pipes"),
                    help="profiling mode: run just this workload (--galaxies of it) for --warmup + --steps "
                         "and print its time")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# Algorithmic work of the method per galaxy (what it must compute).
# ----------------------------------------------------------------------------

def split_counts(gals, tables, kpsf):
    """Per galaxy: Fourier components (w_F > 0) and real-space terms
    (components with w_F < 1 times PSF-mixture components), from the
    aliasing split of Step 4 at each galaxy's own patch side."""
    import numpy as np
    nf = np.zeros(len(gals), dtype=np.int64)
    nr = np.zeros(len(gals), dtype=np.int64)
    e = np.hypot(gals.e1.astype(np.float64), gals.e2.astype(np.float64))
    beta = (1 - e) / (1 + e)
    tr = np.exp(2 * gals.log_re.astype(np.float64)) * (1 + beta * beta)
    side = np.asarray(gals.size, dtype=np.float64)
    for pid, t in tables.items():
        sel = np.nonzero(gals.profile == pid)[0]
        if len(sel) == 0:
            continue
        if len(t.nodes) == 1:
            a = np.broadcast_to(t.amp[0], (len(sel), t.amp.shape[1]))
            v = np.broadcast_to(t.var[0], (len(sel), t.var.shape[1]))
        else:
            u = np.clip((gals.sersic_n[sel] - t.nodes[0]) / (t.nodes[1] - t.nodes[0]), 0, len(t.nodes) - 1)
            j = np.minimum(u.astype(np.int64), len(t.nodes) - 2)
            w = (u - j)[:, None]
            a = (1 - w) * t.amp[j] + w * t.amp[j + 1]
            v = np.exp((1 - w) * np.log(t.var[j]) + w * np.log(t.var[j + 1]))
        ns = 0.5 * side[sel, None] / np.sqrt(v * tr[sel, None])
        tt = np.clip(ns - 3.0, 0.0, 1.0)
        wf = tt * tt * (3 - 2 * tt)
        nf[sel] = ((a > 0) & (wf > 0)).sum(axis=1)
        nr[sel] = ((a > 0) & (wf < 1)).sum(axis=1) * kpsf
    return nf, nr


def algorithmic_work(gals, tables, kpsf):
    """What the forward method must compute for these galaxies (each at its
    own patch side N), counted as the scope table of the hot path does:
    HBM bytes = the patch written + the parameters read; MUFU ex2 = one per
    Fourier component per half-spectrum bin + one per real-space term per
    pixel; FP32 flops = 5 N^2 log2 N (the inverse real 2-D FFT) +
    (14 + 2 n_F) per bin (quadratic form, PSF and phase products, and per
    component a scale and an accumulate) + 8 per real-space term per pixel."""
    import numpy as np
    nf, nr = split_counts(gals, tables, kpsf)
    n = np.asarray(gals.size, dtype=np.float64)
    bins = n * (n // 2 + 1)
    ex2 = float((nf * bins + nr * n * n).sum())
    flops = float((5.0 * n * n * np.log2(n) + bins * (14.0 + 2.0 * nf) + 8.0 * nr * n * n).sum())
    hbm = float((n * n * 4 + PARAM_BYTES).sum())
    comps = float(nf.sum() + nr.sum() / kpsf)
    return dict(ex2=ex2, flops=flops, hbm_bytes=hbm, real_fraction=float(nr.sum() / kpsf) / max(comps, 1.0),
                fourier_components=float(nf.sum()), real_terms=float(nr.sum()))


def adjoint_work(gals, tables, kpsf):
    """What the adjoint must compute (6 gradients per galaxy): HBM bytes =
    the upstream-gradient patch read + parameters read + 6 floats written;
    MUFU ex2 as the forward (every Gaussian is evaluated once per bin or
    pixel); FP32 flops = 5 N^2 log2 N (the forward real 2-D FFT of the
    gradient patch) + (32 + 7 n_F) per bin (conj(G) P phase: 12, the six
    gradient accumulations: 20; per component a scale and three
    accumulations of value, q- and ramp-derivative) + 14 per real-space
    term per pixel (the forward's 8 plus the three moments)."""
    import numpy as np
    nf, nr = split_counts(gals, tables, kpsf)
    n = np.asarray(gals.size, dtype=np.float64)
    bins = n * (n // 2 + 1)
    ex2 = float((nf * bins + nr * n * n).sum())
    flops = float((5.0 * n * n * np.log2(n) + bins * (32.0 + 7.0 * nf) + 14.0 * nr * n * n).sum())
    hbm = float((n * n * 4 + PARAM_BYTES + 6 * 4).sum())
    return dict(ex2=ex2, flops=flops, hbm_bytes=hbm)


def add_work(a, b):
    return {k: a[k] + b[k] for k in ("ex2", "flops", "hbm_bytes")}


def roofline(work, ms, pk, kernel, traffic=None):
    """Achieved / peak of the binding pipe for `work` done in `ms`, with the
    fractions of all three (HBM bytes, MUFU ex2, FP32 flops)."""
    t = {"hbm": work["hbm_bytes"] / pk["hbm"], "sfu": work["ex2"] / pk["sfu"], "fp32": work["flops"] / pk["fp32"]}
    bound = max(t, key=t.get)
    sec = ms / 1e3
    if bound == "hbm":
        roof = {"bound": "hbm", "achieved": work["hbm_bytes"] / sec / 1e9, "peak": pk["hbm"] / 1e9, "unit": "GB/s"}
    elif bound == "sfu":
        roof = {"bound": "alu", "pipe": "MUFU ex2", "achieved": work["ex2"] / sec / 1e12, "peak": pk["sfu"] / 1e12,
                "unit": "Tex2/s"}
    else:
        roof = {"bound": "alu", "pipe": "FP32", "achieved": work["flops"] / sec / 1e12, "peak": pk["fp32"] / 1e12,
                "unit": "TFLOP/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic
    roof["kernel"] = kernel
    roof["kernel_ms"] = ms
    roof["peak_source"] = {"hbm": f"{pk['hbm_src']} HBM copy GB/s (MEASURED_PEAKS.json)",
                           "sfu": f"{pk['num_sms']} SMs x {SFU_PER_CLK_SM} ex2/clk x {pk['sm_mhz']:.0f} MHz "
                                  f"(ex2 rate measured, profiles/pipe_throughput.md)",
                           "fp32": f"{pk['num_sms']} SMs x {FP32_FLOP_PER_CLK_SM} flop/clk x {pk['sm_mhz']:.0f} MHz "
                                   f"(FFMA rate measured, profiles/pipe_throughput.md)"}[bound]
    roof["fractions"] = {k: round(v / sec, 4) for k, v in t.items()}
    roof["algorithmic_per_launch"] = {"hbm_bytes": work["hbm_bytes"], "ex2": work["ex2"], "flops": work["flops"]}
    return roof


def peaks(num_sms):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    src = "measured"
    try:
        with open(path) as f:
            mp = json.load(f)
        hbm = float(mp["hbm_gbs"]) * 1e9
        mhz = float(mp.get("sm_max_mhz", 2070.0))
    except (OSError, KeyError, ValueError):
        hbm, mhz, src = 6.8e12, 2070.0, "fallback"
    clk = mhz * 1e6
    return dict(hbm=hbm, hbm_src=src, sfu=num_sms * SFU_PER_CLK_SM * clk, fp32=num_sms * FP32_FLOP_PER_CLK_SM * clk,
                sm_mhz=mhz, num_sms=num_sms)


def kernel_source_sha():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(galaxies):
    """DRAM bytes per launch from the committed ncu summary, scaled to
    ``galaxies``; None when the kernel changed since the capture."""
    try:
        txt = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    per = re.search(r"dram_bytes_per_galaxy:\s*([0-9.eE+]+)", txt)
    if not sha or not per or sha.group(1) != kernel_source_sha():
        return None
    return float(per.group(1)) * galaxies


def measure_pipes(r, gpu_index, reps=300):
    """Rates of the MUFU ex2 and FP32 FMA pipes on this GPU (library probe
    kernels), per SM and clock at the SM clock sampled meanwhile."""
    from paper_2012_15797_gb300 import capi
    capi.mog_measure_pipe_rates(r.ctx, 3)
    sampler = ClockSampler(gpu_index)
    sampler.start()
    ex2, fma = capi.mog_measure_pipe_rates(r.ctx, reps)
    clocks = sampler.stop()
    import torch
    sms = torch.cuda.get_device_properties(gpu_index).multi_processor_count
    mhz = clocks["sm_mhz"] or 2070.0
    return {"ex2_per_s": ex2, "fma_per_s": fma, "sm_mhz": mhz, "clock_samples": clocks["samples"],
            "ex2_per_clk_sm": ex2 / (sms * mhz * 1e6), "fma_lanes_per_clk_sm": fma / (sms * mhz * 1e6),
            "method": f"{reps} launches each of 8 independent ex2.approx / FFMA chains of 4096 per thread, "
                      f"8 x 256-thread CTAs per SM, CUDA events; per clock at the median sampled SM clock"}


# ----------------------------------------------------------------------------
# Clocks during the timed region.
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6], swt=parts[7],
                                 pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sms = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                              ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sms[len(sms) // 2], "sm_max_mhz": rows[0]["smax"], "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm): a spawn pool over the host cores.
# ----------------------------------------------------------------------------

_W = {}


def _worker_init(seed_g):
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import render as R
    from workloads import single_psf, fixed_galaxies_64, load_profile_tables
    _W["R"] = R
    _W["tables"] = load_profile_tables()
    _W["psf"] = single_psf()
    _W["gals"] = fixed_galaxies_64(seed_g)
    _W["hat"] = R.psf_spectrum(_W["psf"].image, N_PATCH)


def _worker_render(idx):
    R, gals = _W["R"], _W["gals"]
    t = time.perf_counter()
    for i in idx:
        R.render(gals.row(int(i)), None, _W["psf"].mog, _W["tables"], psf_hat=_W["hat"])
    return len(idx), time.perf_counter() - t


def _worker_timed(args):
    start, stride, budget = args
    R, gals = _W["R"], _W["gals"]
    t0 = time.perf_counter()
    n = 0
    i = start
    while time.perf_counter() - t0 < budget and i < len(gals):
        R.render(gals.row(int(i)), None, _W["psf"].mog, _W["tables"], psf_hat=_W["hat"])
        n += 1
        i += stride
    return n


# The oracle on the secondary workloads (the 200k mixed batch, the 50k fit
# problem): each worker takes every `cores`-th galaxy from its start for a
# bounded wall time.
def _oracle_init(kind, psfs):
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle import adjoint as A
    from oracle import render as R
    from workloads import fixed_galaxies_64, load_profile_tables, mixed_galaxies
    _W.update(R=R, A=A, tables=load_profile_tables(), kind=kind, psfs=psfs, hats={})
    _W["gals"] = mixed_galaxies(200_000) if kind == "mixed" else fixed_galaxies_64(50_000, 3)


def _oracle_timed(args):
    import numpy as np
    start, stride, budget = args
    R, A, gals, psfs, tables, hats = _W["R"], _W["A"], _W["gals"], _W["psfs"], _W["tables"], _W["hats"]
    t0 = time.perf_counter()
    n, i = 0, start
    while time.perf_counter() - t0 < budget and i < len(gals):
        g = gals.row(int(i))
        key = (int(g["psf"]), int(g["size"]))
        if key not in hats:
            hats[key] = R.psf_spectrum(psfs[key[0]].image, key[1])
        mog = psfs[key[0]].mog
        model = R.render(g, None, mog, tables, psf_hat=hats[key])
        if _W["kind"] == "render_grad":
            # the step: loss gradient 2 ivar (model - data) and its VJP; the
            # data (here 1.01 x the model, ivar 1) do not change its cost
            resid = model - 1.01 * model
            _ = float(np.sum(resid * resid))
            A.vjp(g, hats[key], mog, tables, 2.0 * resid)
        n += 1
        i += stride
    return n


def oracle_baseline(kind, psfs, seconds):
    """The FP64 oracle on a bounded sample of a secondary workload, spawn
    workers over every host core: galaxies per wall second."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_init, initargs=(kind, psfs))
    try:
        pool.map(_oracle_timed, [(c, cores, 0.2) for c in range(cores)])   # warm
        t0 = time.perf_counter()
        counts = pool.map(_oracle_timed, [(c + cores * 64, cores, seconds) for c in range(cores)])
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    done = sum(counts)
    what = ("the 200k mixed batch (every galaxy's own side and PSF)" if kind == "mixed" else
            "the 50k fit problem: render, loss gradient and its vector-Jacobian product per galaxy")
    return {"value": done / wall, "unit": UNIT if kind == "mixed" else "patches rendered+grad/s", "cores": cores,
            "kind": "oracle", "sample": f"{done} galaxies of {what}, interleaved over {cores} spawn workers, "
                                        f"{seconds:.0f} s wall budget, FP64 numpy oracle"}


def cpu_pool(galaxies):
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_worker_init, initargs=(galaxies,)), cores


def cpu_baseline(galaxies, seconds):
    pool, cores = cpu_pool(galaxies)
    try:
        pool.map(_worker_render, [[i] for i in range(cores)])     # warm the workers
        t0 = time.perf_counter()
        counts = pool.map(_worker_timed, [(c, cores, seconds) for c in range(cores)])
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    done = sum(counts)
    return {"value": done / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} galaxies of the 100k fixed-size batch (indices interleaved over {cores} spawn "
                      f"workers, {seconds:.0f} s wall budget), FP64 numpy oracle",
            "single_core": cpu_single_core(galaxies, max(2.0, seconds / 4))}


def cpu_single_core(galaxies, seconds):
    """The same oracle on one core (one spawn worker, one BLAS thread), for
    a bounded wall time."""
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(1, initializer=_worker_init, initargs=(galaxies,))
    try:
        pool.map(_worker_render, [list(range(20))])   # warm: first calls are slower
        t0 = time.perf_counter()
        done = pool.apply(_worker_timed, ((20, 1, seconds),))
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    return {"value": done / wall, "unit": UNIT, "cores": 1,
            "sample": f"{done} galaxies of the 100k fixed-size batch in order from index 20, {seconds:.0f} s "
                      f"wall budget"}


# ----------------------------------------------------------------------------
# Secondary workloads: mixed sizes (graph + autotuner), render + gradient,
# one launch per galaxy.
# ----------------------------------------------------------------------------

def _event_ms(fn, steps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def extra_mixed(tables, device, steps, pk, cpu_seconds=0.0):
    """200k galaxies, Sersic n U(0.5, 6), N = smallest of 32..256 >= 8 r_e,
    64 PSFs: eager calls with default launch shapes vs one CUDA-graph launch
    per step after the autotuner."""
    import numpy as np
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import mixed_galaxies, psf_set

    psfs = psf_set(64)
    gals = mixed_galaxies(200_000)
    r = Renderer(tables, psfs, device=device)
    b = to_device(gals, device=f"cuda:{device}")
    out = torch.empty(b.total, dtype=torch.float32, device=f"cuda:{device}")
    st = torch.cuda.current_stream()
    for _ in range(3):
        r.render(b, out)
    r.sync_status()
    eager_ms = _event_ms(lambda: r.render(b, out), steps, st)
    shapes = r.autotune(b, out, reps=2)
    g = r.graph(b, out)
    for _ in range(3):
        g.launch()
    capi.mog_set_timing(r.ctx, True)
    capi.mog_read_timing(r.ctx)
    tuned_eager_ms = _event_ms(lambda: r.render(b, out), steps, st)
    kms, kn = capi.mog_read_timing(r.ctx)
    capi.mog_set_timing(r.ctx, False)
    graph_ms = _event_ms(g.launch, steps, st)
    r.sync_status()
    g.close()
    sizes, counts = np.unique(gals.size, return_counts=True)
    res = {
        "workload": "200000 galaxies, Sersic n U(0.5, 6) (8-12 components), r_e log-U(0.3, 20) px, "
                    "N = smallest of {32, 64, 128, 256} >= 8 r_e, 64 PSFs (2-Gaussian core + Moffat wings)",
        "bucket_mix": {int(n): int(c) for n, c in zip(sizes, counts)},
        "value_graph": len(gals) / (graph_ms / 1e3), "unit": UNIT, "ms_graph": graph_ms,
        "value_eager_default_shapes": len(gals) / (eager_ms / 1e3), "ms_eager_default": eager_ms,
        "ms_eager_tuned": tuned_eager_ms,
        "kernel_ms_per_size": {32 << i: (kms[i] / kn[i] if kn[i] else None) for i in range(4)},
        "autotuned_shapes": {(k if isinstance(k, str) else f"{k[0]}{k[1]}"): v for k, v in shapes.items()},
        "bytes_written": int(b.total) * 4,
    }
    # roofline of the whole launch (the four size kernels run side by side in
    # it) against the method's work for the 200k galaxies, and each size's
    # kernel against its own galaxies' work over its event time
    kpsf = psfs[0].mog.shape[0]
    res["roofline"] = roofline(algorithmic_work(gals, tables, kpsf), graph_ms, pk,
                               "graph: render_fwd_kernel<32|64|128> + render_fwd256_kernel")
    # each size's kernel alone (batch size mask = that side), CUDA events
    # around its launches: its own time and roofline
    per = {}
    for i in range(4):
        sel = np.flatnonzero(gals.size == (32 << i))
        if not len(sel):
            continue
        bi = capi.make_batch(b.count, b.ptrs(), 1 << i)
        capi.mog_render_batch(r.ctx, bi, out.data_ptr(), st.cuda_stream)
        capi.mog_set_timing(r.ctx, True)
        capi.mog_read_timing(r.ctx)
        _event_ms(lambda: capi.mog_render_batch(r.ctx, bi, out.data_ptr(), st.cuda_stream), steps, st)
        kms1, kn1 = capi.mog_read_timing(r.ctx)
        capi.mog_set_timing(r.ctx, False)
        k_ms = kms1[i] / max(kn1[i], 1)
        rf = roofline(algorithmic_work(gals.subset(sel), tables, kpsf), k_ms, pk, f"size {32 << i}")
        per[32 << i] = {"galaxies": int(len(sel)), "kernel_ms_alone": k_ms, "bound": rf.get("pipe", rf["bound"]),
                        "frac": round(rf["frac"], 4), "fractions": rf["fractions"]}
    r.sync_status()
    res["roofline_per_size_alone"] = per
    # the plain form: one library call per galaxy, on 2000 of them
    sample = np.arange(0, len(gals), len(gals) // 2000)[:2000]
    singles = [to_device(gals.subset([int(i)]), device=f"cuda:{device}") for i in sample]
    one = torch.empty(256 * 256, dtype=torch.float32, device=f"cuda:{device}")
    for bb in singles[:20]:
        r.render(bb, one)
    r.sync_status()
    ms1 = _event_ms(lambda: [r.render(bb, one) for bb in singles], 1, st)
    res["one_launch_per_galaxy"] = {"value": len(singles) / (ms1 / 1e3), "unit": UNIT, "galaxies": len(singles),
                                    "note": "one mog_render_batch call per galaxy of the mixed batch (every 100th)"}
    r.sync_status()
    r.close()
    if cpu_seconds > 0:
        res["cpu_baseline"] = oracle_baseline("mixed", psfs, cpu_seconds)
    return res


def extra_render_grad(tables, psf, device, steps, pk, cpu_seconds=0.0):
    """50k galaxies at 64^2: render, inverse-variance-weighted residual
    gradient (data from perturbed parameters + noise 0.01 peak), adjoint.
    The forward and adjoint kernels are also timed each on its own, for
    their rooflines."""
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import fit_problem

    model, truth, noise = fit_problem(50_000)
    r = Renderer(tables, [psf], device=device)
    dev = f"cuda:{device}"
    data = r.render(to_device(truth, device=dev)).view(len(truth), 64, 64)
    sigma = 0.01 * data.amax(dim=(1, 2), keepdim=True)
    data = data + sigma * torch.from_numpy(noise).to(dev)
    ivar = (1.0 / sigma ** 2).reshape(-1).contiguous()
    data = data.reshape(-1).contiguous()
    bm = to_device(model, device=dev)
    out = torch.empty(bm.total, device=dev)
    gpix = torch.empty(bm.total, device=dev)
    gp = torch.empty(len(model), 6, device=dev)
    chi2 = torch.empty(len(model), device=dev)

    def step():
        # render with the loss (mog_render_chi2: the gradient 2 ivar (model -
        # data) and chi^2 per galaxy, computed as the patches are stored),
        # adjoint: every step in the library's kernels
        r.render_chi2(bm, data, ivar, gpix, chi2)
        r.render_backward(bm, gpix, gp)

    def step_unfused():
        # the same with the model written out and the loss as its own kernel
        r.render(bm, out)
        r.chi2_gradient(bm, out, data, ivar, gpix, chi2)
        r.render_backward(bm, gpix, gp)

    st = torch.cuda.current_stream()
    for _ in range(3):
        step()
        step_unfused()
    r.sync_status()
    ms = _event_ms(step, steps, st)
    ms_unfused = _event_ms(step_unfused, steps, st)

    def kernel_ms(fn):
        capi.mog_set_timing(r.ctx, True)
        capi.mog_read_timing(r.ctx)
        _event_ms(fn, steps, st)
        kms, kn = capi.mog_read_timing(r.ctx)
        capi.mog_set_timing(r.ctx, False)
        return kms[1] / max(kn[1], 1)

    fwd_ms = kernel_ms(lambda: r.render(bm, out))
    bwd_ms = kernel_ms(lambda: r.render_backward(bm, gpix, gp))
    r.sync_status()
    kpsf = psf.mog.shape[0]
    wf, wb = algorithmic_work(model, tables, kpsf), adjoint_work(model, tables, kpsf)
    res = {"workload": "50000 galaxies as the fixed-size batch; loss = sum ivar (model - data)^2, data from "
                       "perturbed parameters + Gaussian noise sigma = 0.01 peak; gradients w.r.t. "
                       "(flux, x, y, log r_e, e1, e2); step = mog_render_chi2 (render and loss in one pass), "
                       "adjoint",
           "value": len(model) / (ms / 1e3), "unit": "patches rendered+grad/s", "ms_per_step": ms,
           "ms_per_step_unfused": ms_unfused,
           "kernel_ms_forward": fwd_ms, "kernel_ms_adjoint": bwd_ms,
           "roofline": roofline(wb, bwd_ms, pk, "render_bwd_kernel<64>"),
           "roofline_forward_plus_adjoint_kernels": roofline(add_work(wf, wb), fwd_ms + bwd_ms, pk,
                                                             "render_fwd_kernel<64> + render_bwd_kernel<64>")}
    # the plain form: one render-with-loss and one adjoint call per galaxy, on 2000 of them
    singles = [to_device(model.subset([i]), device=dev) for i in range(2000)]
    g1 = torch.empty(64 * 64, device=dev)
    c1 = torch.empty(1, device=dev)
    p1 = torch.empty(1, 6, device=dev)

    def per_galaxy():
        for i, bb in enumerate(singles):
            r.render_chi2(bb, data[i * 4096:(i + 1) * 4096], ivar[i:i + 1], g1, c1)
            r.render_backward(bb, g1, p1)

    per_galaxy()
    r.sync_status()
    ms1 = _event_ms(per_galaxy, 1, st)
    res["one_launch_per_galaxy"] = {"value": len(singles) / (ms1 / 1e3), "unit": "patches rendered+grad/s",
                                    "galaxies": len(singles),
                                    "note": "one mog_render_chi2 and one mog_render_backward call per galaxy"}
    r.sync_status()
    r.close()
    if cpu_seconds > 0:
        res["cpu_baseline"] = oracle_baseline("render_grad", [psf], cpu_seconds)
    return res


def extra_lanczos(tables, psf, device, steps):
    """The fixed-size batch (100k x 64^2) with the sub-pixel shift done by
    Lanczos-3 convolution (mog_render_batch_lanczos) instead of the Fourier
    phase."""
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import fixed_galaxies_64

    gals = fixed_galaxies_64()
    r = Renderer(tables, [psf], device=device)
    b = to_device(gals, device=f"cuda:{device}")
    out = torch.empty(b.total, device=f"cuda:{device}")
    st = torch.cuda.current_stream()
    for _ in range(3):
        r.render(b, out, shift="lanczos")
    r.sync_status()
    capi.mog_set_timing(r.ctx, True)
    capi.mog_read_timing(r.ctx)
    ms = _event_ms(lambda: r.render(b, out, shift="lanczos"), steps, st)
    kms, kn = capi.mog_read_timing(r.ctx)
    capi.mog_set_timing(r.ctx, False)
    r.sync_status()
    r.close()
    return {"workload": "the 100k-galaxy 64x64 batch, sub-pixel shift by Lanczos-3 convolution",
            "value": len(gals) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "kernel_ms": kms[1] / max(kn[1], 1)}


def extra_eigen(tables, psf, device, steps):
    """The fixed-size batch (100k x 64^2) on a spatially varying PSF: a
    degree-2 eigen-PSF model (6 pixelized components) with galaxies at
    uniform positions in a 4096^2 image; every galaxy forms its own PSF
    spectrum from the 6 component spectra."""
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import fixed_galaxies_64, eigen_positions, eigen_psf

    gals = fixed_galaxies_64()
    gals.psf[:] = 1
    r = Renderer(tables, [psf, eigen_psf()], device=device)
    b = to_device(gals, device=f"cuda:{device}", positions=eigen_positions(len(gals)))
    out = torch.empty(b.total, device=f"cuda:{device}")
    st = torch.cuda.current_stream()
    for _ in range(3):
        r.render(b, out)
    r.sync_status()
    capi.mog_set_timing(r.ctx, True)
    capi.mog_read_timing(r.ctx)
    ms = _event_ms(lambda: r.render(b, out), steps, st)
    kms, kn = capi.mog_read_timing(r.ctx)
    capi.mog_set_timing(r.ctx, False)
    r.sync_status()
    r.close()
    return {"workload": "the 100k-galaxy 64x64 batch on a degree-2 eigen-PSF (6 components), uniform positions",
            "value": len(gals) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "kernel_ms": kms[1] / max(kn[1], 1)}


def extra_composite(tables, psf, device, steps):
    """100k bulge + disk composites (exp disk, deV bulge, one centre), patch
    sides 32-128 by the disk's radius, in one pass (mog_render_composite:
    both profiles on one frequency grid, one transform per galaxy) and in
    two (the disks rendered, then the bulges added into the same patches,
    mog_render_batch_ex with MOG_RENDER_ADD)."""
    import numpy as np
    import torch
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer, pack_offsets, to_device
    from workloads import composite_galaxies

    disk, bulge = composite_galaxies(100_000)
    r = Renderer(tables, [psf], device=device)
    bd = to_device(disk, device=f"cuda:{device}")
    bb = to_device(bulge, device=f"cuda:{device}")
    out = torch.empty(bd.total, device=f"cuda:{device}")
    st = torch.cuda.current_stream()
    two = torch.empty(bd.total, device=f"cuda:{device}")
    for _ in range(3):
        r.render_composite(bd, bb, out)
        r.render_composite(bd, bb, two, fused=False)
    r.sync_status()
    ms = _event_ms(lambda: r.render_composite(bd, bb, out), steps, st)
    ms2 = _event_ms(lambda: r.render_composite(bd, bb, two, fused=False), steps, st)
    for _ in range(2):
        r.render_composite(bd, bb, two, shift="lanczos")
        r.render_composite(bd, bb, two, shift="lanczos", fused=False)
    ms_lz = _event_ms(lambda: r.render_composite(bd, bb, two, shift="lanczos"), steps, st)
    ms_lz2 = _event_ms(lambda: r.render_composite(bd, bb, two, shift="lanczos", fused=False), steps, st)
    r.sync_status()
    r.render_composite(bd, bb, two, fused=False)   # the phase-shift two-pass result again, compared below
    tot = torch.from_numpy((disk.flux + bulge.flux).astype(np.float32)).to(out.device)
    offs, _ = pack_offsets(disk.size)
    diff = max(((out[int(o):int(o) + int(n) ** 2] - two[int(o):int(o) + int(n) ** 2]).abs().max() / tot[g]).item()
               for g, (o, n) in enumerate(zip(offs, disk.size)) if g % 997 == 0)
    # the same distribution on 256 x 256 patches
    d256, b256 = composite_galaxies(5000, seed=8, sizes=(256,))
    d256.size[:] = 256
    b256.size[:] = 256
    bd2 = to_device(d256, device=f"cuda:{device}")
    bb2 = to_device(b256, device=f"cuda:{device}")
    o1 = torch.empty(bd2.total, device=f"cuda:{device}")
    o2 = torch.empty(bd2.total, device=f"cuda:{device}")
    for _ in range(3):
        r.render_composite(bd2, bb2, o1)
        r.render_composite(bd2, bb2, o2, fused=False)
    r.sync_status()
    ms256 = _event_ms(lambda: r.render_composite(bd2, bb2, o1), steps, st)
    ms256_two = _event_ms(lambda: r.render_composite(bd2, bb2, o2, fused=False), steps, st)
    r.sync_status()
    r.close()
    sizes, counts = np.unique(disk.size, return_counts=True)
    return {"side_256": {"galaxies": 5000, "ms_one_pass": ms256, "ms_two_pass": ms256_two,
                         "value": 5000 / (ms256 / 1e3), "unit": "composite patches/s"},
            "workload": "100000 bulge + disk composites: exp disk r_e log-U(0.5, 15) px, deV bulge r_e 0.2-0.6 of "
                        "the disk's, bulge fraction U(0, 1), sides by 8 r_e(disk)",
            "bucket_mix": {int(n): int(c) for n, c in zip(sizes, counts)},
            "value": len(disk) / (ms / 1e3), "unit": "composite patches/s", "ms_per_step": ms,
            "two_pass": {"value": len(disk) / (ms2 / 1e3), "ms_per_step": ms2,
                         "note": "disks rendered, bulges added (MOG_RENDER_ADD)"},
            "lanczos_shift": {"ms_one_pass": ms_lz, "ms_two_pass": ms_lz2, "value": len(disk) / (ms_lz / 1e3)},
            "max_abs_diff_over_flux_sampled": diff}


def extra_sersic_grad(tables, device, steps):
    """The 200k mixed-size Sersic batch: the adjoint (6 gradients per galaxy)
    and the adjoint with d L / d sersic_n (7 gradients)."""
    import torch
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import mixed_galaxies, psf_set

    gals = mixed_galaxies(200_000)
    r = Renderer(tables, psf_set(64), device=device)
    b = to_device(gals, device=f"cuda:{device}")
    go = torch.randn(b.total, device=f"cuda:{device}")
    g6 = torch.empty(len(gals), 6, device=f"cuda:{device}")
    g7 = torch.empty(len(gals), 7, device=f"cuda:{device}")
    st = torch.cuda.current_stream()
    for _ in range(2):
        r.render_backward(b, go, g6)
        r.render_backward(b, go, g7, sersic=True)
    r.sync_status()
    ms6 = _event_ms(lambda: r.render_backward(b, go, g6), steps, st)
    ms7 = _event_ms(lambda: r.render_backward(b, go, g7, sersic=True), steps, st)
    r.sync_status()
    r.close()
    return {"workload": "200000 galaxies as the mixed-size batch, adjoint only",
            "ms_grad6": ms6, "ms_grad7_with_sersic_n": ms7, "value": len(gals) / (ms7 / 1e3),
            "unit": "patches grad (7 gradients)/s"}


def extra_psf_fit(tables, device):
    """3-component Gaussian-mixture fits of the 64 Moffat-winged 64x64 PSFs
    of the mixed workload on the device (mog_fit_psf_mixture, 400 iterations
    at most)."""
    import numpy as np
    import torch
    from paper_2012_15797_gb300.renderer import Renderer
    from workloads import psf_set

    imgs = torch.from_numpy(np.stack([p.image for p in psf_set(64, fit=False)])).cuda(device)
    r = Renderer(tables, [], device=device)
    r.fit_psf_mixtures(imgs)
    torch.cuda.synchronize()
    ms = _event_ms(lambda: r.fit_psf_mixtures(imgs), 3, torch.cuda.current_stream())
    r.sync_status()
    r.close()
    return {"workload": "64 PSFs of 64x64 (2-Gaussian core + Moffat wings), k = 3", "ms_per_call": ms,
            "value": 64 / (ms / 1e3), "unit": "PSF fits/s"}


def extra_psf_create(tables, device, n=64):
    """mog_create_psf for the 64 Moffat-winged 64x64 PSFs of the mixed
    workload: each call embeds the PSF and takes its FP32 real 2-D FFT for
    every patch side (32, 64, 128, 256) on the device; host clock around the
    synchronous calls."""
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.renderer import Renderer
    from workloads import psf_set
    psfs = psf_set(n)
    r = Renderer(tables, [], device=device)
    for p in psfs[:4]:   # warm: loads the kernels
        capi.mog_destroy_psf(r.ctx, capi.mog_create_psf(r.ctx, p.image, p.mog))
    t0 = time.perf_counter()
    ids = [capi.mog_create_psf(r.ctx, p.image, p.mog) for p in psfs]
    ms = (time.perf_counter() - t0) * 1e3
    for i in ids:
        capi.mog_destroy_psf(r.ctx, i)
    r.close()
    return {"workload": f"{n} PSFs of 64x64, spectra for sides 32-256 (FP32 shared-memory FFTs)",
            "ms_per_psf": ms / n, "value": n / (ms / 1e3), "unit": "PSFs created/s"}


def extra_cufft(tables, psf, device, steps, pk, cases=((64, 100_000), (256, 5_000))):
    """The library comparator (mog_render_batch_cufft: every galaxy's half
    spectrum written out, one batched cuFFT inverse real transform, a
    real-space pass) timed beside the fused render on the same batch, with
    their largest difference and the comparator's HBM floor (its stages move
    8 (N/2 + 1) N bytes of spectrum twice and 4 N^2 bytes of image three
    times per galaxy)."""
    import torch
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import fixed_galaxies_64

    r = Renderer(tables, [psf], device=device)
    st = torch.cuda.current_stream()
    res = {}
    for n, g in cases:
        gals = fixed_galaxies_64(g, seed=6, size=n)
        b = to_device(gals, device=f"cuda:{device}")
        out_f = torch.empty(b.total, device=f"cuda:{device}")
        out_c = torch.empty(b.total, device=f"cuda:{device}")
        for _ in range(3):
            r.render(b, out_f)
            r.render_cufft(b, out_c)
        r.sync_status()
        ms_f = _event_ms(lambda: r.render(b, out_f), steps, st)
        ms_c = _event_ms(lambda: r.render_cufft(b, out_c), steps, st)
        r.sync_status()
        flux = torch.from_numpy(gals.flux.astype("float32")).to(out_f.device)
        d = ((out_c - out_f).abs().view(g, -1).amax(dim=1) / flux).max().item()
        hbm = g * (2 * 8 * (n // 2 + 1) * n + 3 * 4 * n * n)
        res[f"{n}x{n}"] = {"galaxies": g, "ms_fused": ms_f, "ms_cufft": ms_c, "cufft_over_fused": ms_c / ms_f,
                           "max_abs_diff_over_flux": d, "cufft_hbm_bytes": hbm,
                           "cufft_hbm_floor_ms": hbm / (pk["hbm"] / 1e3) if pk.get("hbm") else None}
        del out_f, out_c, b
    r.close()
    return res


def cufft_or_reason(tables, psf, device, steps, pk):
    """extra_cufft, or why it could not run (the comparator needs the cuFFT
    library at run time; the rest of the line does not)."""
    from paper_2012_15797_gb300 import capi
    try:
        return extra_cufft(tables, psf, device, steps, pk)
    except capi.MogError as e:
        return {"unavailable": str(e)}


def extra_per_galaxy(tables, psf, device, n=2000):
    """The plain form: the same math with one library call (planner, record,
    render launches) per galaxy."""
    import torch
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import fixed_galaxies_64

    gals = fixed_galaxies_64(n, seed=5)
    r = Renderer(tables, [psf], device=device)
    singles = [to_device(gals.subset([i]), device=f"cuda:{device}") for i in range(n)]
    out = torch.empty(64 * 64, device=f"cuda:{device}")
    for b in singles[:20]:
        r.render(b, out)
    r.sync_status()
    ms = _event_ms(lambda: [r.render(b, out) for b in singles], 1, torch.cuda.current_stream())
    r.close()
    return {"value": n / (ms / 1e3), "unit": UNIT, "galaxies": n,
            "note": "one mog_render_batch call per 64x64 galaxy of the fixed-size distribution"}


def parse_node_list(spec):
    """A kernel node list such as "0-1,4" as a list of ids."""
    nodes = []
    for part in spec.strip().split(","):
        if "-" in part:
            a, b = part.split("-")
            nodes.extend(range(int(a), int(b) + 1))
        elif part:
            nodes.append(int(part))
    return nodes


def host_numa_nodes():
    """The host's online NUMA nodes (a list of node ids), or None."""
    try:
        with open("/sys/devices/system/node/online") as f:
            return parse_node_list(f.read())
    except (OSError, ValueError):
        return None


def host_cpu_snapshot():
    """Process CPU time, context switches and (where the cgroup exposes
    them) CPU-quota throttling counters, to tell host-side stalls apart."""
    import resource
    ru = resource.getrusage(resource.RUSAGE_SELF)
    snap = {"cpu_s": ru.ru_utime + ru.ru_stime, "involuntary_switches": ru.ru_nivcsw,
            "voluntary_switches": ru.ru_nvcsw}
    try:
        with open("/sys/fs/cgroup/cpu.stat") as f:
            for line in f:
                k, v = line.split()
                if k in ("nr_throttled", "throttled_usec", "nr_periods"):
                    snap[k] = int(v)
    except (OSError, ValueError):
        pass
    return snap


def host_cpu_delta(a, b, wall_s):
    d = {k: b[k] - a[k] for k in a if k in b}
    d["cpu_cores_busy"] = d.pop("cpu_s") / max(wall_s, 1e-9)
    try:
        with open("/sys/fs/cgroup/cpu.max") as f:
            d["cgroup_cpu_max"] = f.read().strip()
    except OSError:
        pass
    return d


def trace_steady_rate(tr, keys, lo=0.1, hi=0.9):
    """Galaxies per second completed while the cumulative completed count
    goes from lo to hi of the total: the server's rate with the start-up
    (lanes filling, micro-batches growing) and the drain left out."""
    import numpy as np
    if len(tr) < 4:
        return None
    col = {k: i for i, k in enumerate(keys)}
    tr = tr[np.argsort(tr[:, col["done_ms"]], kind="stable")]
    cum = np.cumsum(tr[:, col["galaxies"]])
    a = int(np.searchsorted(cum, lo * cum[-1]))
    b = int(np.searchsorted(cum, hi * cum[-1]))
    if b <= a:
        return None
    dt = (tr[b, col["done_ms"]] - tr[a, col["done_ms"]]) / 1e3
    return float((cum[b] - cum[a]) / dt) if dt > 0 else None


def trace_episode(tr, keys, before=4):
    """The micro-batch that took longest from admission to completion, the
    ones admitted just before it, and the largest gap between admissions."""
    import numpy as np
    if len(tr) == 0:
        return None
    col = {k: i for i, k in enumerate(keys)}
    tr = tr[np.argsort(tr[:, col["admit_ms"]], kind="stable")]
    span = tr[:, col["done_ms"]] - tr[:, col["admit_ms"]]
    w = int(np.argmax(span))
    rows = tr[max(0, w - before):w + 1]
    gaps = np.diff(tr[:, col["admit_ms"]])
    return {"columns": list(keys), "rows": [[round(float(v), 3) for v in r] for r in rows],
            "admission_to_done_ms": round(float(span[w]), 3),
            "max_admission_gap_ms": round(float(gaps.max()), 3) if len(gaps) else 0.0,
            "batches_over_5ms_device": int((tr[:, col["device_ms"]] > 5.0).sum())}


def extra_serving(tables, device, full_ms=500.0, half_window_s=10.0, single_ms=200.0, max_side=256,
                  kernel_bound=None):
    """1000 concurrent fits of 512 galaxies (Sersic, sizes as the mixed
    workload), render + gradient requests of 1-512 galaxies with Poisson
    arrivals, 64 PSFs resident, 16 GB admission budget.  Runs the offered
    load (20k galaxies/ms for full_ms, which saturates the server and gives
    its capacity), then a fresh request stream at half that capacity for
    half_window_s seconds (the latency measurement), then the
    one-launch-per-request form on the first single_ms of that stream."""
    import numpy as np
    import torch
    from paper_2012_15797_gb300.renderer import Renderer
    from paper_2012_15797_gb300.serving import Server, make_fits
    from workloads import psf_set, serving_workload

    fits, arrival_ms, reqs = serving_workload(n_fits=1000, duration_ms=full_ms, max_side=max_side)
    r = Renderer(tables, psf_set(64), device=device)
    state = make_fits(r, fits)
    torch.cuda.synchronize()

    def run(reqs, times_s, **cfg):
        gal = np.array([len(q[2]) for q in reqs], dtype=np.int64)
        srv = Server(r, **cfg)
        for st in state:
            srv.add_fit(**st)
        warm = min(300, len(reqs))
        t, k = srv.replay(reqs[:warm], np.zeros(warm))
        srv.wait_replayed(t, k)
        srv.timing(reset=True)
        h0 = host_cpu_snapshot()
        t0 = time.perf_counter()
        t, k = srv.replay(reqs, times_s)
        lat = srv.wait_replayed(t, k)
        wall = time.perf_counter() - t0
        host = host_cpu_delta(h0, host_cpu_snapshot(), wall)
        stats = srv.stats()
        breakdown = srv.timing()
        tr = srv.trace()
        episode = trace_episode(tr, Server.TRACE_KEYS)
        steady = trace_steady_rate(tr, Server.TRACE_KEYS)
        srv.close()
        return {"achieved_galaxies_per_s": float(gal.sum() / wall), "steady_galaxies_per_s": steady,
                "requests": len(reqs),
                "window_s": float(times_s[-1]), "offered_galaxies_per_s": float(gal.sum() / max(times_s[-1], 1e-9)),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "p999_ms": float(np.percentile(lat, 99.9) * 1e3), "max_ms": float(lat.max() * 1e3),
                "mean_ms": float(lat.mean() * 1e3), "micro_batches": stats["batches"] - 1,
                "largest_micro_batch": stats["max_batch_galaxies"], "max_lanes_in_flight": stats["max_lanes_in_flight"],
                "breakdown": breakdown, "slowest_batch": episode, "host": host}

    cfg = dict(budget_bytes=16 << 30, lanes=4, max_batch_galaxies=32768)
    full = run(reqs, arrival_ms / 1e3, **cfg)
    cap = full["achieved_galaxies_per_s"]
    _, half_ms, half_reqs = serving_workload(n_fits=1000, max_side=max_side, rate_per_ms=0.5 * cap / 1e3,
                                             duration_ms=half_window_s * 1e3, request_seed=40)
    half = run(half_reqs, half_ms / 1e3, **cfg)
    k = int(np.searchsorted(half_ms, single_ms))
    single = run(half_reqs[:k], half_ms[:k] / 1e3, budget_bytes=16 << 30, lanes=1, max_batch_galaxies=0)
    r.close()
    return {"workload": f"1000 fits x 512 galaxies (Sersic n U(0.5, 6), sides <= {max_side}), 64 PSFs, "
                        f"render + gradient requests of U{{1..512}} galaxies, Poisson arrivals; offered 20k "
                        f"galaxies/ms for {full_ms:.0f} ms, then half the measured capacity for "
                        f"{half_window_s:.0f} s; 16 GB budget, 4 lanes",
            "unit": "galaxies rendered+grad/s; latency = submission to results on the host",
            "offered_load": full, "sustained_fraction_of_offered": cap / full["offered_galaxies_per_s"],
            "kernel_bound_galaxies_per_s": kernel_bound,
            "fraction_of_kernel_bound": (cap / kernel_bound) if kernel_bound else None,
            "steady_fraction_of_kernel_bound": (full["steady_galaxies_per_s"] / kernel_bound)
            if (kernel_bound and full["steady_galaxies_per_s"]) else None,
            "capacity_note": "capacity = galaxies / wall time of the saturated window (start-up and drain "
                             "included); steady = the rate while the middle 80% of its galaxies complete; "
                             "the half load is half the former",
            "kernel_bound_note": "render + adjoint kernel time of the 200k mixed batch (one graph launch of the "
                                 "forward, one adjoint call): the galaxies per second the kernels allow",
            "half_capacity_load": half, "one_launch_per_request_at_half_load": single}


# ----------------------------------------------------------------------------
# Distributed helpers (replicas).
# ----------------------------------------------------------------------------

def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != n_gpus and world > 1:
        raise SystemExit(f"--gpus {n_gpus} but WORLD_SIZE={world}")
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job units per second: every rank (replica) processes
    units_per_rank in the slowest rank's ms."""
    return world * units_per_rank / (ms / 1e3)


# ----------------------------------------------------------------------------
# Arms.
# ----------------------------------------------------------------------------

def workload_config(galaxies, world):
    """The workload both arms report."""
    return {"workload": f"{galaxies} galaxies x 64x64 patches per GPU per step: 50/50 exp (6 comp) / "
                        f"deV (10 comp), r_e log-U(0.3, 20) px, |e| U(0, 0.6), flux log-U(1, 1e4), "
                        f"offsets U[-0.5, 0.5), one 2-Gaussian PSF (sigma 1.5/3.0) + 3-Gaussian fit",
            "galaxies_per_step": galaxies * world, "patch": N_PATCH, "parallelism": "replicas",
            "l2": f"each step writes {galaxies * N_PATCH * N_PATCH * 4 / 1e9:.2f} GB of patches "
                  f"(> 129 MB L2), which evicts the {galaxies * PARAM_BYTES / 1e6:.1f} MB of parameters; "
                  f"no separate flush"}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    from paper_2012_15797_gb300 import capi
    from paper_2012_15797_gb300.build import build
    if rank == 0 or world == 1:
        build()
    barrier(world)
    from paper_2012_15797_gb300.renderer import Renderer, host_batch, to_device
    from workloads import single_psf, fixed_galaxies_64, load_profile_tables

    tables = load_profile_tables()
    psf = single_psf()
    gals = fixed_galaxies_64(args.galaxies)
    r = Renderer(tables, [psf], device=local)
    batch = to_device(gals, device=f"cuda:{local}")
    out = torch.empty(batch.total, dtype=torch.float32, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 0)):
        r.render(batch, out)
    r.sync_status()

    sampler = ClockSampler(local)
    sampler.start()
    capi.mog_set_timing(r.ctx, True)
    capi.mog_read_timing(r.ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        r.render(batch, out)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    capi.mog_set_timing(r.ctx, False)
    kms, kn = capi.mog_read_timing(r.ctx)
    r.sync_status()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world)
    value = job_throughput(args.galaxies * args.steps, world, ms_max)

    # end to end with host buffers, through the C-ABI call for host memory
    # (mog_render_batch_host: parameters copied in and patches copied out in
    # chunks pipelined over two streams).  The call is synchronous on the
    # library's own streams, so it is timed by the host clock around it.
    e2e = None
    if not args.no_e2e:
        host = host_batch(gals, pin=True)
        out_host = torch.empty(host[1], dtype=torch.float32).pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host[0].values())
        d2h = out_host.numel() * 4
        k2 = max(3, min(args.steps, 20))
        for _ in range(2):
            r.render_host(host, out_host)
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            r.render_host(host, out_host)
        e2e_ms = (time.perf_counter() - t0) * 1e3
        barrier(world)
        e2e_ms = max_over_ranks(e2e_ms, world)
        e2e = {"value": job_throughput(args.galaxies * k2, world, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k2,
               "api": "mog_render_batch_host: pinned host parameters in, pinned host patches out, chunks of "
                      "64 MiB of patches pipelined over two streams; host clock around the synchronous call"}
        r.sync_status()
        # what bounds it on this machine: one plain device-to-host copy of the
        # same bytes into the same pinned buffer
        copy_ms = _event_ms(lambda: out_host.copy_(out, non_blocking=True), 3, stream)
        gbs = d2h / (copy_ms / 1e3) / 1e9
        e2e["d2h_copy"] = {"gb_per_s": gbs, "ms": copy_ms,
                           "patches_per_s_bound": args.galaxies / (copy_ms / 1e3),
                           "fraction_of_bound": e2e["value"] / world / (args.galaxies / (copy_ms / 1e3)),
                           "numa_nodes": host_numa_nodes()}

    if rank != 0:
        r.close()
        return

    pipes = measure_pipes(r, local)

    # roofline of the dominant kernel (64 x 64 render), from live CUDA events
    props = torch.cuda.get_device_properties(local)
    pk = peaks(props.multi_processor_count)
    work = algorithmic_work(gals, tables, psf.mog.shape[0])
    k_ms = kms[1] / max(kn[1], 1)
    roof = roofline(work, k_ms, pk, "render_fwd_kernel<64>", traffic=recorded_traffic(args.galaxies))

    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args.galaxies, args.cpu_seconds)
    extra = None
    if world == 1 and not args.no_extra:
        ocpu = 0.0 if args.no_cpu else 8.0
        extra = {"mixed_sizes": extra_mixed(tables, local, args.extra_steps, pk, ocpu),
                 "render_grad": extra_render_grad(tables, psf, local, args.extra_steps, pk, ocpu),
                 "lanczos_shift": extra_lanczos(tables, psf, local, args.extra_steps),
                 "eigen_psf": extra_eigen(tables, psf, local, args.extra_steps),
                 "composite": extra_composite(tables, psf, local, args.extra_steps),
                 "sersic_gradient": extra_sersic_grad(tables, local, args.extra_steps),
                 "psf_fit": extra_psf_fit(tables, local),
                 "psf_create": extra_psf_create(tables, local),
                 "one_launch_per_galaxy": extra_per_galaxy(tables, psf, local),
                 "cufft_comparator": cufft_or_reason(tables, psf, local, args.extra_steps, pk)}
        bound = 200_000 / ((extra["mixed_sizes"]["ms_graph"] + extra["sersic_gradient"]["ms_grad6"]) / 1e3)
        extra["serving"] = extra_serving(tables, local, kernel_bound=bound)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args.galaxies, world),
        "real_space_component_fraction": work["real_fraction"],
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        # per step: plan_histogram, plan_scan, plan_scatter, galaxy_prep and
        # render_fwd_kernel<64> (the launch list in profiles/render_fwd_64_100k.md)
        "gpu_launches": args.steps * KERNELS_PER_RENDER, "clocks": clocks, "pipe_rates": pipes,
        "extra": extra,
    }
    print(json.dumps(line))
    r.close()


REF_PER_WORKER = 400   # galaxies per worker per step of the reference arm (about 0.25 s of FP64 work)


def _worker_range(args):
    start, count = args
    return _worker_render(range(start, start + count))


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    pool, cores = cpu_pool(args.galaxies)
    per = min(REF_PER_WORKER, max(1, args.galaxies // cores))
    try:
        pool.map(_worker_render, [range(i * 20, i * 20 + 20) for i in range(cores)])   # warm the workers
        nxt = 0

        def step():
            # one contiguous range of `per` galaxies per worker: one message each way per worker and step
            nonlocal nxt
            chunks = [((nxt + c * per) % (args.galaxies - per), per) for c in range(cores)]
            nxt = (nxt + cores * per) % args.galaxies
            return sum(n for n, _ in pool.map(_worker_range, chunks))

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        done = sum(step() for _ in range(args.steps))
        wall = time.perf_counter() - t0
    finally:
        pool.close()
        pool.join()
    value = done / wall
    sample = (f"{cores * per} galaxies per step ({per} consecutive ones per worker) of the 100k fixed-size batch "
              f"over {cores} spawn workers, FP64 numpy oracle")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": wall / max(args.steps, 1) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.galaxies, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_only(args):
    """Small single-workload runs for profilers (no JSON bench line)."""
    import torch
    if args.only == "pipes":
        from paper_2012_15797_gb300.build import build
        build()
        from paper_2012_15797_gb300.renderer import Renderer
        from workloads import load_profile_tables
        r = Renderer(load_profile_tables(), [])
        print(json.dumps(measure_pipes(r, 0)))
        r.close()
        return
    if args.only == "serving":
        from paper_2012_15797_gb300.build import build
        build()
        from workloads import load_profile_tables
        print(json.dumps(extra_serving(load_profile_tables(), 0)))
        return
    from paper_2012_15797_gb300.build import build
    build()
    from paper_2012_15797_gb300.renderer import Renderer, to_device
    from workloads import single_psf, fixed_galaxies_64, mixed_galaxies, psf_set, load_profile_tables
    tables = load_profile_tables()
    pos = None
    if args.only == "mixed":
        psfs = psf_set(8)
        gals = mixed_galaxies(args.galaxies, n_psf=8)
    elif args.only == "eigen":
        from workloads import eigen_positions, eigen_psf
        psfs = [single_psf(), eigen_psf()]
        gals = fixed_galaxies_64(args.galaxies)
        gals.psf[:] = 1
        pos = eigen_positions(len(gals))
    elif args.size:
        import numpy as np
        psfs = psf_set(16)
        mixed = mixed_galaxies(args.galaxies, n_psf=16)
        gals = mixed.subset(np.flatnonzero(mixed.size == args.size))
    else:
        psfs = [single_psf()]
        gals = fixed_galaxies_64(args.galaxies)
    r = Renderer(tables, psfs)
    b = to_device(gals, positions=pos)
    out = torch.empty(b.total, device="cuda")
    go = torch.randn(b.total, device="cuda") if args.only == "grad" else None

    def step():
        if args.only == "grad":
            r.render_backward(b, go)
        else:
            r.render(b, out, shift="lanczos" if args.only == "lanczos" else "phase")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    r.sync_status()
    print(json.dumps({"only": args.only, "galaxies": len(gals), "ms_per_step": (time.perf_counter() - t) / max(args.steps, 1) * 1e3}))
    r.close()


def main():
    args = parse_args()
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
