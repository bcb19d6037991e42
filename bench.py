#!/usr/bin/env python3
"""Benchmark of the readout DSP stage on GB300.

Default workload (one step = one push of the whole buffer through the C ABI):
  PFB at the paper-rate shape: 2^28 complex int16 samples, N = 4096 channels,
  T = 8 taps Kaiser(beta=9) windowed-sinc prototype, 1000 tones at random bin
  centres, full spectrum + tone bins out (FP32 FIR + FFT in the fused kernel).
Inputs (1 GiB) and outputs (2.5 GiB) are larger than L2, so no L2 flush is
needed between steps.

Also reported in the same JSON line: the plain FP32 GPU form (FP32 FIR +
cuFFT + gather) on the same input, the split-FP16 tensor-core demodulation
workload (2^27 samples, 2048 tones, L = 4096, D = 2048) when available, the
end-to-end rate through rfr_process_host with pinned host buffers, and the
FP64 oracle on the host cores (bounded sample).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import siggen  # noqa: E402

METRIC = ("input Ms/s per GB300 (PFB, demod) vs plain FP32 form at ≤1e-5 rel err; "
          "p99 latency")
UNIT = "Ms/s"
N_CHAN, TAPS, BETA, N_TONES = 4096, 8, 9.0, 1000
N_SAMPLES = 1 << 28
BYTES_PER_SAMPLE = 4 + 8 + 8.0 * N_TONES / N_CHAN    # in + full + tones (algorithmic)
DEMOD_L, DEMOD_D, DEMOD_TONES, DEMOD_FC = 4096, 2048, 2048, 40e3 / 200e6
DEMOD_SOURCES = ["paper_1812_02200_gb300/csrc/demod.cu", "paper_1812_02200_gb300/csrc/umma.cuh",
                 "paper_1812_02200_gb300/csrc/dev_common.cuh"]
PFB_SOURCES = ["paper_1812_02200_gb300/csrc/pfb_kernels.cu",
               "paper_1812_02200_gb300/csrc/fft_dev.cuh",
               "paper_1812_02200_gb300/csrc/dev_common.cuh",
               "paper_1812_02200_gb300/csrc/umma.cuh"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profile_value(name, paths, key):
    """A number from a committed ncu summary taken on the current source."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    with open(p) as f:
        txt = f.read()
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_v = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_v or m_sha.group(1) != source_sha(paths):
        return None
    return float(m_v.group(1))


def profile_traffic(name, paths):
    """Per-launch DRAM traffic from a committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_sha = re.search(r"source_sha:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != source_sha(paths):
        return None
    return float(m_tr.group(1))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get(
            "bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, v):
    """Largest value over the ranks (timing only; the data path shards with
    no collective)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(ws, steps, samples_per_rank_step, ms_max):
    """Whole-job Ms/s: every rank runs its own replica of the workload (weak
    scaling), so the job processes ws * steps * samples in the slowest rank's
    time."""
    return ws * steps * samples_per_rank_step / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------- oracle
def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the ISA)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip().lower() == "model name":
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


_POOL = None


def oracle_pool():
    """Process pool over every host core for the oracle (spawned processes:
    safe after the parent has touched the GPU)."""
    global _POOL
    if _POOL is None:
        import multiprocessing as mp

        import oracle
        oracle.build()                     # once, before the workers load it
        _POOL = mp.get_context("spawn").Pool(os.cpu_count() or 1)
        _POOL.map(_w_noop, range(4 * (os.cpu_count() or 1)))
    return _POOL


def _w_noop(_):
    return 0


def _w_demod(a):
    import oracle
    x, m0, L, D, h, words, k0, k1 = a
    return oracle.demod(x, L, D, h, words, k0, k1, m0=m0)


def _w_pfb_time(a):
    import oracle
    x, N, T, h, k0, k1, bins = a
    t0 = time.perf_counter()
    oracle.pfb(x, N, T, h, k_begin=k0, k_end=k1, bins=bins)
    return time.perf_counter() - t0


def oracle_pfb_rate_all_cores(frames_per_core: int, c):
    """The FP64 oracle on disjoint frame ranges of the workload, one range per
    host core, all at once; returns (Ms/s, wall seconds, samples, cores)."""
    pool = oracle_pool()
    cores = os.cpu_count() or 1
    _, h32 = __import__("oracle").pfb_prototype(N_CHAN, TAPS, "kaiser", BETA)
    h = h32.astype(np.float64)
    bins = np.array([__import__("oracle").word_to_bin(int(w), N_CHAN) for w in c["words"]], np.int32)
    tasks = []
    for i in range(cores):
        k0 = TAPS - 1 + i * frames_per_core
        s0 = (k0 + 1 - TAPS) * N_CHAN
        x = np.ascontiguousarray(c["x"][s0:(k0 + frames_per_core) * N_CHAN])
        tasks.append((x, N_CHAN, TAPS, h, TAPS - 1, TAPS - 1 + frames_per_core, bins))
    t0 = time.perf_counter()
    pool.map(_w_pfb_time, tasks, chunksize=1)
    dt = time.perf_counter() - t0
    samples = cores * frames_per_core * N_CHAN
    return samples / dt / 1e6, dt, samples, cores


def oracle_pfb_rate(sample_frames: int, c=None):
    """FP64 oracle on the first `sample_frames` frames of the workload, one
    host core; returns (Ms/s, seconds, samples)."""
    import oracle
    n = (sample_frames + TAPS - 1) * N_CHAN
    if c is None:
        c = siggen.c2(n=n)
    _, h32 = oracle.pfb_prototype(N_CHAN, TAPS, "kaiser", BETA)
    h = h32.astype(np.float64)
    bins = np.array([oracle.word_to_bin(int(w), N_CHAN) for w in c["words"]], np.int32)
    oracle.build()
    t0 = time.perf_counter()
    oracle.pfb(c["x"], N_CHAN, TAPS, h, k_begin=TAPS - 1, k_end=TAPS - 1 + sample_frames,
               bins=bins)
    dt = time.perf_counter() - t0
    samples = sample_frames * N_CHAN
    return samples / dt / 1e6, dt, samples


def pfb_full_spectrum_error(c, full, F, bins, h, slices=8, frames=32):
    """Full-spectrum error of the timed configuration against the FP64 oracle
    on `slices` runs of `frames` frames spread over the stream, per channel c
    over those frames: strict ||y_c - y*_c|| / ||y*_c|| (maxima over the tone
    channels and over the noise-only channels) and the same divided by
    max(own, RMS channel norm)."""
    import oracle
    got, ref = [], []
    for i in range(slices):
        a = min(F - frames, i * (F // slices))
        ref.append(oracle.pfb(c["x"], N_CHAN, TAPS, h, k_begin=a, k_end=a + frames)["full"])
        got.append(full[a:a + frames].cpu().numpy())
    g, r = np.concatenate(got), np.concatenate(ref)
    num = np.linalg.norm(g - r, axis=0)
    own = np.maximum(np.linalg.norm(r, axis=0), 1e-300)
    rms = np.sqrt(np.mean(own ** 2))
    tone = np.zeros(N_CHAN, bool)
    tone[np.asarray(bins, int)] = True
    strict = num / own
    return {"frames_checked": slices * frames, "channels": N_CHAN,
            "strict_tone_max": float(strict[tone].max()), "strict_noise_max": float(strict[~tone].max()),
            "strict_noise_median": float(np.median(strict[~tone])),
            "rms_norm_max": float((num / np.maximum(own, rms)).max()),
            "note": "strict per-channel ratio; noise-only channels are ~1e-3 of the tone power, so FP32 "
                    "rounding of the strong channels dominates their strict ratio"}


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return
    frames = max(16, int(args.ref_frames))
    c = siggen.c2(n=(frames + TAPS - 1) * N_CHAN)
    for _ in range(args.warmup):
        oracle_pfb_rate(frames, c)
    times = []
    samples = 0
    for _ in range(args.steps):
        _, dt, samples = oracle_pfb_rate(frames, c)
        times.append(dt)
    tot = float(np.sum(times))
    val = args.steps * samples / tot / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "PFB N=4096 T=8 Kaiser(9) 1000 tones (2^28-sample stream; "
                               f"each step a {frames}-frame sample)", "samples_per_step": samples},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{frames} frames x 4096 samples of the workload, after warm-up"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------- demod
def run_demod(args, dev, stream, rank):
    """Workload 3: 2^27 samples, 2048 off-bin tones, L=4096 Blackman-sinc
    40 kHz, D=2048 -> 65536 frames x 2048 tones, split-FP16 tensor cores."""
    import torch

    from paper_1812_02200_gb300 import rfr
    _, bf16_peak, _, peak_kind = measured_peaks()
    t0 = time.time()
    c = siggen.c3(n=1 << args.demod_log2_samples)
    log(f"[bench] generated demod input in {time.time() - t0:.1f}s")
    x = torch.from_numpy(c["x"]).to(dev)
    plan = rfr.Plan(0, DEMOD_L, window="blackman", cutoff=DEMOD_FC, words=c["words"],
                    decimation=DEMOD_D)
    tune_ms = plan.autotune(x.shape[0], use_cache=False)      # result-neutral choices
    F = plan.frames_for(x.shape[0])
    out = torch.empty((DEMOD_TONES, F), dtype=torch.complex64, device=dev)
    plan.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    rel = None
    plain_rel = None
    sel = np.concatenate([np.argsort(c["amps"])[:4], [0, 1000]])
    fr = [(0, 4), (F // 2, F // 2 + 4), (F - 4, F)]
    if rank == 0 and not args.no_check:
        import oracle
        h = oracle.lowpass("blackman", DEMOD_L, DEMOD_FC)
        refs = [oracle.demod(c["x"], DEMOD_L, DEMOD_D, h, c["words"][sel], a, b) for a, b in fr]
        got = np.concatenate([out[sel, a:b].cpu().numpy() for a, b in fr], axis=1)
        ref = np.concatenate(refs, axis=1)
        rel = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    all_tones = None
    if rank == 0 and not args.no_check and not args.no_cpu:
        all_tones = demod_all_tones_error(c, out, F, args.demod_check_slices)
    for _ in range(2):
        plan.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    k = max(3, args.steps // 4)
    e0.record(stream)
    for _ in range(k):
        plan.push_into(x, tones=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / k
    samples = x.shape[0]
    flops = 8.0 * DEMOD_L * DEMOD_TONES / DEMOD_D * samples      # complex MACs x 8
    achieved = flops / (ms * 1e-3) / 1e12
    res = {"workload": "demod: 2^%d complex int16 samples, 2048 off-bin tones, L=4096 "
                       "Blackman-sinc 40 kHz, D=2048" % args.demod_log2_samples,
           "form": "Gauss three-product split-FP16 tensor-core GEMM (plan default for D %% 64 == 0)",
           "tune": plan.tune(),
           "value": samples / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "rel_err_max_checked_tones": rel,
           "rel_err_all_tones": all_tones,
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_peak,
                        "unit": "TFLOP/s", "frac": achieved / bf16_peak,
                        "traffic": profile_traffic("demod3m_gemm_kernel_c3.md", DEMOD_SOURCES),
                        "tensor_pipe_tflops": 2.25 * achieved,
                        "note": "algorithmic flops = 8*L*tones/D per sample; the default Gauss "
                                "form issues 3 real products per complex MAC, each as 3 split-FP16 "
                                "MMAs (2.25x the algorithmic flops on the tensor pipe); push time "
                                "includes the rotation, pre-split and carry kernels",
                        "peak_kind": f"{peak_kind} dense bf16 (fp16 has the same nominal rate)"}}
    # -- the other cluster form of the same GEMM (two-CTA clusters sharing
    # the frame tiles by multicast, or one CTA per tile), same tile and raster
    tn = plan.tune()
    pp = rfr.Plan(0, DEMOD_L, window="blackman", cutoff=DEMOD_FC, words=c["words"], decimation=DEMOD_D)
    pp.set_tone_tile(tn["tone_tile"] or 128)
    pp.set_demod_pair(not tn["pair"])
    pp.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(k):
        pp.push_into(x, tones=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    msp = e0.elapsed_time(e1) / k
    res["single_cta" if tn["pair"] else "pair_clusters"] = {
        "value": samples / (msp * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": msp,
        "note": "the same GEMM with one CTA per tile" if tn["pair"] else
                "the same GEMM in two-CTA clusters sharing each frame tile by TMA multicast"}
    pp.close()
    # -- the same three-product GEMM with the FP16 split fused into its
    # producer warps (no pre-split kernel; each A tile converted once per tone
    # tile and product)
    pf = rfr.Plan(0, DEMOD_L, window="blackman", cutoff=DEMOD_FC, words=c["words"], decimation=DEMOD_D)
    pf.set_tone_tile(plan.tune()["tone_tile"] or 128)
    pf.set_fused_presplit(True)
    pf.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(2):
        pf.push_into(x, tones=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    msf = e0.elapsed_time(e1) / 2
    res["fused_presplit"] = {"value": samples / (msf * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": msf,
                             "note": "pre-split fused into two producer warps of the GEMM: no 12 B/sample "
                                     "pass through HBM, but every A tile is converted once per tone tile and "
                                     "product (48 times per sample at 2048 tones)"}
    pf.close()
    # -- the four-product (real-embedding) form of the same contraction
    p4 = rfr.Plan(0, DEMOD_L, window="blackman", cutoff=DEMOD_FC, words=c["words"], decimation=DEMOD_D)
    p4.set_demod_products(4)
    p4.autotune(x.shape[0], use_cache=False)                     # raster order, as above
    p4.push_into(x, tones=out, stream=stream)                     # first push: frames from sample 0
    torch.cuda.synchronize(dev)
    rel4 = None
    if rank == 0 and not args.no_check:
        got = np.concatenate([out[sel, a:b].cpu().numpy() for a, b in fr], axis=1)
        rel4 = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
    for _ in range(2):
        p4.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(k):
        p4.push_into(x, tones=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms4 = e0.elapsed_time(e1) / k
    a4 = flops / (ms4 * 1e-3) / 1e12
    res["four_products"] = {"value": samples / (ms4 * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms4,
                            "rel_err_max_checked_tones": rel4,
                            "roofline": {"bound": "tensor", "achieved": a4, "peak": bf16_peak, "unit": "TFLOP/s",
                                         "frac": a4 / bf16_peak, "tensor_pipe_tflops": 3.0 * a4,
                                         "note": "real embedding: 4 real products per complex MAC, 3 split MMAs each"},
                            "tune": p4.tune(), "three_product_speedup": ms4 / ms}
    p4.close()
    if not args.no_plain:
        plan.plain_oneshot(x, tones=out, stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        plan.plain_oneshot(x, tones=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1)
        if rank == 0 and not args.no_check:
            got = np.concatenate([out[sel, a:b].cpu().numpy() for a, b in fr], axis=1)
            plain_rel = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        res["plain_fp32"] = {"value": samples / (pms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pms,
                             "form": "FP32 CUDA-core tiled kernel over the Toeplitz view",
                             "rel_err_max_checked_tones": plain_rel,
                             "speedup_of_tensor_path": pms / ms}
        # the library GEMM form: cublasCgemm (pedantic FP32) on the materialised Toeplitz matrix
        plan.plain_oneshot(x, tones=out, stream=stream, form=rfr.PLAIN_CGEMM)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        plan.plain_oneshot(x, tones=out, stream=stream, form=rfr.PLAIN_CGEMM)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        gms = e0.elapsed_time(e1)
        cg_rel = None
        if rank == 0 and not args.no_check:
            got = np.concatenate([out[sel, a:b].cpu().numpy() for a, b in fr], axis=1)
            cg_rel = float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))
        res["plain_fp32_cgemm"] = {"value": samples / (gms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": gms,
                                   "form": "cublasCgemm, pedantic FP32, on the Toeplitz matrix materialised "
                                           "in 512 MiB frame chunks, then the rotation kernel",
                                   "fp32_tflops": flops / (gms * 1e-3) / 1e12,
                                   "rel_err_max_checked_tones": cg_rel,
                                   "speedup_of_tensor_path": gms / ms}
    if rank == 0 and not args.no_cpu:
        # FP64 oracle on a bounded sample: all 2048 tones over 32 frames
        import oracle
        h = oracle.lowpass("blackman", DEMOD_L, DEMOD_FC)
        t0 = time.perf_counter()
        oracle.demod(c["x"], DEMOD_L, DEMOD_D, h, c["words"], 100, 132)
        dt = time.perf_counter() - t0
        res["cpu_baseline"] = {"value": 32 * DEMOD_D / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"all 2048 tones x 32 frames ({32 * DEMOD_D} input samples), {dt:.1f} s"}
    del out, x
    plan.close()
    return res


def demod_all_tones_error(c, out, F, slices, frames=4):
    """Per-tone relative RMS error of ALL tones of the demodulation workload
    against the FP64 oracle, over `slices` runs of `frames` frames spread
    across the stream, the oracle spread over every host core (each task one
    frame run x 256 tones, given only the samples it reads, at their absolute
    origin)."""
    import oracle
    h = oracle.lowpass("blackman", DEMOD_L, DEMOD_FC)
    pool = oracle_pool()
    starts = [min(F - frames, i * (F // slices)) for i in range(slices)]
    tasks, keys = [], []
    nt = len(c["words"])
    for a in starts:
        m0 = max(0, (a + 1) * DEMOD_D - DEMOD_L)
        xs = np.ascontiguousarray(c["x"][m0:(a + frames) * DEMOD_D])
        for t0 in range(0, nt, 256):
            tasks.append((xs, m0, DEMOD_L, DEMOD_D, h, c["words"][t0:t0 + 256], a, a + frames))
            keys.append((a, t0))
    t_0 = time.perf_counter()
    res = pool.map(_w_demod, tasks, chunksize=1)
    dt = time.perf_counter() - t_0
    ref = np.zeros((nt, slices * frames), np.complex128)
    for (a, t0), r in zip(keys, res):
        j = starts.index(a)
        ref[t0:t0 + r.shape[0], j * frames:(j + 1) * frames] = r
    got = np.concatenate([out[:, a:a + frames].cpu().numpy() for a in starts], axis=1)
    e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return {"tones": nt, "frames_checked": slices * frames, "max": float(e.max()),
            "median": float(np.median(e)), "p99": float(np.percentile(e, 99)),
            "oracle_seconds": dt, "cores": os.cpu_count() or 1}


# ------------------------------------------------------------------- chirp
def run_chirp(args, dev, stream):
    """Chirped readout (Sec. III.C): synthesis of a 2^28-sample transmit chirp
    on the GPU (HBM-bound: 4 B written per sample), and demodulation of a
    2^26-sample stream against 8 chirps (L = 4096 Blackman, D = 2048)."""
    import torch

    from paper_1812_02200_gb300 import rfr
    hbm_peak = measured_peaks()[0]
    fs = 200e6
    s0, r0 = rfr.freq_to_word(-90e6, fs), rfr.chirp_rate_word(1.8e8 / 1.34, fs)   # -90..+90 MHz in 1.34 s
    n = 1 << 28
    tx = torch.empty((n, 2), dtype=torch.int16, device=dev)
    rfr.chirp_synthesize(s0, r0, 8000.0, 0, tx, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(5):
        rfr.chirp_synthesize(s0, r0, 8000.0, i * n, tx, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_syn = e0.elapsed_time(e1) / 5
    del tx
    r = np.random.default_rng(3)
    sw = [rfr.freq_to_word(f, fs) for f in r.uniform(-80e6, 80e6, 8)]
    rw = [rfr.chirp_rate_word(k, fs) for k in r.uniform(-5e13, 5e13, 8)]
    c = siggen.c3(n=1 << 26, n_tones=256)
    x = torch.from_numpy(c["x"]).to(dev)
    plan = rfr.Plan.chirp(DEMOD_L, sw, rw, window="blackman", cutoff=DEMOD_FC, decimation=DEMOD_D)
    F = plan.frames_for(x.shape[0])
    out = torch.empty((8, F), dtype=torch.complex64, device=dev)
    plan.push_into(x, tones=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(3):
        plan.push_into(x, tones=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_dem = e0.elapsed_time(e1) / 3
    res = {"synthesis": {"workload": "2^28-sample complex int16 chirp, -90..+90 MHz sweep at 200 Ms/s",
                         "value": n / (ms_syn * 1e-3) / 1e6, "unit": UNIT, "ms": ms_syn,
                         "roofline": {"bound": "hbm", "achieved": 4.0 * n / (ms_syn * 1e-3) / 1e9,
                                      "peak": hbm_peak, "unit": "GB/s",
                                      "frac": 4.0 * n / (ms_syn * 1e-3) / 1e9 / hbm_peak}},
           "demod": {"workload": "2^26 samples against 8 chirps, L=4096 Blackman-sinc, D=2048",
                     "value": x.shape[0] / (ms_dem * 1e-3) / 1e6, "unit": UNIT, "ms": ms_dem}}
    lane_peak = 152 * 128 * 2.07e9
    i_syn = profile_value("chirp_kernels.md", CHIRP_SOURCES, "inst_per_sample_synth")
    i_dem = profile_value("chirp_kernels.md", CHIRP_SOURCES, "inst_per_tap_chirp_demod")
    if i_syn:
        a = n / (ms_syn * 1e-3) * i_syn
        res["synthesis"]["roofline_alu"] = {"bound": "alu", "achieved": a / 1e12, "peak": lane_peak / 1e12,
                                            "unit": "T lane-instructions/s", "frac": a / lane_peak,
                                            "inst_per_sample": i_syn,
                                            "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    if i_dem:
        evals = x.shape[0] * 8 * DEMOD_L / DEMOD_D
        a = evals / (ms_dem * 1e-3) * i_dem
        res["demod"]["roofline"] = {"bound": "alu", "achieved": a / 1e12, "peak": lane_peak / 1e12,
                                    "unit": "T lane-instructions/s", "frac": a / lane_peak,
                                    "inst_per_mixer_evaluation": i_dem,
                                    "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    plan.close()
    del x, out
    return res


# -------------------------------------------------------- transmit buffer
TX_SOURCES = ["paper_1812_02200_gb300/csrc/tx.cu"]
CHIRP_SOURCES = ["paper_1812_02200_gb300/csrc/chirp.cu"]


def run_tx(args, dev, stream, words):
    """Transmit buffer (Sec. III): 2^24 complex int16 samples of the workload's
    1000 tones at full scale (sum A = 8191 - 32), FP32 sines of the exact
    integer phase.  ALU-bound: the roofline is the FP32 lane-issue rate
    (152 SMs x 128 lanes x SM clock) over the instructions one tone-sample
    takes (from the committed ncu summary of the same source, if any)."""
    import torch

    from paper_1812_02200_gb300 import rfr
    r = siggen.rng_for(1812)
    amps = r.uniform(0.5, 1.0, len(words))
    amps *= (8191.0 - 32.0) / amps.sum()
    tx = rfr.Tx(words, amps, siggen.random_words(r, len(words)))
    n = 1 << 24
    out = torch.empty((n, 2), dtype=torch.int16, device=dev)
    tx.synthesize(0, out, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for i in range(reps):
        tx.synthesize(i * n, out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    ts = n * len(words) / (ms * 1e-3)
    res = {"workload": f"2^24 complex int16 samples of {len(words)} tones (sum A = 8159)",
           "value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "ms": ms,
           "tone_samples_per_s": ts, "error_bound_lsb": tx.error_bound}
    inst = profile_value("tx_synth_kernel.md", TX_SOURCES, "inst_per_tone_sample")
    if inst:
        peak = 152 * 128 * 2.07e9
        res["roofline"] = {"bound": "alu", "achieved": ts * inst / 1e12, "peak": peak / 1e12,
                           "unit": "T lane-instructions/s", "frac": ts * inst / peak,
                           "inst_per_tone_sample": inst,
                           "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    tx.close()
    del out
    return res


# ----------------------------------------------------------- any-N PFB
def run_large_n(args, dev, stream, x, words):
    """PFB beyond the fused kernels (Sec. III.A): Fig. 3's N = 10^5 and the
    section's largest, 10^7, with A_v = T = 4 and a Hamming window (four-step
    two-pass form), and the workload's N = 4096, T = 8 Kaiser(9) oversampled
    4x (hop 1024, the mixed-radix one-pass form); and the batched workload's
    power-of-two shapes whose FP32 delay line does not fit one SM's tensor
    memory (N = 16384 and 8192 with T = 8, direct kernel with its pre-sum
    FIR pass, and cluster kernel; N = 4096 T = 16 (pre-sum pass + TMEM
    kernel), N = 16384 T = 16 (pre-sum pass + direct kernel); Kaiser(9));
    each on the workload's 2^28-sample stream, full spectrum + its 1000 tones."""
    import torch

    from paper_1812_02200_gb300 import rfr
    hbm_peak = measured_peaks()[0]
    out = []
    n = x.shape[0]
    for N, T, win, hop, reps in ((100000, 4, "hamming", 100000, 5), (10 ** 7, 4, "hamming", 10 ** 7, 3),
                                 (4096, 8, "kaiser", 1024, 3), (16384, 8, "kaiser", 16384, 3),
                                 (8192, 8, "kaiser", 8192, 3),
                                 (4096, 16, "kaiser", 4096, 3), (16384, 16, "kaiser", 16384, 3)):
        plan = rfr.Plan(N, T, window=win, beta=BETA if win == "kaiser" else 0.0, words=words, full=True,
                        tones=True, decimation=hop)
        F = plan.frames_for(n)
        # pushes after the first may complete one more frame (residue)
        full = torch.empty((F + 1, N), dtype=torch.complex64, device=dev)
        tones = torch.empty((len(words), F + 1), dtype=torch.complex64, device=dev)
        plan.push_into(x, full, tones, stream=stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.push_into(x, full, tones, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        bps = 4.0 + (8.0 * N + 8.0 * len(words)) / hop
        gbs = bps * n / (ms * 1e-3) / 1e9
        wname = "Kaiser(9)" if win == "kaiser" else win.capitalize()
        res = {"workload": f"PFB N={N} T={T} {wname}" + (f" hop {hop}" if hop != N else "") +
                           f", 2^{int(np.log2(n))} complex int16 samples, full spectrum + {len(words)} tones",
               "value": n / (ms * 1e-3) / 1e6, "unit": UNIT, "ms": ms, "frames": F,
               "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                            "frac": gbs / hbm_peak, "bytes_per_sample": bps}}
        if N in (8192, 16384) and T <= 8:
            # the cluster kernel (clusters of N / 4096 CTAs) on the same stream
            pc = rfr.Plan(N, T, window=win, beta=BETA if win == "kaiser" else 0.0, words=words, full=True,
                          tones=True, decimation=hop)
            pc.set_pfb_cluster(True)
            pc.push_into(x, full, tones, stream=stream)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(reps):
                pc.push_into(x, full, tones, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            cms = e0.elapsed_time(e1) / reps
            res["cluster_kernel"] = {"value": n / (cms * 1e-3) / 1e6, "unit": UNIT, "ms": cms,
                                     "form": f"clusters of {N // 4096} CTAs, filtered slices exchanged through "
                                             "distributed shared memory (the default is the direct kernel)"}
            pc.close()
        if not args.no_plain and N <= 100000 and hop == N:
            # the plain FP32 form on the same stream: FP32 FIR kernel + cuFFT + gather
            plan.plain_oneshot(x, full, tones, stream=stream)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            plan.plain_oneshot(x, full, tones, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            pms = e0.elapsed_time(e1)
            res["plain_fp32"] = {"value": n / (pms * 1e-3) / 1e6, "unit": UNIT, "ms": pms,
                                 "form": "FP32 FIR kernel + cuFFT C2C batched + gather kernel"}
        out.append(res)
        plan.close()
        del full, tones
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------- batch
def make_spec_plan(rfr, spec, words, full=False):
    if spec["kind"] == "pfb":
        return rfr.Plan(spec["N"], spec["T"], window="kaiser", beta=BETA, words=words, full=full)
    return rfr.Plan(0, spec["L"], window="blackman", cutoff=DEMOD_FC, words=words, decimation=spec["D"])


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12     # FMA lanes x 2 flops x max SM clock


def batch_roofline(specs, ns, ms):
    """Roof time of the batched step = the sum over streams of each stream's
    own roof time: the larger of its HBM time (algorithmic bytes: 4 B in plus
    8 B per output value) and its compute time (PFB: 4T FIR + 5 log2 N FFT
    flops per sample at the FP32 FMA rate; demodulation: 8 L tones / D flops
    per sample at the measured dense bf16 rate)."""
    hbm, bf16, _, kind = measured_peaks()
    tot, parts = 0.0, {"pfb_hbm": 0.0, "pfb_fp32": 0.0, "demod_hbm": 0.0, "demod_tensor": 0.0}
    for sp, n in zip(specs, ns):
        if sp["kind"] == "pfb":
            t_b = n * (4.0 + 8.0 * sp["tones"] / sp["N"]) / (hbm * 1e9)
            t_c = n * (4.0 * sp["T"] + 5.0 * np.log2(sp["N"])) / (FP32_PEAK_TFLOPS * 1e12)
            parts["pfb_hbm" if t_b >= t_c else "pfb_fp32"] += max(t_b, t_c)
        else:
            t_b = n * (4.0 + 8.0 * sp["tones"] / sp["D"]) / (hbm * 1e9)
            t_c = n * 8.0 * sp["L"] * sp["tones"] / sp["D"] / (bf16 * 1e12)
            parts["demod_hbm" if t_b >= t_c else "demod_tensor"] += max(t_b, t_c)
        tot += max(t_b, t_c)
    return {"bound": "mixed", "roof_ms": tot * 1e3, "achieved_ms": ms, "frac": tot * 1e3 / ms,
            "roof_ms_by_bound": {k: v * 1e3 for k, v in parts.items()},
            "peak": {"hbm_gbs": hbm, "bf16_tflops": bf16, "fp32_tflops": FP32_PEAK_TFLOPS, "kind": kind},
            "note": "sum over streams of max(algorithmic bytes / HBM peak, algorithmic flops / compute "
                    "peak); frac = roof time / measured step time"}


def run_batch(args, dev, stream):
    """Workload 4: 24 mixed PFB / demodulation streams of 2^22..2^26 samples
    per step, one CUDA-graph launch per step, launch choices autotuned."""
    import torch

    from paper_1812_02200_gb300 import rfr
    t0 = time.time()
    specs = siggen.c4_specs()
    cases = [siggen.spec_input(sp) for sp in specs]
    log(f"[bench] generated batch inputs in {time.time() - t0:.1f}s")
    xs = [torch.from_numpy(c["x"]).to(dev) for c in cases]
    plans = [make_spec_plan(rfr, sp, c["words"]) for sp, c in zip(specs, cases)]
    seq_plans = [make_spec_plan(rfr, sp, c["words"]) for sp, c in zip(specs, cases)]
    # tune each stream shape once; the sequential comparison loads the same
    # choices from the cache file
    os.environ.setdefault("RFR_TUNE_CACHE", os.path.join(tempfile.gettempdir(), "rfr_tune_cache.json"))
    for p, q, x in zip(plans, seq_plans, xs):
        p.autotune(x.shape[0], use_cache=True)
        q.autotune(x.shape[0], use_cache=True)
    outs = [torch.empty((p.n_tones, p.frames_for(x.shape[0]) + 1), dtype=torch.complex64, device=dev)
            for p, x in zip(plans, xs)]
    batch = rfr.Batch(plans)
    samples = sum(x.shape[0] for x in xs)
    for _ in range(2):
        batch.push(xs, None, outs)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k = max(3, args.steps // 4)
    e0.record(stream)
    for _ in range(k):
        batch.push(xs, None, outs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_batch = e0.elapsed_time(e1) / k
    # the same streams as sequential per-stream pushes (no graph, one stream)
    for p, x, o in zip(seq_plans, xs, outs):
        p.push_into(x, tones=o, stream=stream)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(k):
        for p, x, o in zip(seq_plans, xs, outs):
            p.push_into(x, tones=o, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_seq = e0.elapsed_time(e1) / k
    # per-stream plain FP32 launches
    ms_plain = None
    if not args.no_plain:
        for p, x, o in zip(seq_plans, xs, outs):
            p.plain_oneshot(x, tones=o, stream=stream)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for p, x, o in zip(seq_plans, xs, outs):
            p.plain_oneshot(x, tones=o, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_plain = e0.elapsed_time(e1)
    st = batch.stats()
    roof = batch_roofline(specs, [x.shape[0] for x in xs], ms_batch)
    res = {"workload": "24 streams of 2^22..2^26 samples (log-uniform), 16 PFB "
                       "(N in {256..16384}, T in {4,8,16}, tones out) + 8 demodulation "
                       "(64..4096 tones, L in {1024,4096}, D in {512,2048})",
           "samples_per_step": samples,
           "value": samples / (ms_batch * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms_batch,
           "graph": st,
           "roofline": roof,
           "sequential_fused": {"value": samples / (ms_seq * 1e-3) / 1e6, "ms_per_step": ms_seq,
                                "batch_speedup": ms_seq / ms_batch},
           "plain_fp32_per_stream": None if ms_plain is None else
           {"value": samples / (ms_plain * 1e-3) / 1e6, "ms_per_step": ms_plain},
           "tune": [p.tune() for p in plans][:4] + ["..."]}
    batch.close()
    del outs, xs
    return res


# ------------------------------------------------------------------- serve
def run_serve(args, dev):
    """Workload 5: 32 readouts (plans drawn as in the batched workload),
    buffers of 1..32 MB arriving as Poisson processes, admission under a 40 GB
    device budget; p50/p99 latency from submit to completion and the
    sustained rate per offered load.  Two modes: host-resident input and
    output (pinned; the copies are part of each request) and device-resident
    (inputs and outputs already in device memory).  Each load point runs for
    args.serve_seconds of arrivals and is repeated; the spread of p99 over the
    repeats is reported."""
    import threading as th

    import torch

    from paper_1812_02200_gb300 import rfr
    specs = siggen.c5_specs()
    max_n = 8 << 20                      # 32 MB of complex int16
    t0 = time.time()
    host_x, dev_x, plans, outs, dev_outs = [], [], [], [], []
    for sp in specs:
        c = siggen.spec_input(sp, n=max_n)
        host_x.append(torch.from_numpy(c["x"]).pin_memory())
        dev_x.append(torch.from_numpy(c["x"]).to(dev))
        plans.append(make_spec_plan(rfr, sp, c["words"]))
    for p in plans:
        f = p.frames_for(max_n) + 2
        outs.append(torch.empty((max(p.n_tones, 1), 4 * f), dtype=torch.complex64).pin_memory())
        dev_outs.append(torch.empty((max(p.n_tones, 1), 4 * f), dtype=torch.complex64, device=dev))
    log(f"[bench] serve setup {time.time() - t0:.1f}s")
    srv = rfr.Server(plans, 40 << 30, max_n)
    # warm-up, outside the statistics: a small and a full-size buffer per
    # readout through the server in each mode (first launches of every plan's
    # kernels, first-use setup at both ends of the size range)
    n_warm = 0
    for r in range(len(specs)):
        for xs, os_ in ((host_x, outs), (dev_x, dev_outs)):
            srv.submit(r, xs[r][: 1 << 18], tones=os_[r], frame_offset=0, tag=(1 << 40) + n_warm)
            srv.submit(r, xs[r], tones=os_[r], frame_offset=os_[r].shape[1] // 4, tag=(1 << 41) + n_warm)
            n_warm += 2
    got = 0
    t_w = time.time()
    while got < n_warm and time.time() - t_w < 180:
        got += len(srv.poll(1024, wait_ms=20))
    loads = [float(v) for v in args.serve_loads.split(",") if v]
    rng = np.random.default_rng(55)
    mean_n = float(np.mean(siggen.c5_buffer_samples(np.random.default_rng(1), 1 << 16)))

    def one_point(load, xs, os_):
        rate = load * 1e9 / mean_n / len(specs)          # buffers/s per readout
        dur = args.serve_seconds
        arr = []
        for r in range(len(specs)):
            t = rng.exponential(1.0 / rate)
            while t < dur:
                arr.append((t, r))
                t += rng.exponential(1.0 / rate)
        arr.sort()
        sizes = siggen.c5_buffer_samples(rng, len(arr))
        done = []
        stop = [False]

        def poller():
            while not stop[0] or len(done) < len(arr):
                done.extend(srv.poll(1024, wait_ms=20))
                if stop[0] and len(done) >= len(arr):
                    break

        pt = th.Thread(target=poller, daemon=True)
        pt.start()
        slot = [0] * len(specs)
        base = rfr.now_us()
        for tag, ((t, r), n) in enumerate(zip(arr, sizes)):
            # sleep until just before the arrival, then spin: the submitting
            # thread leaves the host cores to the server's worker and poller
            ahead = t * 1e6 - (rfr.now_us() - base)
            if ahead > 300.0:
                time.sleep((ahead - 200.0) * 1e-6)
            while rfr.now_us() - base < t * 1e6:
                pass
            # four rotating output regions per readout, each large enough for
            # the frames of the largest buffer
            off = (slot[r] % 4) * (os_[r].shape[1] // 4)
            slot[r] += 1
            srv.submit(r, xs[r][: int(n)], tones=os_[r], frame_offset=off, tag=tag)
        t_sub_end = rfr.now_us() - base
        stop[0] = True
        pt.join(timeout=180)
        lat = np.array([d["t_done_us"] - d["t_submit_us"] for d in done]) / 1e3
        wait = np.array([d["t_admit_us"] - d["t_submit_us"] for d in done]) / 1e3
        t_first = min(d["t_submit_us"] for d in done)
        t_last = max(d["t_done_us"] for d in done)
        tot = float(sum(d["samples"] for d in done))
        bad = sum(1 for d in done if d["status"] != 0)
        return {"buffers": len(done), "failed": bad,
                "offered_realised_gsps": tot / (t_sub_end * 1e-6) / 1e9,
                "sustained_gsps": tot / ((t_last - t_first) * 1e-6) / 1e9,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max()), "admit_wait_p50_ms": float(np.percentile(wait, 50)),
                "admit_wait_p99_ms": float(np.percentile(wait, 99))}

    modes = {}
    for mode, xs, os_, reps in (("host_pinned", host_x, outs, args.serve_reps),
                                ("device_resident", dev_x, dev_outs, args.serve_reps_device)):
        pts = []
        for load in loads:
            runs = [one_point(load, xs, os_) for _ in range(max(1, reps))]
            p99 = [r["p99_ms"] for r in runs]
            pt = {"offered_gsps": load, "repeats": len(runs),
                  "buffers": int(sum(r["buffers"] for r in runs)),
                  "failed": int(sum(r["failed"] for r in runs)),
                  "offered_realised_gsps": float(np.mean([r["offered_realised_gsps"] for r in runs])),
                  "sustained_gsps": float(np.mean([r["sustained_gsps"] for r in runs])),
                  "p50_ms": float(np.median([r["p50_ms"] for r in runs])),
                  "p99_ms": float(np.median(p99)), "p99_ms_min": float(min(p99)),
                  "p99_ms_max": float(max(p99)), "max_ms": float(max(r["max_ms"] for r in runs)),
                  "admit_wait_p50_ms": float(np.median([r["admit_wait_p50_ms"] for r in runs])),
                  "admit_wait_p99_ms": float(np.median([r["admit_wait_p99_ms"] for r in runs]))}
            pts.append(pt)
            log(f"[bench] serve {mode} load {load}: {pt}")
        modes[mode] = pts
    st = srv.stats()
    srv.close()
    return {"workload": "32 readouts (plans as the batched workload), Poisson arrivals, "
                        "buffers log-uniform 1..32 MB, 40 GB budget",
            "points": modes["host_pinned"], "device_resident": modes["device_resident"],
            "peak_device_bytes": st["peak_bytes"], "seconds_per_point": args.serve_seconds,
            "note": "points: pinned host input and output (the copies are part of each request); "
                    "device_resident: inputs and outputs in device memory.  offered_realised is the "
                    "submitted samples over the submission window (Poisson draws make it differ from "
                    "the nominal load); sustained is the completed samples from first submit to last "
                    "completion, which includes the last buffer's latency."}


# --------------------------------------------------------------------- ours
def run_ours(args, ws, rank, local):
    import torch

    from paper_1812_02200_gb300 import rfr

    dev = torch.device("cuda", local if ws > 1 else 0)
    hbm_peak, bf16_peak, bf16_sus, peak_kind = measured_peaks()
    t_gen = time.time()
    c = siggen.c2(n=1 << args.log2_samples)
    log(f"[bench] generated c2 input in {time.time() - t_gen:.1f}s")
    x = torch.from_numpy(c["x"]).to(dev)
    plan = rfr.Plan(N_CHAN, TAPS, window="kaiser", beta=BETA, words=c["words"])
    F = plan.frames_for(x.shape[0])
    full = torch.empty((F, N_CHAN), dtype=torch.complex64, device=dev)
    tones = torch.empty((N_TONES, F), dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)

    # -- parity spot check of the configuration that is timed (first push)
    plan.push_into(x, full, tones, stream=stream)
    torch.cuda.synchronize(dev)
    rel_err = None
    full_err = None
    if rank == 0 and not args.no_check:
        import oracle
        _, h32 = oracle.pfb_prototype(N_CHAN, TAPS, "kaiser", BETA)
        bins = plan.bins()
        errs = []
        for a, b in [(0, 4), (F // 2, F // 2 + 4), (F - 4, F)]:
            ref = oracle.pfb(c["x"], N_CHAN, TAPS, h32.astype(np.float64), k_begin=a, k_end=b,
                             bins=bins, want_full=False)["tones"]
            got = tones[:, a:b].cpu().numpy()
            errs.append(float(np.max(np.linalg.norm(got - ref, axis=1) /
                                     np.linalg.norm(ref, axis=1))))
        rel_err = max(errs)
        full_err = pfb_full_spectrum_error(c, full, F, plan.bins(), h32.astype(np.float64))

    # -- timed region: K pushes (the stream continues; each push = F frames)
    for _ in range(args.warmup):
        plan.push_into(x, full, tones, stream=stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local if ws > 1 else int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or 0))
    clocks.start()
    time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.push_into(x, full, tones, stream=stream)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ws, ms)
    samples_step = x.shape[0]
    value = aggregate_rate(ws, args.steps, samples_step, ms_max)
    kernel_ms = ms / args.steps          # fused kernel + the tiny carry-update kernel
    achieved = samples_step * BYTES_PER_SAMPLE / (kernel_ms * 1e-3) / 1e9
    traffic = profile_traffic("pfb_tmem_sym_kernel_c2.md", PFB_SOURCES)

    # -- plain FP32 GPU form on the same input (FP32 FIR + cuFFT + gather)
    plain = None
    if not args.no_plain:
        plan.plain_oneshot(x, full, tones, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kp = max(3, args.steps // 2)
        e0.record(stream)
        for _ in range(kp):
            plan.plain_oneshot(x, full, tones, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        pms = e0.elapsed_time(e1) / kp
        plain = {"value": samples_step / (pms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": pms,
                 "form": "FP32 FIR kernel + cuFFT C2C batched + gather kernel",
                 "speedup_of_fused": pms / kernel_ms}

    # -- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(c["x"]).pin_memory()
        fh = torch.empty((F, N_CHAN), dtype=torch.complex64).pin_memory()
        th = torch.empty((N_TONES, F), dtype=torch.complex64).pin_memory()
        plan.process_host(xh, fh, th)
        ke = max(2, min(args.steps, 5))
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(ke):
            plan.process_host(xh, fh, th)
        dt = max_over_ranks(ws, (time.perf_counter() - t0) / ke)
        e2e = {"value": ws * samples_step / dt / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * 2),
               "d2h_bytes_per_step": int(fh.numel() * 8 + th.numel() * 8),
               "call": "rfr_process_host (pinned host in/out, chunked copies overlapped)"}

    # -- oracle on the host cores, bounded sample (rank 0 only): one core,
    # then every core on disjoint frame ranges
    cpu = None
    if rank == 0 and not args.no_cpu:
        nf = min(args.cpu_frames, F - TAPS)
        v, dt, s = oracle_pfb_rate(nf, c)
        cores = os.cpu_count() or 1
        fpc = max(16, min(args.cpu_frames_per_core, (F - TAPS) // cores))
        va, dta, sa, na = oracle_pfb_rate_all_cores(fpc, c)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nf} frames ({s} samples) of the workload, {dt:.1f} s",
               "value_all_cores": va, "cores_all": na,
               "sample_all_cores": f"{na} processes x {fpc} disjoint frames ({sa} samples), {dta:.1f} s wall",
               "cpu_model": cpu_model(), "nproc": cores}

    demod = None
    del full, tones
    torch.cuda.empty_cache()
    large_n = None if args.no_large_n else run_large_n(args, dev, stream, x, c["words"])
    txr = None if args.no_tx else run_tx(args, dev, stream, c["words"])
    if not args.no_demod:
        demod = run_demod(args, dev, stream, rank)
    chirp = None if args.no_chirp else run_chirp(args, dev, stream)
    batch = None if args.no_batch else run_batch(args, dev, stream)
    torch.cuda.empty_cache()
    serve = None if (args.no_serve or ws > 1) else run_serve(args, dev)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "PFB N=4096 T=8 Kaiser(9) windowed sinc, 1000 tones at random "
                               f"bin centres, 2^{args.log2_samples} complex int16 samples, "
                               "full spectrum + tones",
                   "samples_per_step": samples_step, "frames_per_step": F,
                   "l2": "inputs and outputs larger than L2 (no flush)",
                   "parallelism": f"replicas x{ws}"},
        "rel_err_max_tone": rel_err,
        "rel_err_full_strict": None if full_err is None else full_err["strict_noise_max"],
        "rel_err_full_rms": None if full_err is None else full_err["rms_norm_max"],
        "full_spectrum_error": full_err,
        "gpu_launches": 2 * args.steps,
        "gpu_launches_note": "fused PFB kernel (pfb_tmem_sym_kernel) + carry-update kernel per step",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "kernel": "pfb_tmem_sym_kernel (N=4096 T=8, symmetric taps, TMA-fed, FP32 delay line in TMEM)",
                     "bytes_per_sample": BYTES_PER_SAMPLE,
                     "peak_kind": f"{peak_kind} (STREAM copy)"},
        "plain_fp32": plain,
        "demod": demod,
        "batch": batch,
        "serve": serve,
        "chirp": chirp,
        "any_n_pfb": large_n,
        "tx": txr,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-demod", action="store_true")
    ap.add_argument("--demod-log2-samples", type=int, default=27)
    ap.add_argument("--demod-check-slices", type=int, default=16)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-chirp", action="store_true")
    ap.add_argument("--no-large-n", action="store_true")
    ap.add_argument("--no-tx", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-loads", default="0.5,1,2,5,10,15,20", help="offered loads, Gsamples/s")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--serve-reps", type=int, default=3)
    ap.add_argument("--serve-reps-device", type=int, default=1)
    ap.add_argument("--log2-samples", type=int, default=28,
                    help="stream length (28 = the workload; smaller only for profiling)")
    ap.add_argument("--cpu-frames", type=int, default=32768)
    ap.add_argument("--cpu-frames-per-core", type=int, default=4096)
    ap.add_argument("--ref-frames", type=int, default=2048)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_setup(args.gpus) if args.impl == "ours" else (
        int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)
    if ws > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
