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
               "paper_1812_02200_gb300/csrc/dev_common.cuh"]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


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
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------- oracle
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
           "value": samples / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
           "rel_err_max_checked_tones": rel,
           "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_peak,
                        "unit": "TFLOP/s", "frac": achieved / bf16_peak,
                        "traffic": profile_traffic("demod_gemm_kernel_c3.md", DEMOD_SOURCES),
                        "tensor_pipe_tflops": 3 * achieved,
                        "note": "algorithmic flops = 8*L*tones/D per sample; the split-FP16 "
                                "scheme issues 3 MMA products per algorithmic product; "
                                "push time includes the rotation, pre-split and carry kernels",
                        "peak_kind": f"{peak_kind} dense bf16 (fp16 has the same nominal rate)"}}
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
    del out, x
    plan.close()
    return res


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
    value = ws * args.steps * samples_step / (ms_max * 1e-3) / 1e6
    kernel_ms = ms / args.steps          # fused kernel + the tiny carry-update kernel
    achieved = samples_step * BYTES_PER_SAMPLE / (kernel_ms * 1e-3) / 1e9
    traffic = profile_traffic("pfb_ring_kernel_c2.md", PFB_SOURCES)

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

    # -- oracle on the host cores, bounded sample (rank 0 only)
    cpu = None
    if rank == 0 and not args.no_cpu:
        nf = min(args.cpu_frames, F - TAPS)
        v, dt, s = oracle_pfb_rate(nf, c)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{nf} frames ({s} samples) of the workload, {dt:.1f} s"}

    demod = None
    if not args.no_demod:
        del full, tones
        torch.cuda.empty_cache()
        demod = run_demod(args, dev, stream, rank)

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
        "gpu_launches": 2 * args.steps,
        "gpu_launches_note": "fused PFB kernel + carry-update kernel per step",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "kernel": "pfb_ring_kernel<12,8>",
                     "bytes_per_sample": BYTES_PER_SAMPLE,
                     "peak_kind": f"{peak_kind} (STREAM copy)"},
        "plain_fp32": plain,
        "demod": demod,
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
    ap.add_argument("--log2-samples", type=int, default=28,
                    help="stream length (28 = the workload; smaller only for profiling)")
    ap.add_argument("--cpu-frames", type=int, default=32768)
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
