"""Host-side arithmetic of the benchmark, on CPU: the algorithmic bytes per
input sample of the PFB workload (int16 IQ in, the FP32 complex spectrum
out, the tone rows out), the batched workload's roof time (the sum over
streams of max(HBM time, compute time)), and that the committed ncu
summaries behind the reported DRAM traffic were taken on the kernel sources
as they are now (a kernel changed after its capture reports no traffic)."""
import math

import bench


def test_pfb_bytes_per_sample():
    # 4 B in (complex int16), 8 B of spectrum per sample (N bins per N
    # samples), 8 B per tone per frame of N samples
    assert bench.BYTES_PER_SAMPLE == 4 + 8 + 8 * 1000 / 4096 == 13.953125


def test_batch_roof_time_by_hand():
    hbm, bf16, _, _ = bench.measured_peaks()
    fp32 = bench.FP32_PEAK_TFLOPS
    specs = [{"kind": "pfb", "N": 4096, "T": 8, "tones": 1000},
             {"kind": "demod", "L": 4096, "D": 2048, "tones": 2048}]
    ns = [1 << 24, 1 << 22]
    r = bench.batch_roofline(specs, ns, 10.0)
    pfb = max((1 << 24) * (4 + 8 * 1000 / 4096) / (hbm * 1e9),
              (1 << 24) * (4 * 8 + 5 * 12) / (fp32 * 1e12))
    dem = max((1 << 22) * (4 + 8 * 2048 / 2048) / (hbm * 1e9),
              (1 << 22) * 8 * 4096 * 2048 / 2048 / (bf16 * 1e12))
    assert math.isclose(r["roof_ms"], (pfb + dem) * 1e3, rel_tol=1e-12)
    assert math.isclose(r["frac"], r["roof_ms"] / 10.0, rel_tol=1e-12)
    # the demodulation stream is tensor-bound; the tones-only PFB stream
    # (6 B per sample) is bound by its 92 FP32 flops per sample
    assert r["roof_ms_by_bound"]["demod_tensor"] > 0 and r["roof_ms_by_bound"]["pfb_fp32"] > 0
    assert r["roof_ms_by_bound"]["pfb_hbm"] == 0 and r["roof_ms_by_bound"]["demod_hbm"] == 0


def test_profiles_match_current_kernel_sources():
    pfb = bench.profile_traffic("pfb_tmem_sym_kernel_c2.md", bench.PFB_SOURCES)
    dem = bench.profile_traffic("demod3m_gemm_kernel_c3.md", bench.DEMOD_SOURCES)
    assert pfb is not None and dem is not None
    # the fused PFB moves no more than its algorithmic bytes per 2^28-sample push
    assert pfb <= bench.BYTES_PER_SAMPLE * (1 << 28)
