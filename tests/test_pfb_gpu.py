"""GPU parity of the fused PFB kernel (Sec. III.A) against the FP64 oracle,
through the C ABI.  Tolerance: relative RMS error <= 1e-5 per tone channel,
and per full-spectrum channel relative to the RMS channel norm (FP32 FIR and
FFT have ~1e-7..1e-6 relative error; noise-only bins are ~1e3 times weaker
than tone bins, so their strict per-channel ratio is reported, not bounded)."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import STRICT_NOISE_BOUND, TOL, full_spectrum_errors, rel_channels_vs_rms, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _plan(lib, N, T, win, beta, words, full=True, tones=True):
    return lib.Plan(N, T, window=win, beta=beta, words=words, full=full, tones=tones)


def _oracle_taps(N, T, win, beta):
    _, h32 = oracle.pfb_prototype(N, T, win, beta)
    return h32.astype(np.float64)


def _run_gpu(plan, x_np, n_tones, N, full=True):
    x = torch.from_numpy(x_np).to(DEV)
    F = plan.frames_for(x.shape[0])
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV) if full else None
    to = torch.zeros((n_tones, F), dtype=torch.complex64, device=DEV) if n_tones else None
    got = plan.push_into(x, fo, to)
    torch.cuda.synchronize()
    assert got == F
    return (None if fo is None else fo.cpu().numpy()), (None if to is None else to.cpu().numpy())


def test_c1_full_size_parity(lib):
    """Workload 1: 2^20 samples, N=64, T=4 Hann, 16 tones, sigma 8, clipped."""
    c = siggen.c1()
    N, T = 64, 4
    plan = _plan(lib, N, T, "hann", 0.0, c["words"])
    bins = plan.bins()
    assert np.array_equal(bins, [oracle.word_to_bin(int(w), N) for w in c["words"]])
    assert np.array_equal(bins, c["bins"])
    h64p, h32p = plan.taps_table()
    h64o, h32o = oracle.pfb_prototype(N, T, "hann")
    ulp = np.abs(h32p.view(np.int32).astype(np.int64) - h32o.view(np.int32).astype(np.int64))
    assert ulp.max() <= 1
    assert np.allclose(h64p, h64o, rtol=1e-13, atol=1e-17)
    full, tones = _run_gpu(plan, c["x"], 16, N)
    ref = oracle.pfb(c["x"], N, T, h32o.astype(np.float64), bins=bins)
    e_t = rel_rows(tones, ref["tones"])
    e_f = rel_channels_vs_rms(full, ref["full"])
    fe = full_spectrum_errors(full, ref["full"], bins)
    print(f"c1 max tone rel err {e_t.max():.3e}, max full-channel err {e_f.max():.3e}; strict per-channel: "
          f"tone channels {fe['strict_tone_max']:.3e}, noise-only channels max {fe['strict_noise_max']:.3e} "
          f"(median {fe['strict_noise_median']:.3e})")
    assert e_t.max() < TOL
    assert e_f.max() < TOL
    assert fe["strict_tone_max"] < TOL and fe["strict_noise_max"] < STRICT_NOISE_BOUND
    assert np.array_equal(tones, full[:, bins].T)   # gather is an exact copy


CASES = [
    # N, T, window, beta, frames
    (16, 4, "hann", 0.0, 700),
    (32, 3, "hamming", 0.0, 500),
    (64, 1, "rect", 0.0, 400),
    (128, 8, "kaiser", 9.0, 400),
    (256, 5, "blackman", 0.0, 300),
    (512, 7, "hann", 0.0, 300),
    (1024, 8, "kaiser", 9.0, 300),
    (2048, 2, "hann", 0.0, 300),
    (4096, 8, "kaiser", 9.0, 400),
    (4096, 12, "kaiser", 9.0, 60),    # first-half FIR pass + TMEM kernel (taps padded to 16)
    (4096, 16, "hann", 0.0, 50),      # first-half FIR pass + TMEM kernel
    (1024, 16, "hann", 0.0, 80),      # DIRECT variant, FIR as a pre-sum pass
    (256, 12, "kaiser", 9.0, 120),    # DIRECT variant, T > 8 at small N
    (2048, 9, "hamming", 0.0, 60),    # DIRECT variant, pre-sum pass, odd T
    (8192, 4, "hann", 0.0, 40),       # DIRECT variant (N > 4096), pre-sum pass
    (8192, 8, "kaiser", 9.0, 30),     # DIRECT variant, pre-sum pass
    (16384, 2, "kaiser", 9.0, 30),    # DIRECT variant, taps padded to 4, FIR in the kernel
    (16384, 12, "kaiser", 9.0, 20),   # DIRECT variant, largest N, T > 8, pre-sum pass
    (16384, 8, "kaiser", 9.0, 20),    # DIRECT variant, pre-sum pass (the large-N default at T = 8)
    (512, 16, "blackman", 0.0, 100),  # DIRECT variant, pre-sum pass, 16 taps
]


@pytest.mark.parametrize("N,T,win,beta,frames", CASES)
def test_pfb_parity_shapes(lib, N, T, win, beta, frames):
    n_tones = min(32, N // 2)
    extra = N // 3 + 1                      # ragged tail (residue, no frame)
    case = siggen.pfb_case(N * frames + extra, N, n_tones, seed=1000 + N + T,
                           amp=(200.0, 1500.0), sigma=8.0)
    plan = _plan(lib, N, T, win, beta, case["words"])
    full, tones = _run_gpu(plan, case["x"], n_tones, N)
    assert full.shape[0] == frames
    ref = oracle.pfb(case["x"], N, T, _oracle_taps(N, T, win, beta), bins=plan.bins())
    e_t = rel_rows(tones, ref["tones"])
    e_f = rel_channels_vs_rms(full, ref["full"])
    fe = full_spectrum_errors(full, ref["full"], plan.bins())
    print(f"N={N} T={T}: tones {e_t.max():.3e}, full (max(own, RMS)) {e_f.max():.3e}, strict tone channels "
          f"{fe['strict_tone_max']:.3e}, strict noise-only channels {fe['strict_noise_max']:.3e}")
    assert e_t.max() < TOL, e_t.max()
    assert e_f.max() < TOL, e_f.max()
    assert fe["strict_tone_max"] < TOL and fe["strict_noise_max"] < STRICT_NOISE_BOUND


@pytest.mark.parametrize("N,T,cluster", [(64, 4, 0), (4096, 8, 0), (1024, 16, 0), (8192, 8, 0), (16384, 3, 0),
                                         (8192, 8, 1), (16384, 3, 1), (4096, 16, 0), (4096, 11, 0)])
def test_streamed_equals_one_shot_bit_exact(lib, N, T, cluster):
    """Random splits (aligned and odd sizes, some shorter than a frame) give
    bit-identical frames to one push of the whole stream (for N = 8192 and
    16384 on the direct and on the cluster kernel)."""
    rng = np.random.default_rng(N + T)
    frames = 120 if N <= 1024 else 60
    case = siggen.pfb_case(N * frames + 5, N, 8, seed=77 + N)
    x = torch.from_numpy(case["x"]).to(DEV)
    one = _plan(lib, N, T, "hann", 0.0, case["words"])
    st = _plan(lib, N, T, "hann", 0.0, case["words"])
    if cluster:
        one.set_pfb_cluster(True)
        st.set_pfb_cluster(True)
        assert st.tune()["pfb_cluster"] == 1
    f1, t1 = _run_gpu(one, case["x"], 8, N)
    F = f1.shape[0]
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((8, F), dtype=torch.complex64, device=DEV)
    pos, off = 0, 0
    n = x.shape[0]
    while pos < n:
        kind = rng.integers(0, 4)
        if kind == 0:
            cnt = int(rng.integers(1, max(2, N // 2)))          # shorter than a frame
        elif kind == 1:
            cnt = int(rng.integers(1, 5 * N))                   # odd sizes
        else:
            cnt = int(rng.integers(1, 5 * N // 4)) * 4          # 16-byte multiples
        cnt = min(cnt, n - pos)
        off += st.push_into(x[pos:pos + cnt], fo, to, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F
    assert st.info()["samples_consumed"] == n
    assert np.array_equal(fo.cpu().numpy(), f1)
    assert np.array_equal(to.cpu().numpy(), t1)


def test_state_export_import_resume(lib):
    N, T = 256, 8
    case = siggen.pfb_case(N * 200 + 17, N, 12, seed=5)
    x = torch.from_numpy(case["x"]).to(DEV)
    ref_plan = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    f1, t1 = _run_gpu(ref_plan, case["x"], 12, N)
    a = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    F = f1.shape[0]
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((12, F), dtype=torch.complex64, device=DEV)
    cut = N * 77 + 101
    k = a.push_into(x[:cut], fo, to)
    blob = a.state_export()
    a.close()
    b = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    b.state_import(blob)
    k += b.push_into(x[cut:], fo, to, frame_offset=k)
    torch.cuda.synchronize()
    assert k == F
    assert np.array_equal(fo.cpu().numpy(), f1)
    assert np.array_equal(to.cpu().numpy(), t1)
    c = _plan(lib, N, 4, "kaiser", 9.0, case["words"])
    with pytest.raises(lib.RfrError):
        c.state_import(blob)                      # different plan parameters


def test_push_pull_queue_and_host_path(lib):
    N, T = 1024, 8
    case = siggen.pfb_case(N * 150 + 300, N, 20, seed=9)
    ref_plan = _plan(lib, N, T, "hann", 0.0, case["words"])
    f1, t1 = _run_gpu(ref_plan, case["x"], 20, N)
    F = f1.shape[0]
    q = _plan(lib, N, T, "hann", 0.0, case["words"])
    x = torch.from_numpy(case["x"]).to(DEV)
    for a, b in [(0, 5000), (5000, 5001), (5001, 90000), (90000, x.shape[0])]:
        q.push(x[a:b])
    assert q.info()["frames_pending"] == F
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((20, F), dtype=torch.complex64, device=DEV)
    small = torch.zeros((20, F - 1), dtype=torch.complex64, device=DEV)
    with pytest.raises(lib.RfrError) as ei:
        q.pull(fo, small)
    assert ei.value.status == lib.E_SHORT
    assert q.pull(fo, to) == F
    assert np.array_equal(fo.cpu().numpy(), f1)
    assert np.array_equal(to.cpu().numpy(), t1)
    # host-staged end-to-end path (pinned host buffers)
    h = _plan(lib, N, T, "hann", 0.0, case["words"])
    xh = torch.from_numpy(case["x"]).pin_memory()
    fh = torch.zeros((F, N), dtype=torch.complex64).pin_memory()
    th = torch.zeros((20, F), dtype=torch.complex64).pin_memory()
    assert h.process_host(xh, fh, th) == F
    assert np.array_equal(fh.numpy(), f1)
    assert np.array_equal(th.numpy(), t1)


def test_process_host_tone_groups(lib):
    """Host-staged run long enough that tone rows leave the device in several
    groups of chunks and a group buffer is reused (9 chunks of 2^24 samples
    and a ragged tail, 4 chunks per group); a second call continues the
    stream.  Equal, bit for bit, to one device push of the same samples."""
    N, T, nt = 4096, 8, 48
    rng = siggen.rng_for(77)
    words = siggen.bin_words(siggen.distinct_bins(rng, N, nt), N)
    n1, n2 = 9 * (1 << 24) + 12345, (1 << 24) + 777
    g = torch.Generator().manual_seed(78)
    xh = torch.randint(-2000, 2000, (n1 + n2, 2), dtype=torch.int16, generator=g).pin_memory()
    ref = _plan(lib, N, T, "kaiser", 9.0, words, full=False)
    F = ref.frames_for(n1 + n2)
    tr = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert ref.push_into(xh.to(DEV), None, tr) == F
    h = _plan(lib, N, T, "kaiser", 9.0, words, full=False)
    th = torch.full((nt, F), float("nan"), dtype=torch.complex64).pin_memory()
    F1 = h.frames_for(n1)
    assert h.process_host(xh[:n1], None, th) == F1
    assert F1 + h.process_host(xh[n1:], None, th, frame_offset=F1) == F
    assert np.array_equal(th.numpy(), tr.cpu().numpy())


def test_tones_only_and_full_only(lib):
    N, T = 512, 4
    case = siggen.pfb_case(N * 90, N, 10, seed=21)
    both = _plan(lib, N, T, "hann", 0.0, case["words"])
    f1, t1 = _run_gpu(both, case["x"], 10, N)
    to_plan = _plan(lib, N, T, "hann", 0.0, case["words"], full=False)
    _, t2 = _run_gpu(to_plan, case["x"], 10, N, full=False)
    assert np.array_equal(t1, t2)
    fo_plan = _plan(lib, N, T, "hann", 0.0, case["words"], tones=False)
    f3, _ = _run_gpu(fo_plan, case["x"], 0, N)
    assert np.array_equal(f1, f3)


def test_degenerate_pushes(lib):
    N, T = 64, 4
    case = siggen.pfb_case(N * 10, N, 4, seed=3)
    p = _plan(lib, N, T, "hann", 0.0, case["words"])
    x = torch.from_numpy(case["x"]).to(DEV)
    fo = torch.zeros((10, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((4, 10), dtype=torch.complex64, device=DEV)
    assert p.push_into(x[:0], fo, to) == 0          # empty push
    assert p.push_into(x[:N - 1], fo, to) == 0      # shorter than a frame
    k = p.push_into(x[N - 1:], fo, to)
    torch.cuda.synchronize()
    assert k == 10
    ref = oracle.pfb(case["x"], N, T, _oracle_taps(N, T, "hann", 0.0), bins=p.bins())
    assert rel_rows(to.cpu().numpy(), ref["tones"]).max() < TOL
    # capacity too small: RFR_E_SHORT and the stream state is unchanged
    q = _plan(lib, N, T, "hann", 0.0, case["words"])
    with pytest.raises(lib.RfrError) as ei:
        q.push_into(x, fo[:5], to)
    assert ei.value.status == lib.E_SHORT
    assert q.info()["samples_consumed"] == 0


def test_invalid_plans(lib):
    w = np.array([1 << 60], np.uint64)
    bad = [dict(channels=1, taps=4), dict(channels=64, taps=0), dict(channels=64, taps=17),
           dict(channels=-3, taps=4, decimation=64), dict(channels=1 << 25, taps=2),
           dict(channels=64, taps=4, decimation=65), dict(channels=100, taps=4, decimation=0)]
    for kw in bad:
        with pytest.raises(lib.RfrError) as ei:
            lib.Plan(window="hann", words=w, **kw)
        assert ei.value.status == lib.E_INVALID
    with pytest.raises(lib.RfrError):
        lib.Plan(64, 4, window="hann", words=None, full=False, tones=True)


def test_plain_fp32_form_parity(lib):
    c = siggen.pfb_case(1 << 18, 256, 16, seed=44)
    N, T = 256, 8
    plan = _plan(lib, N, T, "kaiser", 9.0, c["words"])
    x = torch.from_numpy(c["x"]).to(DEV)
    F = x.shape[0] // N
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((16, F), dtype=torch.complex64, device=DEV)
    assert plan.plain_oneshot(x, fo, to) == F
    torch.cuda.synchronize()
    ref = oracle.pfb(c["x"], N, T, _oracle_taps(N, T, "kaiser", 9.0), bins=plan.bins())
    assert rel_rows(to.cpu().numpy(), ref["tones"]).max() < TOL
    assert rel_channels_vs_rms(fo.cpu().numpy(), ref["full"]).max() < TOL


def test_c2_full_size_sampled(lib):
    """Workload 2 at full size (2^28 samples, N=4096, T=8 Kaiser(9), 1000
    tones), in the launch configuration the benchmark times; frames sampled at
    the start, middle and end are checked against the oracle one by one."""
    c = siggen.c2()
    N, T = 4096, 8
    plan = _plan(lib, N, T, "kaiser", 9.0, c["words"])
    bins = plan.bins()
    assert np.array_equal(np.sort(bins), np.sort(c["bins"]))
    x = torch.from_numpy(c["x"]).to(DEV)
    F = plan.frames_for(x.shape[0])
    assert F == 65536
    fo = torch.empty((F, N), dtype=torch.complex64, device=DEV)
    to = torch.empty((1000, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x, fo, to) == F
    torch.cuda.synchronize()
    h = _oracle_taps(N, T, "kaiser", 9.0)
    for a, b in [(0, 6), (31000, 31004), (65530, 65536)]:
        ref = oracle.pfb(c["x"], N, T, h, k_begin=a, k_end=b, bins=bins)
        got_f = fo[a:b].cpu().numpy()
        got_t = to[:, a:b].cpu().numpy()
        scale = np.sqrt(np.mean(np.abs(ref["full"]) ** 2))
        assert np.abs(got_f - ref["full"]).max() / scale < 1e-4
        assert np.linalg.norm(got_f - ref["full"]) / np.linalg.norm(ref["full"]) < TOL
        e_t = np.linalg.norm(got_t - ref["tones"], axis=1) / np.linalg.norm(ref["tones"], axis=1)
        assert e_t.max() < TOL, e_t.max()


@pytest.mark.parametrize("n_tones,frame_offset", [(1500, 0), (1500, 3), (2048, 0)])
def test_many_tones_and_offsets(lib, n_tones, frame_offset):
    """Tone counts that fit the shared-memory tone staging (1500) and one that
    does not (2048 -> direct stores), at even and odd output frame offsets."""
    N, T = 4096, 8
    case = siggen.pfb_case(N * 70, N, n_tones, seed=n_tones + frame_offset, amp=(100.0, 900.0))
    plan = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    x = torch.from_numpy(case["x"]).to(DEV)
    F = plan.frames_for(x.shape[0])
    fo = torch.zeros((F + frame_offset, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((n_tones, F + frame_offset + 1), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x, fo, to, frame_offset=frame_offset) == F
    torch.cuda.synchronize()
    ref = oracle.pfb(case["x"], N, T, _oracle_taps(N, T, "kaiser", 9.0), bins=plan.bins())
    got_t = to[:, frame_offset:frame_offset + F].cpu().numpy()
    assert rel_rows(got_t, ref["tones"]).max() < TOL
    assert np.array_equal(got_t, fo[frame_offset:].cpu().numpy()[:, plan.bins()].T)
    assert not to[:, :frame_offset].abs().any() and not to[:, frame_offset + F:].abs().any()


# N, T, window, beta, frames, tones, outputs (full, tones)
CLUSTER_CASES = [
    (16384, 8, "kaiser", 9.0, 24, 1000, (True, True)),    # the batched workload's largest plan
    (16384, 4, "hann", 0.0, 30, 100, (True, True)),       # tones on the first CTA only
    (8192, 8, "blackman", 0.0, 40, 700, (True, True)),    # two tone boxes per CTA
    (8192, 5, "hamming", 0.0, 37, 3000, (False, True)),   # 1536 tone rows per CTA: per-frame tone stores
    (16384, 7, "kaiser", 9.0, 21, 3000, (True, False)),   # full spectrum only
]


@pytest.mark.parametrize("N,T,win,beta,frames,nt,outs", CLUSTER_CASES)
def test_cluster_pfb_parity(lib, N, T, win, beta, frames, nt, outs):
    """N = 8192 and 16384 with T <= 8 on the cluster kernel (clusters of
    N / 4096 CTAs that split the channels, exchange the filtered slices for
    the cross-CTA step of the FFT and assemble the output rows through
    distributed shared memory): full spectrum and tones against the oracle,
    with ragged input (a residue that makes no frame); the direct kernel's
    frames agree with them to FP32 rounding."""
    full_on, tones_on = outs
    case = siggen.pfb_case(N * frames + N // 5 + 3, N, nt, seed=8800 + N + T + nt,
                           amp=(200.0, 1500.0), sigma=8.0)
    plan = _plan(lib, N, T, win, beta, case["words"], full=full_on, tones=tones_on)
    assert plan.tune()["pfb_cluster"] == 0
    plan.set_pfb_cluster(True)
    full, tones = _run_gpu(plan, case["x"], nt if tones_on else 0, N, full=full_on)
    direct = _plan(lib, N, T, win, beta, case["words"], full=full_on, tones=tones_on)
    dfull, dtones = _run_gpu(direct, case["x"], nt if tones_on else 0, N, full=full_on)
    if tones_on:
        assert rel_rows(tones, dtones).max() < 1e-5
    if full_on:
        assert rel_channels_vs_rms(full, dfull).max() < 1e-5
    ref = oracle.pfb(case["x"], N, T, _oracle_taps(N, T, win, beta), bins=plan.bins())
    msg = f"cluster N={N} T={T} tones={nt}:"
    if tones_on:
        assert np.isfinite(tones).all()
        e_t = rel_rows(tones, ref["tones"])
        msg += f" tones {e_t.max():.3e}"
        assert e_t.max() < TOL, e_t.max()
    if full_on:
        assert full.shape[0] == frames and np.isfinite(full).all()
        e_f = rel_channels_vs_rms(full, ref["full"])
        fe = full_spectrum_errors(full, ref["full"], plan.bins())
        msg += (f", full (max(own, RMS)) {e_f.max():.3e}, strict tone channels {fe['strict_tone_max']:.3e}, "
                f"strict noise-only {fe['strict_noise_max']:.3e}")
        assert e_f.max() < TOL, e_f.max()
        assert fe["strict_tone_max"] < TOL and fe["strict_noise_max"] < STRICT_NOISE_BOUND
    print(msg)


def test_cluster_pfb_frame_offsets_and_partial_tone_groups(lib):
    """Cluster kernel: pushes that start at output frame offsets that are not multiples of
    the 4-frame tone group (partial groups leave by plain stores), into
    output buffers with a row pitch larger than N: the same frames as one
    push into a tight buffer."""
    N, T, nt = 16384, 8, 600
    case = siggen.pfb_case(N * 45, N, nt, seed=8901)
    x = torch.from_numpy(case["x"]).to(DEV)
    one = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    one.set_pfb_cluster(True)
    f1, t1 = _run_gpu(one, case["x"], nt, N)
    F = f1.shape[0]
    st = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    st.set_pfb_cluster(True)
    fo = torch.zeros((F + 3, N + 8), dtype=torch.complex64, device=DEV)
    to = torch.zeros((nt, F + 5), dtype=torch.complex64, device=DEV)
    off = 1
    for a, b in [(0, N * 9), (N * 9, N * 22 + 100), (N * 22 + 100, N * 45)]:
        off += st.push_into(x[a:b], fo, to, frame_offset=off)
    torch.cuda.synchronize()
    assert off == F + 1
    assert np.array_equal(fo.cpu().numpy()[1:F + 1, :N], f1)
    assert np.array_equal(to.cpu().numpy()[:, 1:F + 1], t1)


def test_cluster_pfb_choice_is_validated(lib):
    words = np.array([1 << 58], np.uint64)
    p = lib.Plan(4096, 8, window="hann", words=words)
    with pytest.raises(lib.RfrError):
        p.set_pfb_cluster(True)                 # one SM holds N = 4096, T = 8
    assert p.tune()["pfb_cluster"] == 0
    q = lib.Plan(16384, 16, window="hann", words=words)
    with pytest.raises(lib.RfrError):
        q.set_pfb_cluster(True)                 # T > 8: direct kernel only
    r = lib.Plan(8192, 8, window="hann", words=words)
    r.set_pfb_cluster(True)
    assert r.tune()["pfb_cluster"] == 1
    r.set_pfb_cluster(False)
    assert r.tune()["pfb_cluster"] == 0
    for x in (p, q, r):
        x.close()


def test_two_pass_16_taps_outputs(lib):
    """N = 4096, T = 16 as a first-half FIR pass (taps 0..7) and the TMEM
    kernel continuing those sums with taps 8..15: tones only, full only and
    both agree bit for bit, the tones equal the spectrum's bin columns, and a
    push at an odd output frame offset with a row pitch above N (the
    plain-store paths) equals the tight push."""
    N, T, nt = 4096, 16, 700
    case = siggen.pfb_case(N * 60 + 9, N, nt, seed=9301)
    x = torch.from_numpy(case["x"]).to(DEV)
    both = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    f_b, t_b = _run_gpu(both, case["x"], nt, N)
    assert np.array_equal(t_b, f_b[:, both.bins()].T)
    _, t_t = _run_gpu(_plan(lib, N, T, "kaiser", 9.0, case["words"], full=False), case["x"], nt, N, full=False)
    f_f, _ = _run_gpu(_plan(lib, N, T, "kaiser", 9.0, case["words"], tones=False), case["x"], 0, N)
    assert np.array_equal(t_t, t_b) and np.array_equal(f_f, f_b)
    F = f_b.shape[0]
    p = _plan(lib, N, T, "kaiser", 9.0, case["words"])
    fo = torch.zeros((F + 3, N + 1), dtype=torch.complex64, device=DEV)     # odd pitch: plain row stores
    to = torch.zeros((nt, F + 5), dtype=torch.complex64, device=DEV)
    assert p.push_into(x, fo, to, frame_offset=3) == F
    torch.cuda.synchronize()
    assert np.array_equal(fo.cpu().numpy()[3:F + 3, :N], f_b)
    assert np.array_equal(to.cpu().numpy()[:, 3:F + 3], t_b)
