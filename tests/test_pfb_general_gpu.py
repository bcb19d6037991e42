"""GPU parity of the PFB for any channel count N = 2^a 3^b 5^c 7^d up to
2^24 (Sec. III.A: Fig. 3 channelizes with N = 10^5, the section reports up to
10^7 bins) against the FP64 oracle, through the C ABI: the one-pass
mixed-radix kernel (N <= 8192), the four-step two-pass form above it, and
powers of two outside the fused kernels' range.  Same tolerance as the
power-of-two path: relative error <= 1e-5 per tone channel and per spectrum
channel against the RMS channel norm."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import STRICT_NOISE_BOUND, TOL, full_spectrum_errors, rel_channels_vs_rms, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _taps(N, T, win, beta):
    _, h32 = oracle.pfb_prototype(N, T, win, beta)
    return h32.astype(np.float64)


def _run(plan, x_np, n_tones, N, full=True):
    x = torch.from_numpy(x_np).to(DEV)
    F = plan.frames_for(x.shape[0])
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV) if full else None
    to = torch.zeros((n_tones, F), dtype=torch.complex64, device=DEV) if n_tones else None
    assert plan.push_into(x, fo, to) == F
    torch.cuda.synchronize()
    return (None if fo is None else fo.cpu().numpy()), (None if to is None else to.cpu().numpy())


CASES = [
    # N, T, window, beta, frames
    (2, 4, "hann", 0.0, 300),             # below the fused kernels' range
    (3, 1, "rect", 0.0, 300),
    (8, 2, "hamming", 0.0, 300),
    (100, 4, "hamming", 0.0, 200),
    (1000, 8, "kaiser", 9.0, 100),
    (2401, 3, "hann", 0.0, 60),           # 7^4: radix-7 stages only
    (6000, 16, "blackman", 0.0, 30),
    (6720, 4, "hann", 0.0, 40),           # 2^6 * 3 * 5 * 7
    (10000, 4, "kaiser", 9.0, 20),        # two passes
    (19683, 2, "hann", 0.0, 10),          # 3^9, two passes of radix-3 stages
    (32768, 8, "kaiser", 9.0, 10),        # power of two above the fused kernels
    (100000, 4, "hamming", 0.0, 8),       # Fig. 3's N and A_v
    (20000, 5, "hann", 0.0, 12),          # two passes, FIR ahead with any T
    (30000, 3, "blackman", 0.0, 10),      # two passes, T = 3
    (40000, 1, "rect", 0.0, 10),          # two passes, T = 1
]


@pytest.mark.parametrize("N,T,win,beta,frames", CASES)
def test_any_n_parity(lib, N, T, win, beta, frames):
    n_tones = min(24, N)
    extra = N // 3 + 1                     # ragged tail (residue, no frame)
    case = siggen.pfb_case(N * frames + extra, N, n_tones, seed=4000 + N + T,
                           amp=(200.0, 1500.0), sigma=8.0)
    plan = lib.Plan(N, T, window=win, beta=beta, words=case["words"], full=True, tones=True)
    bins = plan.bins()
    assert np.array_equal(bins, [oracle.word_to_bin(int(w), N) for w in case["words"]])
    h64p, h32p = plan.taps_table()
    h64o, h32o = oracle.pfb_prototype(N, T, win, beta)
    assert np.abs(h32p.view(np.int32).astype(np.int64) - h32o.view(np.int32).astype(np.int64)).max() <= 1
    full, tones = _run(plan, case["x"], n_tones, N)
    assert full.shape[0] == frames
    ref = oracle.pfb(case["x"], N, T, h32o.astype(np.float64), bins=bins)
    e_t = rel_rows(tones, ref["tones"])
    e_f = rel_channels_vs_rms(full, ref["full"])
    fe = full_spectrum_errors(full, ref["full"], bins)
    print(f"N={N} T={T}: max tone rel err {e_t.max():.3e}, max channel err {e_f.max():.3e}; strict: tone "
          f"channels {fe['strict_tone_max']:.3e}, noise-only channels {fe['strict_noise_max']:.3e}")
    assert e_t.max() < TOL, e_t.max()
    assert e_f.max() < TOL, e_f.max()
    assert fe["strict_tone_max"] < TOL and fe["strict_noise_max"] < STRICT_NOISE_BOUND
    assert np.array_equal(tones, full[:, bins].T)     # the gather is an exact copy


@pytest.mark.parametrize("N,T,frames", [(10 ** 7, 4, 2), (1 << 24, 2, 2)])
def test_largest_n_parity(lib, N, T, frames):
    """The section's largest channel count (10^7) and the largest N accepted
    (2^24): two frames against the oracle's FIR and length-N FFT; tones in
    full, the spectrum on every 997th channel plus the tone bins."""
    n_tones = 16
    case = siggen.pfb_case(N * frames + 7, N, n_tones, seed=91 + T, amp=(500.0, 2000.0), sigma=8.0)
    plan = lib.Plan(N, T, window="hann", words=case["words"], full=True, tones=True)
    full, tones = _run(plan, case["x"], n_tones, N)
    ref = oracle.pfb(case["x"], N, T, _taps(N, T, "hann", 0.0), bins=plan.bins())
    e_t = rel_rows(tones, ref["tones"])
    assert e_t.max() < TOL, e_t.max()
    cols = np.union1d(np.arange(0, N, 997), plan.bins())
    e_f = rel_channels_vs_rms(full[:, cols], ref["full"][:, cols])
    print(f"N={N}: max tone rel err {e_t.max():.3e}, sampled channel err {e_f.max():.3e}")
    assert e_f.max() < TOL, e_f.max()


def test_paper_fig3_crossover_on_gpu(lib):
    """Fig. 3 on the GPU path: N = 10^5, A_v = 4, Hamming; a tone half-way
    between channels b and b+1 shows in both at about -6 dB of a
    channel-centred tone of the same amplitude (int16 input)."""
    N, T, b, A = 100000, 4, 31415, 6000.0
    m = np.arange(N * (T + 2), dtype=np.float64)

    def q(z):
        return np.stack([np.rint(z.real), np.rint(z.imag)], axis=1).astype(np.int16)

    centred = q(A * np.exp(2j * np.pi * ((b * m) % N) / N))
    half = q(A * np.exp(2j * np.pi * (((2 * b + 1) * m) % (2 * N)) / (2 * N)))
    out = []
    for x in (centred, half):
        plan = lib.Plan(N, T, window="hamming", words=[], full=True, tones=False)
        full, _ = _run(plan, x, 0, N)
        out.append(np.abs(full[T + 1]))
    ref = out[0][b]
    for c in (b, b + 1):
        db = 20 * np.log10(out[1][c] / ref)
        assert abs(db + 6.0) < 0.25, (c, db)


@pytest.mark.parametrize("N,T", [(1000, 8), (10000, 4)])
def test_any_n_streamed_and_resumed_bit_exact(lib, N, T):
    """Random push sizes, and a state export / import half-way, give the
    same frames bit for bit as one push of the whole stream."""
    rng = np.random.default_rng(N)
    frames = 40 if N <= 1000 else 12
    case = siggen.pfb_case(N * frames + 11, N, 6, seed=5 + N)
    x = torch.from_numpy(case["x"]).to(DEV)
    one = lib.Plan(N, T, window="hann", words=case["words"], full=True, tones=True)
    f1, t1 = _run(one, case["x"], 6, N)
    F = f1.shape[0]
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((6, F), dtype=torch.complex64, device=DEV)
    st = lib.Plan(N, T, window="hann", words=case["words"], full=True, tones=True)
    pos = off = 0
    n = x.shape[0]
    half_done = False
    while pos < n:
        cnt = int(min(n - pos, rng.integers(1, 3 * N)))
        off += st.push_into(x[pos:pos + cnt], fo, to, frame_offset=off)
        pos += cnt
        if not half_done and pos > n // 2:
            torch.cuda.synchronize()
            blob = st.state_export()
            st = lib.Plan(N, T, window="hann", words=case["words"], full=True, tones=True)
            st.state_import(blob)
            half_done = True
    torch.cuda.synchronize()
    assert off == F
    assert np.array_equal(fo.cpu().numpy(), f1) and np.array_equal(to.cpu().numpy(), t1)


def test_unsupported_n_is_rejected(lib):
    """N with a prime factor above 7 is refused with RFR_E_UNSUPPORTED."""
    for N in (11, 13 * 64, 10007):
        with pytest.raises(lib.RfrError) as e:
            lib.Plan(N, 4, window="hann", words=[], full=True, tones=False)
        assert e.value.status == -7


# ------------------------------------------------------ oversampled (hop < N)
OVERSAMPLED = [
    # N, T, hop, window, frames
    (1024, 8, 512, "kaiser", 200),       # power of two, half hop
    (4096, 8, 1024, "kaiser", 60),       # the workload's N, quarter hop
    (1000, 4, 250, "hann", 120),
    (64, 4, 48, "hamming", 300),         # a hop that does not divide N
    (10000, 4, 5000, "kaiser", 16),      # four-step form
    (20000, 4, 7000, "hann", 12),        # four-step form, hop not dividing N (a shift per frame)
]


@pytest.mark.parametrize("N,T,hop,win,frames", OVERSAMPLED)
def test_oversampled_parity(lib, N, T, hop, win, frames):
    beta = 9.0 if win == "kaiser" else 0.0
    n_tones = min(16, N)
    case = siggen.pfb_case(hop * frames + N * T, N, n_tones, seed=600 + N + hop, amp=(200.0, 1500.0))
    plan = lib.Plan(N, T, window=win, beta=beta, words=case["words"], decimation=hop, full=True, tones=True)
    full, tones = _run(plan, case["x"], n_tones, N)
    ref = oracle.pfb_hop(case["x"], N, T, hop, _taps(N, T, win, beta), k_end=full.shape[0], bins=plan.bins())
    e_t = rel_rows(tones, ref["tones"])
    e_f = rel_channels_vs_rms(full, ref["full"])
    print(f"N={N} T={T} hop={hop}: max tone rel err {e_t.max():.3e}, max channel err {e_f.max():.3e}")
    assert e_t.max() < TOL and e_f.max() < TOL


def test_oversampled_channel_is_the_gpu_demodulator(lib):
    """Channel c of the oversampled PFB (hop 512, N = 1024, T = 8) and the
    tensor-core demodulator at the bin-centred word c 2^64/N with L = N T,
    D = hop and the same FP32 taps agree within the tolerance."""
    N, T, hop = 1024, 8, 512
    case = siggen.pfb_case(hop * 160 + N * T, N, 6, seed=17, amp=(300.0, 2000.0))
    pfb = lib.Plan(N, T, window="hann", words=case["words"], decimation=hop, full=False, tones=True)
    _, tp = _run(pfb, case["x"], 6, N, full=False)
    dem = lib.Plan(0, N * T, window="hann", cutoff=0.5 / N, words=case["words"], decimation=hop)
    h64p, _ = pfb.taps_table()
    h64d, _ = dem.taps_table()
    assert np.allclose(h64p, h64d, rtol=1e-12, atol=1e-18)
    x = torch.from_numpy(case["x"]).to(DEV)
    td = torch.zeros((6, dem.frames_for(x.shape[0])), dtype=torch.complex64, device=DEV)
    dem.push_into(x, tones=td)
    torch.cuda.synchronize()
    F = min(tp.shape[1], td.shape[1])
    assert rel_rows(tp[:, :F], td.cpu().numpy()[:, :F]).max() < TOL


@pytest.mark.parametrize("N,hop", [(1000, 250), (1024, 512)])
def test_oversampled_streamed_equals_one_shot(lib, N, hop):
    rng = np.random.default_rng(N + hop)
    case = siggen.pfb_case(hop * 150 + 5, N, 6, seed=9 + N)
    x = torch.from_numpy(case["x"]).to(DEV)
    mk = lambda: lib.Plan(N, 4, window="hann", words=case["words"], decimation=hop, full=True, tones=True)
    f1, t1 = _run(mk(), case["x"], 6, N)
    F = f1.shape[0]
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((6, F), dtype=torch.complex64, device=DEV)
    st = mk()
    pos = off = 0
    while pos < x.shape[0]:
        cnt = int(min(x.shape[0] - pos, rng.integers(1, 3 * hop)))
        off += st.push_into(x[pos:pos + cnt], fo, to, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F
    assert np.array_equal(fo.cpu().numpy(), f1) and np.array_equal(to.cpu().numpy(), t1)


@pytest.mark.parametrize("N,T,hop", [(100000, 4, 100000),     # two passes, FIR ahead (V by TMA)
                                     (19683, 2, 19683),       # two passes, FIR inside pass A
                                     (1000, 8, 1000),         # one pass, 4 frames per CTA iteration
                                     (20000, 4, 7000)])       # two passes, oversampled
def test_any_n_output_subsets_bit_exact(lib, N, T, hop):
    """Tones-only and full-only plans (other branches of the output stages)
    give, bit for bit, the tones and the spectrum of a full + tones plan."""
    n_tones = 20
    frames = 10
    case = siggen.pfb_case(hop * frames + N * T, N, n_tones, seed=700 + N + hop, amp=(200.0, 1500.0))
    mk = lambda full, tones: lib.Plan(N, T, window="hann", words=case["words"], decimation=hop,
                                      full=full, tones=tones)
    f1, t1 = _run(mk(True, True), case["x"], n_tones, N)
    _, t2 = _run(mk(False, True), case["x"], n_tones, N, full=False)
    f3, _ = _run(mk(True, False), case["x"], 0, N)
    assert np.array_equal(t2, t1)
    assert np.array_equal(f3, f1)


@pytest.mark.parametrize("hop", [1024, 2048])
def test_oversampled_4096_phase_passes(lib, hop):
    """N = 4096, T = 8 with hop N/4 or N/2 runs as N/hop critically sampled
    passes of the fused kernel on the stream shifted by k*hop, each bin turned
    by an exact quarter-turn power: parity with the oracle (full spectrum and
    tones), one push = random pieces bit for bit (odd sizes take the
    contiguous-view copy), and the output subsets equal the full + tones plan."""
    N, T = 4096, 8
    frames = 90
    case = siggen.pfb_case(hop * frames + N * T + 77, N, 40, seed=810 + hop, amp=(200.0, 1500.0))
    mk = lambda full=True, tones=True: lib.Plan(N, T, window="kaiser", beta=9.0, words=case["words"],
                                                decimation=hop, full=full, tones=tones)
    plan = mk()
    full, tones = _run(plan, case["x"], 40, N)
    F = full.shape[0]
    ref = oracle.pfb_hop(case["x"], N, T, hop, _taps(N, T, "kaiser", 9.0), k_end=F, bins=plan.bins())
    e_t = rel_rows(tones, ref["tones"])
    fe = full_spectrum_errors(full, ref["full"], plan.bins())
    print(f"N=4096 hop={hop} phase passes: tones {e_t.max():.3e}, full {fe['rms_norm_max']:.3e}, strict tone "
          f"channels {fe['strict_tone_max']:.3e}, noise-only {fe['strict_noise_max']:.3e}")
    assert e_t.max() < TOL and fe["rms_norm_max"] < TOL and fe["strict_tone_max"] < TOL
    assert np.array_equal(tones, full[:, plan.bins()].T)
    # streamed in random pieces (odd sizes, some shorter than a hop)
    rng = np.random.default_rng(hop)
    x = torch.from_numpy(case["x"]).to(DEV)
    st = mk()
    fo = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((40, F), dtype=torch.complex64, device=DEV)
    pos, off = 0, 0
    while pos < x.shape[0]:
        cnt = int(min(x.shape[0] - pos, rng.integers(1, 3 * hop) if rng.uniform() < 0.5 else
                      4 * rng.integers(1, hop)))
        off += st.push_into(x[pos:pos + cnt], fo, to, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F
    assert np.array_equal(fo.cpu().numpy(), full) and np.array_equal(to.cpu().numpy(), tones)
    # tones only / full only
    ft, tt = _run(mk(full=False), case["x"], 40, N, full=False)
    assert ft is None and np.array_equal(tt, tones)
    fonly, _ = _run(mk(tones=False), case["x"], 0, N)
    assert np.array_equal(fonly, full)


def test_oversampled_phase_passes_many_tones(lib):
    """Hop N/2 with 1500 tones (more than the fused kernel's tone tile holds:
    each pass stores its tones per frame into its dense rows), pushed at an
    odd output frame offset: the tones equal the full spectrum's bin columns
    and the oracle."""
    N, T, hop, nt = 4096, 8, 2048, 1500
    case = siggen.pfb_case(hop * 70 + N * T + 5, N, nt, seed=8123, amp=(200.0, 1500.0))
    plan = lib.Plan(N, T, window="kaiser", beta=9.0, words=case["words"], decimation=hop, full=True, tones=True)
    x = torch.from_numpy(case["x"]).to(DEV)
    F = plan.frames_for(x.shape[0])
    fo = torch.zeros((F + 3, N), dtype=torch.complex64, device=DEV)
    to = torch.zeros((nt, F + 3), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x, fo, to, frame_offset=3) == F
    torch.cuda.synchronize()
    full, tones = fo.cpu().numpy()[3:], to.cpu().numpy()[:, 3:]
    assert np.array_equal(tones, full[:, plan.bins()].T)
    sel = np.linspace(0, nt - 1, 12).astype(int)
    ref = oracle.pfb_hop(case["x"], N, T, hop, _taps(N, T, "kaiser", 9.0), k_end=F, bins=plan.bins()[sel])
    assert rel_rows(tones[sel], ref["tones"]).max() < TOL
