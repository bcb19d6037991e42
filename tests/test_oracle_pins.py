"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
brute force, library routines, closed forms, invariants and the paper's own
design statement (Sec. III.A: adjacent channels cross over near -6 dB)."""
import json
import os

import numpy as np
import pytest
import scipy.signal
import scipy.special

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
rng = np.random.default_rng(7)


def crandn(*shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- DFT / FFT
@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32, 64, 3, 5, 6, 7, 9, 12, 15, 30, 49, 60, 97, 100, 210])
def test_fft_matches_bruteforce_dft(n):
    x = crandn(n)
    # brute force written independently here: explicit double loop
    ref = np.array([sum(x[p] * np.exp(-2j * np.pi * ((c * p) % n) / n) for p in range(n))
                    for c in range(n)])
    scale = np.linalg.norm(ref) + 1e-300
    assert np.linalg.norm(oracle.dft(x) - ref) / scale < 1e-13
    assert np.linalg.norm(oracle.fft(x) - ref) / scale < 1e-13


@pytest.mark.parametrize("n", [128, 1024, 4096, 16384, 1000, 6720, 26880, 100000])
def test_fft_matches_library_fft(n):
    x = crandn(n)
    ref = np.fft.fft(x)
    assert np.linalg.norm(oracle.fft(x) - ref) / np.linalg.norm(ref) < 1e-13


@pytest.mark.parametrize("n", [64, 60, 1000])
def test_fft_unit_impulse_and_dc(n):
    e = np.zeros(n, complex); e[3] = 1.0
    c = np.arange(n)
    assert np.allclose(oracle.fft(e), np.exp(-2j * np.pi * ((3 * c) % n) / n), atol=1e-13)
    assert np.allclose(oracle.fft(np.ones(n)), n * (c == 0), atol=1e-10)


# ---------------------------------------------------------------- windows
@pytest.mark.parametrize("m", [1, 2, 7, 64, 257])
def test_windows_match_scipy(m):
    sw = scipy.signal.windows
    assert np.allclose(oracle.window("rect", m), np.ones(m), atol=0)
    assert np.allclose(oracle.window("hann", m), sw.hann(m, sym=True), atol=1e-15)
    assert np.allclose(oracle.window("hamming", m), sw.hamming(m, sym=True), atol=1e-15)
    assert np.allclose(oracle.window("blackman", m), sw.blackman(m, sym=True), atol=1e-15)
    for beta in (0.0, 5.0, 9.0):
        assert np.allclose(oracle.window("kaiser", m, beta), sw.kaiser(m, beta, sym=True),
                           rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("x", [0.0, 0.5, 1.0, 3.0, 9.0, 20.0, 40.0])
def test_bessel_i0_matches_library(x):
    assert oracle.bessel_i0(x) == pytest.approx(float(scipy.special.i0(x)), rel=1e-14)


def test_window_closed_form_points():
    m = 65
    assert oracle.window("hann", m)[0] == pytest.approx(0.0, abs=1e-16)
    assert oracle.window("hann", m)[32] == pytest.approx(1.0, abs=1e-15)
    assert oracle.window("hamming", m)[0] == pytest.approx(0.08, abs=1e-15)
    assert oracle.window("blackman", m)[32] == pytest.approx(1.0, abs=1e-15)
    assert oracle.window("kaiser", m, 9.0)[0] == pytest.approx(1.0 / scipy.special.i0(9.0),
                                                               rel=1e-13)


def test_lowpass_is_normalised_windowed_sinc():
    m, fc = 256, 1.0 / 128
    h = oracle.lowpass("hamming", m, fc)
    j = np.arange(m)
    ref = scipy.signal.windows.hamming(m) * np.sinc(2 * fc * (j - (m - 1) / 2))
    ref /= ref.sum()
    assert np.allclose(h, ref, rtol=1e-13, atol=1e-18)
    assert h.sum() == pytest.approx(1.0, abs=1e-14)
    # scipy.signal.firwin builds the same windowed sinc (cutoff in Nyquist units)
    fw = scipy.signal.firwin(m, 2 * fc, window="hamming", scale=False)
    assert np.allclose(h, fw / fw.sum(), rtol=1e-12, atol=1e-18)


def test_square_window_is_moving_average():
    """Sec. III.B: the demodulator's anti-alias filter is a square-window moving average."""
    h = oracle.lowpass("rect", 500, 0.0)
    assert np.allclose(h, 1.0 / 500, rtol=1e-15)


def test_prototype_fp32_rounding():
    h64, h32 = oracle.pfb_prototype(64, 4, "hann")
    assert h32.dtype == np.float32
    assert np.array_equal(h32, h64.astype(np.float32))
    assert h64.sum() == pytest.approx(1.0, abs=1e-14)


# ------------------------------------------------ paper: -6 dB cross-over
def _resp(h, f):
    j = np.arange(len(h))
    return abs(np.sum(h * np.exp(-2j * np.pi * f * j)))


def test_paper_adjacent_channel_crossover_6db():
    """Sec. III.A / Fig. 3: the sinc cut-off is placed so that adjacent
    channels cross over at about -6 dB.  Fixture cites the paper's parameters."""
    with open(os.path.join(GOLDEN, "paper_pfb_crossover.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        n, taps, win = case["n_chan"], case["taps"], case["window"]
        h64, _ = oracle.pfb_prototype(n, taps, win, case.get("beta", 0.0))
        ratio = _resp(h64, 0.5 / n) / _resp(h64, 0.0)
        db = 20 * np.log10(ratio)
        assert abs(db - g["crossover_db"]) < g["tolerance_db"], (case, db)


def test_paper_fig3_pfb_run_crossover():
    """Sec. III.A, Fig. 3: with N = 10^5 channels, A_v = 4 taps and a Hamming
    window, a tone half-way between two channels shows in both at about -6 dB
    of a channel-centred tone.  Runs the whole oracle PFB (FIR + length-10^5
    FFT) at the paper's size on an FP64 tone."""
    with open(os.path.join(GOLDEN, "paper_pfb_crossover.json")) as f:
        g = json.load(f)
    case = g["cases"][0]
    N, T = case["n_chan"], case["taps"]
    h64, _ = oracle.pfb_prototype(N, T, case["window"])
    m = np.arange(N * (T + 1), dtype=np.float64)
    b = 31415
    centred = np.exp(2j * np.pi * ((b * m) % N) / N)
    half = np.exp(2j * np.pi * (((2 * b + 1) * m) % (2 * N)) / (2 * N))
    yc = oracle.pfb(centred, N, T, h64, k_begin=T, k_end=T + 1)["full"][0]
    yh = oracle.pfb(half, N, T, h64, k_begin=T, k_end=T + 1)["full"][0]
    ref = abs(yc[b])
    for c in (b, b + 1):
        db = 20 * np.log10(abs(yh[c]) / ref)
        assert abs(db - g["crossover_db"]) < g["tolerance_db"], (c, db)
    # and nothing else above the two channels
    others = np.delete(np.abs(yh), [b, b + 1])
    assert others.max() < abs(yh[b])


# ---------------------------------------------------------- integer rules
def test_freq_to_word_exact_values():
    fs = 200e6
    assert oracle.freq_to_word(0.0, fs) == 0
    assert oracle.freq_to_word(fs / 4, fs) == 2 ** 62
    assert oracle.freq_to_word(-fs / 4, fs) == 2 ** 64 - 2 ** 62
    assert oracle.freq_to_word(-fs / 2, fs) == 2 ** 63
    for c in (1, 5, 63):
        assert oracle.freq_to_word(c * fs / 64, fs) == (c << 58)
    # a 40 kHz tone: the rule scales the FP64 quotient f/fs (relative error
    # <= 2^-53), so the word is within one unit of the exact rational value
    from fractions import Fraction
    exact = Fraction(40_000, 200_000_000) * 2 ** 64
    assert abs(oracle.freq_to_word(40e3, fs) - round(exact)) <= 1


def test_word_to_bin_rule():
    from fractions import Fraction
    r = np.random.default_rng(1)
    for n in (2, 64, 4096, 16384):
        words = [int(w) for w in r.integers(0, 2 ** 64, 200, dtype=np.uint64)]
        words += [(c << (64 - int(np.log2(n)))) for c in range(0, n, max(1, n // 16))]
        # exact ties: half a bin above centre rounds up
        words += [((3 << 1) + 1) << (63 - int(np.log2(n))) & (2 ** 64 - 1)]
        for w in words:
            q = Fraction(w * n, 2 ** 64)
            ref = int((q + Fraction(1, 2)).__floor__()) % n   # round half up
            assert oracle.word_to_bin(w, n) == ref
    # any N: random words, words just below and above every half-bin boundary
    for n in (3, 100, 1000, 10 ** 5, 10 ** 7):
        words = [int(w) for w in r.integers(0, 2 ** 64, 200, dtype=np.uint64)]
        for c in range(0, n, max(1, n // 7)):
            edge = (Fraction(2 * c + 1, 2 * n) * 2 ** 64).__ceil__()   # first word of bin c+1
            words += [(edge - 1) % 2 ** 64, edge % 2 ** 64]
        for w in words:
            ref = int((Fraction(w * n, 2 ** 64) + Fraction(1, 2)).__floor__()) % n
            assert oracle.word_to_bin(w, n) == ref


def test_nco_phase_is_product_mod_2_64():
    for w, m in [(3, 5), (2 ** 63 + 12345, 2 ** 40 + 7), (2 ** 64 - 1, 2 ** 64 - 1)]:
        assert oracle.nco_phase(w, m) == (w * m) % 2 ** 64


# ------------------------------------------------------------- PFB pins
def _tone(n, c0, N, A, th):
    m = np.arange(n)
    return A * np.exp(1j * (2 * np.pi * ((c0 * m) % N) / N + th))


@pytest.mark.parametrize("N,T,win,beta", [(8, 4, "hann", 0.0), (16, 3, "kaiser", 9.0),
                                          (32, 8, "hamming", 0.0), (12, 3, "hann", 0.0),
                                          (100, 4, "hamming", 0.0), (35, 2, "kaiser", 5.0)])
def test_pfb_equals_filtered_mixed_stream(N, T, win, beta):
    """Library-routine pin: each PFB channel c is the stream mixed down by
    exp(-2*pi*i*c*m/N), convolved with the time-reversed prototype
    (scipy.signal.lfilter) and sampled every N samples."""
    h64, h32 = oracle.pfb_prototype(N, T, win, beta)
    h = h32.astype(np.float64)
    n = N * 23
    x = crandn(n) * 100
    y = oracle.pfb(x, N, T, h)["full"]
    m = np.arange(n)
    for c in range(N):
        z = x * np.exp(-2j * np.pi * ((c * m) % N) / N)
        conv = scipy.signal.lfilter(h[::-1], [1.0], z)
        ref = conv[N - 1::N][: y.shape[0]]
        assert np.allclose(y[:, c], ref, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("N,c0", [(64, 13), (100, 37), (1000, 999)])
def test_pfb_bin_centred_tone_closed_form(N, c0):
    """A pure tone at bin c0 (FP64, unquantised) gives, after T-1 warm-up frames,
    y_k[c] = A e^{i th} DFT(P)[c - c0] with P[p] = sum_t h[tN+p]; so y_k[c0] =
    A e^{i th} sum(h)."""
    T, A, th = 4, 1234.5, 0.7
    _, h32 = oracle.pfb_prototype(N, T, "hann")
    h = h32.astype(np.float64)
    x = _tone(N * 40, c0, N, A, th)
    y = oracle.pfb(x, N, T, h)["full"]
    P = h.reshape(T, N).sum(axis=0)
    leak = np.fft.fft(P)
    for k in range(T - 1, y.shape[0]):
        # the tone's phase at the frame origin (k+1)N - M is a multiple of 2*pi
        ref = A * np.exp(1j * th) * leak[(np.arange(N) - c0) % N]
        assert np.allclose(y[k], ref, rtol=1e-12, atol=1e-9 * A)
    assert abs(y[T - 1, c0] - A * np.exp(1j * th) * h.sum()) < 1e-10 * A


def test_pfb_parseval_linearity_shift():
    N, T = 32, 4
    _, h32 = oracle.pfb_prototype(N, T, "kaiser", 9.0)
    h = h32.astype(np.float64)
    n = N * 30
    x1, x2 = crandn(n), crandn(n)
    r1 = oracle.pfb(x1, N, T, h, want_v=True)
    # Parseval on every frame
    lhs = np.sum(abs(r1["full"]) ** 2, axis=1)
    rhs = N * np.sum(abs(r1["v"]) ** 2, axis=1)
    assert np.allclose(lhs, rhs, rtol=1e-12)
    # linearity
    a, b = 0.3 - 1.1j, 2.5
    r12 = oracle.pfb(a * x1 + b * x2, N, T, h)["full"]
    r2 = oracle.pfb(x2, N, T, h)["full"]
    assert np.allclose(r12, a * r1["full"] + b * r2, rtol=1e-12, atol=1e-12)
    # a shift by N samples shifts the output by one frame
    xs = np.concatenate([np.zeros(N, complex), x1[:-N]])
    rs = oracle.pfb(xs, N, T, h)["full"]
    assert np.allclose(rs[1:], r1["full"][:-1], rtol=1e-12, atol=1e-12)


def test_pfb_int16_matches_f64_and_slices():
    N, T = 16, 4
    _, h32 = oracle.pfb_prototype(N, T, "hann")
    h = h32.astype(np.float64)
    r = np.random.default_rng(3)
    xi = r.integers(-8192, 8192, size=(N * 50, 2)).astype(np.int16)
    xc = xi[:, 0].astype(float) + 1j * xi[:, 1]
    bins = [0, 5, 15]
    a = oracle.pfb(xi, N, T, h, bins=bins)
    b = oracle.pfb(xc, N, T, h, bins=bins)
    assert np.array_equal(a["full"], b["full"])
    assert np.array_equal(a["tones"], b["tones"])
    assert np.array_equal(a["tones"], b["full"][:, bins].T)
    s = oracle.pfb(xi, N, T, h, k_begin=7, k_end=31, bins=bins)
    assert np.array_equal(s["full"], a["full"][7:31])
    assert np.array_equal(s["tones"], a["tones"][:, 7:31])


# ----------------------------------------------------------- demod pins
def _word_tone(n, w, A, th):
    m = np.arange(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ph = (m * np.uint64(w)).view(np.int64).astype(float) * (np.pi / 2 ** 63)
    return A * np.exp(1j * (ph + th))


def test_demod_own_tone_is_constant():
    L, D = 64, 16
    w = int(np.random.default_rng(5).integers(0, 2 ** 63)) * 2 + 1
    h = oracle.lowpass("blackman", L, 0.05)
    x = _word_tone(D * 40, w, 321.0, -0.4)
    out = oracle.demod(x, L, D, h, [w])[0]
    k0 = L // D - 1
    assert np.allclose(out[k0:], 321.0 * np.exp(-0.4j), rtol=1e-12)


def test_demod_moving_average_dirichlet():
    """Square window, D = L: an off tone at delta cycles/sample gives the
    Dirichlet kernel (1/L) sum_n e^{2 pi i delta (b+n)}."""
    L = D = 50
    fs = 1.0
    w_t = oracle.freq_to_word(0.1, fs)
    w_x = oracle.freq_to_word(0.1 + 0.013, fs)
    delta = ((w_x - w_t) % 2 ** 64) / 2 ** 64
    h = oracle.lowpass("rect", L, 0.0)
    x = _word_tone(D * 12, w_x, 10.0, 0.0)
    out = oracle.demod(x, L, D, h, [w_t])[0]
    for k in range(1, 12):
        b = (k + 1) * D - L
        n = np.arange(L)
        # x e^{-i phi_t} = 10 e^{i (phi_x - phi_t)} and phi_x - phi_t = 2 pi delta m exactly
        ref = 10.0 / L * np.exp(1j * np.pi * delta * (2 * b + L - 1)) \
            * np.sin(np.pi * delta * L) / np.sin(np.pi * delta)
        assert abs(out[k] - ref) < 1e-11 * 10


@pytest.mark.parametrize("N,T,win", [(16, 4, "hann"), (64, 4, "kaiser")])
def test_demod_equals_pfb_channel_for_bin_centred_tones(N, T, win):
    """With word c*2^64/N, L = N*T, D = N and the same taps, demodulation is
    the PFB's channel c: b_k is a multiple of N so the mixer phases agree."""
    beta = 9.0 if win == "kaiser" else 0.0
    h64, _ = oracle.pfb_prototype(N, T, win, beta)
    n = N * 25
    x = crandn(n) * 50
    y = oracle.pfb(x, N, T, h64)["full"]
    for c in (0, 1, N // 2, N - 1):
        w = (c << (64 - int(np.log2(N)))) % 2 ** 64
        d = oracle.demod(x, N * T, N, h64, [w])[0]
        assert np.allclose(d, y[:, c], rtol=1e-12, atol=1e-10)


def test_demod_int16_matches_f64():
    L, D = 40, 8
    r = np.random.default_rng(11)
    xi = r.integers(-8192, 8192, size=(D * 30, 2)).astype(np.int16)
    xc = xi[:, 0].astype(float) + 1j * xi[:, 1]
    h = oracle.lowpass("hann", L, 0.02)
    ws = [int(v) for v in r.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    a = oracle.demod(xi, L, D, h, ws)
    b = oracle.demod(xc, L, D, h, ws)
    assert np.array_equal(a, b)
    s = oracle.demod(xi, L, D, h, ws, k_begin=4, k_end=20)
    assert np.array_equal(s, a[:, 4:20])


# ----------------------------------------------------------- chirp pins
def test_chirp_phase_is_eq1_in_sample_units():
    """Eq. 1, phi_t = 2 pi (f0 t + k t^2), sampled at t = m/fs: the uint64
    phase start*m + rate*m^2 (mod 2^64) with start = f0/fs*2^64, rate =
    k/fs^2*2^64; checked with Python integers and against the FP64 formula."""
    fs, f0, k = 100e6, 3.1e6, 2.5e12            # 2.5 MHz/us sweep
    s = oracle.freq_to_word(f0, fs)
    r = oracle.chirp_rate_word(k, fs)
    for m in (0, 1, 7, 1000, 123457, -5):
        assert oracle.chirp_phase(s, r, m) == (s * m + r * m * m) % 2 ** 64
    for m in (0, 10, 1000, 20000):
        t = m / fs
        turns = (f0 * t + k * t * t) % 1.0
        got = oracle.chirp_phase(s, r, m) / 2 ** 64
        d = abs(got - turns)
        assert min(d, 1 - d) < 1e-9
    # instantaneous frequency: first difference = start + rate*(2m+1) exactly
    for m in (0, 99, 4096):
        d = (oracle.chirp_phase(s, r, m + 1) - oracle.chirp_phase(s, r, m)) % 2 ** 64
        assert d == (s + r * (2 * m + 1)) % 2 ** 64


def test_chirp_with_zero_rate_is_the_nco_demodulator():
    L, D = 64, 16
    rng = np.random.default_rng(9)
    x = rng.integers(-8192, 8192, size=(D * 40, 2)).astype(np.int16)
    h = oracle.lowpass("hann", L, 0.03)
    ws = [int(v) for v in rng.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    a = oracle.chirp_demod(x, L, D, h, ws, [0, 0, 0])
    b = oracle.demod(x, L, D, h, ws)
    assert np.array_equal(a, b)


def test_chirp_loopback_own_chirp_is_constant():
    """A chirp demodulated against itself (square window) gives A*e^{i0}
    apart from the rounding of the synthesised int16 samples."""
    L = D = 128
    s = oracle.freq_to_word(0.01, 1.0)
    r = oracle.chirp_rate_word(1e-6, 1.0)
    amp = 6000.0
    x = oracle.chirp_synth(s, r, amp, 0, D * 30)
    h = oracle.lowpass("rect", L, 0.0)
    out = oracle.chirp_demod(x, L, D, h, [s], [r])[0]
    assert np.allclose(out, amp, atol=0.5)        # int16 rounding: |err| <= 0.5*sqrt(2)/sqrt(L)-ish
    # synthesis matches the FP64 formula up to rounding
    m = np.arange(D * 30)
    ph = np.array([oracle.chirp_phase(s, r, int(i)) for i in m], dtype=np.uint64)
    th = ph.view(np.int64).astype(np.float64) * (np.pi / 2 ** 63)
    assert np.all(np.abs(x[:, 0] - amp * np.cos(th)) <= 0.5 + 1e-9)
    assert np.all(np.abs(x[:, 1] - amp * np.sin(th)) <= 0.5 + 1e-9)


# ------------------------------------------------------- transmit buffer
def test_tones_synth_grid_tones_equal_library_ifft():
    """Tones on an N-point grid (words b*2^64/N, phase words q*2^64/N): one
    period of the transmit buffer is N times the library inverse FFT of the
    sparse spectrum A_t e^{2 pi i q_t/N} at bins b_t; the buffer repeats with
    period N."""
    N = 1024
    r = np.random.default_rng(21)
    bins = r.choice(N, 40, replace=False)
    q = r.integers(0, N, 40)
    amps = r.uniform(10.0, 200.0, 40)
    words = [(int(b) << 54) for b in bins]
    ph = [(int(v) << 54) for v in q]
    val, iq = oracle.tones_synth(words, amps, 0, 2 * N, ph)
    spec = np.zeros(N, complex)
    spec[bins] = amps * np.exp(2j * np.pi * q / N)
    ref = N * np.fft.ifft(spec)
    assert np.allclose(val[:N], ref, rtol=0, atol=1e-9)
    assert np.allclose(val[N:], val[:N], rtol=0, atol=1e-9)
    assert np.array_equal(iq[:, 0], np.clip(np.rint(val.real), -32768, 32767).astype(np.int16))


def test_tones_synth_offgrid_linearity_and_own_demodulation():
    """Off-grid words: the buffer is the sum of its single-tone buffers, and
    demodulating the FP64 buffer at one tone's word with a long square window
    returns that tone's amplitude and phase (the others average out)."""
    r = np.random.default_rng(5)
    words = [int(w) for w in r.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    amps = [300.0, 200.0, 100.0]
    m0, n = 12345, 4096
    val, _ = oracle.tones_synth(words, amps, m0, n)
    parts = sum(oracle.tones_synth([w], [a], m0, n)[0] for w, a in zip(words, amps))
    assert np.allclose(val, parts, rtol=0, atol=1e-9)
    # the single-tone buffer is A exp(i*2*pi*w*m/2^64) at every sample
    from fractions import Fraction
    for m in (m0, m0 + 1, m0 + n - 1):
        ph = (words[0] * m) % 2 ** 64
        ang = 2 * np.pi * float(Fraction(ph if ph < 2 ** 63 else ph - 2 ** 64, 2 ** 64))
        v = oracle.tones_synth([words[0]], [1.0], m, 1)[0][0]
        assert abs(v - np.exp(1j * ang)) < 1e-12
    # demodulation of the buffer from sample 0 at tone 0's word: a square
    # window of L samples returns A_0 (phase 0) up to the other tones' leakage
    L = 4096
    full, _ = oracle.tones_synth(words, amps, 0, 2 * L)
    h = np.full(L, 1.0 / L)
    d = oracle.demod(full, L, L, h, [words[0]])[0]
    # Dirichlet kernel: |sin(pi L f) / (L sin(pi f))| <= 1 / (2 L |f|), |f| <= 1/2
    dmin = min(abs(((w - words[0] + 2 ** 63) % 2 ** 64 - 2 ** 63) / 2 ** 64) for w in words[1:])
    leak = sum(amps[1:]) / (2 * L * dmin)
    assert np.all(np.abs(d[1:] - amps[0]) <= leak + 1e-9)


# ----------------------------------------------------- oversampled PFB
def _i16(n, seed, amp=3000):
    r = np.random.default_rng(seed)
    return r.integers(-amp, amp, size=(n, 2)).astype(np.int16)


def test_pfb_hop_n_is_the_critically_sampled_pfb():
    N, T = 64, 4
    _, h32 = oracle.pfb_prototype(N, T, "hann")
    h = h32.astype(np.float64)
    x = _i16(N * 30, 1)
    a = oracle.pfb(x, N, T, h)["full"]
    b = oracle.pfb_hop(x, N, T, N, h)["full"]
    assert np.allclose(a, b, rtol=1e-13, atol=1e-9)


def test_pfb_hop_brute_force():
    """Tiny case against the definition written out with Python loops:
    y_k[c] = sum_p v_k[p] exp(-2 pi i c (s_k + p) / N), s_k = (k+1) H - N T."""
    N, T, H = 6, 2, 4
    h = np.linspace(0.3, 1.7, N * T)
    x = _i16(40, 2)
    xc = x[:, 0].astype(float) + 1j * x[:, 1]
    got = oracle.pfb_hop(x, N, T, H, h)["full"]
    for k in range(got.shape[0]):
        s = (k + 1) * H - N * T
        v = [sum(h[t * N + p] * (xc[s + t * N + p] if s + t * N + p >= 0 else 0) for t in range(T))
             for p in range(N)]
        for c in range(N):
            ref = sum(v[p] * np.exp(-2j * np.pi * c * (s + p) / N) for p in range(N))
            assert abs(got[k, c] - ref) < 1e-9 * (1 + abs(ref))


@pytest.mark.parametrize("N,T,H", [(64, 4, 32), (64, 4, 16), (32, 8, 24)])
def test_pfb_hop_channel_is_the_demodulator(N, T, H):
    """Channel c of the oversampled PFB equals direct demodulation at the
    bin-centred word c 2^64/N with L = N T and D = H (same taps)."""
    h64, _ = oracle.pfb_prototype(N, T, "kaiser", 9.0)
    x = _i16(N * 40, 3)
    y = oracle.pfb_hop(x, N, T, H, h64)["full"]
    for c in (0, 1, N // 3, N - 1):
        w = (c << (64 - int(np.log2(N)))) % 2 ** 64
        d = oracle.demod(x, N * T, H, h64, [w])[0]
        assert np.allclose(d[: y.shape[0]], y[:, c], rtol=1e-11, atol=1e-7)


def test_pfb_half_hop_odd_frames_are_the_critically_sampled_frames():
    N, T = 100, 4
    _, h32 = oracle.pfb_prototype(N, T, "hamming")
    h = h32.astype(np.float64)
    x = _i16(N * 20, 4)
    crit = oracle.pfb(x, N, T, h)["full"]
    half = oracle.pfb_hop(x, N, T, N // 2, h)["full"]
    assert np.allclose(half[1::2][: crit.shape[0]], crit[: half[1::2].shape[0]], rtol=1e-12, atol=1e-8)


# ------------------------------------------------ absolute stream origin
def _turns_to_phasor(phase_u64: int) -> complex:
    """exp(-i 2 pi phase / 2^64) for a phase given as a Python integer."""
    p = phase_u64 % 2 ** 64
    s = p - 2 ** 64 if p >= 2 ** 63 else p
    return complex(np.exp(-1j * np.pi * (s / 2 ** 63)))


@pytest.mark.parametrize("m0", [1, 17, 96, 250])
def test_absolute_origin_equals_zero_padded_stream(m0):
    """A stream that starts at absolute sample m0 (zero before it) is the
    zero-padded stream [0]*m0 + x seen from 0: the same frames, bit for bit,
    for the demodulator, the chirp demodulator and the oversampled PFB."""
    r = np.random.default_rng(40 + m0)
    x = r.integers(-8192, 8192, size=(700, 2)).astype(np.int16)
    xp = np.concatenate([np.zeros((m0, 2), np.int16), x])
    L, D = 48, 16
    h = oracle.lowpass("hann", L, 0.03)
    ws = [int(v) for v in r.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    rs = [int(v) for v in r.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    k0, k1 = 2, (m0 + 700) // D
    assert np.array_equal(oracle.demod(x, L, D, h, ws, k0, k1, m0=m0), oracle.demod(xp, L, D, h, ws, k0, k1))
    assert np.array_equal(oracle.chirp_demod(x, L, D, h, ws, rs, k0, k1, m0=m0),
                          oracle.chirp_demod(xp, L, D, h, ws, rs, k0, k1))
    N, T, H = 12, 3, 8
    hp = np.linspace(0.2, 1.1, N * T)
    a = oracle.pfb_hop(x, N, T, H, hp, 1, (m0 + 700) // H, bins=[0, 5], m0=m0)
    b = oracle.pfb_hop(xp, N, T, H, hp, 1, (m0 + 700) // H, bins=[0, 5])
    assert np.array_equal(a["full"], b["full"]) and np.array_equal(a["tones"], b["tones"])


LARGE_ORIGINS = [2 ** 31 + 3 * 64, 2 ** 40 + 5 * 64, 2 ** 62 + 7 * 64]


@pytest.mark.parametrize("m0", LARGE_ORIGINS)
def test_demod_far_origin_is_the_shifted_phase(m0):
    """Time shift of the NCO (Sec. III.B mixer): the same samples placed at
    absolute origin m0 (a multiple of D) give, frame for frame, the origin-0
    output times exp(-i 2 pi (w m0 mod 2^64) / 2^64), the factor formed from
    Python integers.  Checks the uint64 phase of the oracle far past 2^31,
    2^40 and 2^62 samples."""
    L, D = 128, 64
    r = np.random.default_rng(m0 % 1000)
    x = r.integers(-8192, 8192, size=(D * 12, 2)).astype(np.int16)
    h = oracle.lowpass("blackman", L, 0.01)
    ws = [int(v) for v in r.integers(0, 2 ** 64, 4, dtype=np.uint64)]
    K0 = m0 // D
    near = oracle.demod(x, L, D, h, ws, 0, 12)
    far = oracle.demod(x, L, D, h, ws, K0, K0 + 12, m0=m0)
    for s, w in enumerate(ws):
        ref = near[s] * _turns_to_phasor(w * m0)
        assert np.max(np.abs(far[s] - ref)) < 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("m0", LARGE_ORIGINS)
def test_chirp_far_origin_is_a_shifted_chirp(m0):
    """Eq. 1 in sample units is quadratic: p(m0 + j) = p(m0) + (s + 2 r m0) j
    + r j^2 (mod 2^64).  So demodulating at origin m0 against (s, r) equals
    demodulating at 0 against (s + 2 r m0, r), times exp(-i 2 pi p(m0) / 2^64),
    all words from Python integers."""
    L, D = 128, 64
    r = np.random.default_rng(m0 % 997)
    x = r.integers(-8192, 8192, size=(D * 12, 2)).astype(np.int16)
    h = oracle.lowpass("hann", L, 0.01)
    ss = [int(v) for v in r.integers(0, 2 ** 64, 3, dtype=np.uint64)]
    rr = [int(v) for v in r.integers(0, 2 ** 40, 3, dtype=np.uint64)]
    K0 = m0 // D
    far = oracle.chirp_demod(x, L, D, h, ss, rr, K0, K0 + 12, m0=m0)
    for i, (s, q) in enumerate(zip(ss, rr)):
        s2 = (s + 2 * q * m0) % 2 ** 64
        near = oracle.chirp_demod(x, L, D, h, [s2], [q], 0, 12)[0]
        ref = near * _turns_to_phasor(s * m0 + q * m0 * m0)
        assert np.max(np.abs(far[i] - ref)) < 1e-11 * np.max(np.abs(ref))
        assert oracle.chirp_phase(s, q, m0) == (s * m0 + q * m0 * m0) % 2 ** 64


@pytest.mark.parametrize("m0", [2 ** 31 + 3 * 8, 2 ** 40 + 5 * 8, 2 ** 62 + 8 * 8])
def test_pfb_hop_far_origin_is_the_channel_phase(m0):
    """Channels keep the absolute time origin's phase: moving the same samples
    to origin m0 (a multiple of the hop) multiplies channel c by
    exp(-2 pi i c (m0 mod N) / N) (N = 12, so m0 mod N is not 0)."""
    N, T, H = 12, 4, 8
    assert m0 % N != 0
    r = np.random.default_rng(m0 % 991)
    x = r.integers(-8192, 8192, size=(H * 20, 2)).astype(np.int16)
    h64, _ = oracle.pfb_prototype(N, T, "kaiser", 9.0)
    K0 = m0 // H
    near = oracle.pfb_hop(x, N, T, H, h64, 0, 20)["full"]
    far = oracle.pfb_hop(x, N, T, H, h64, K0, K0 + 20, m0=m0)["full"]
    c = np.arange(N)
    ref = near * np.exp(-2j * np.pi * c * (m0 % N) / N)[None, :]
    assert np.max(np.abs(far - ref)) < 1e-11 * np.max(np.abs(ref))
