"""Seeded synthetic inputs: complex int16 IQ streams of KID-style tone combs.

This module synthesises INPUTS only (tones plus Gaussian noise, rounded to the
14-bit range of the software radio's ADC, Sec. II.A of arXiv:1812.02200).  It
holds none of the readout method's arithmetic (no windows, filters, FFTs or
demodulation) and is shared by the tests, the benchmark and the smoke check.

Signal model for a stream of n samples:
    x[m] = s * sum_i A_i * exp(i*(2*pi*(w_i*m mod 2^64)/2^64 + theta_i))
           + sigma*(g_I[m] + i*g_Q[m])
rounded half-to-even to integers and clamped to [-8192, 8191].  w_i is the
tone's uint64 phase word (bin-centred words are c*2^64/N), theta_i is uniform
in [0, 2*pi), g are standard normal draws, and the scale s follows one of the
rules below (per workload):
    "none"  s = 1                      (amplitudes as given; clipping allowed)
    "rms"   s chosen so that the per-component RMS of the composite, noise
            included, is 8191/6 (a 6-sigma back-off; rare peaks clip)
"""
from __future__ import annotations

import numpy as np

FULL_SCALE = 8191
TWO64 = 2.0 ** 64
SEED_BASE = 1812022000


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _angle(words_times_m: np.ndarray) -> np.ndarray:
    """2*pi*(phase/2^64) in [-pi, pi) for uint64 phases."""
    return words_times_m.view(np.int64).astype(np.float64) * (np.pi / 2.0 ** 63)


def _period(words: np.ndarray) -> int:
    """Smallest power-of-two period P <= 2^16 of the comb, or 0 if none."""
    for b in range(0, 17):
        mask = np.uint64((1 << (64 - b)) - 1) if b > 0 else np.uint64(0xFFFFFFFFFFFFFFFF)
        if b == 0:
            if np.all(words == 0):
                return 1
            continue
        if np.all((words & mask) == 0):
            return 1 << b
    return 0


class PeriodicComb:
    """A comb whose period P divides 2^16: x[m] = one[m mod P], materialised
    chunk by chunk (slicing returns an ndarray)."""

    def __init__(self, one: np.ndarray, n: int):
        self.one, self.shape, self.dtype = one, (n,), one.dtype

    def __len__(self):
        return self.shape[0]

    def __getitem__(self, sl):
        a, b, _ = sl.indices(self.shape[0])
        return self.one[np.arange(a, b) % len(self.one)]

    def __array__(self, dtype=None, copy=None):
        return self[0:self.shape[0]].astype(dtype or self.dtype)


def tone_comb(n: int, words, amps, phases, block: int = 4096,
              dtype=np.complex128) -> np.ndarray:
    """Noise-free complex comb sum_i A_i exp(i(phi_i(m) + theta_i)), m < n."""
    words = np.asarray(words, np.uint64)
    coef = np.asarray(amps, np.float64) * np.exp(1j * np.asarray(phases, np.float64))
    if len(words) == 0:
        return np.zeros(n, dtype)
    P = _period(words)
    with np.errstate(over="ignore"):
        if P and P <= 65536:
            m = np.arange(P, dtype=np.uint64)
            E = np.exp(1j * _angle(np.multiply.outer(m, words)))      # [P, tones]
            one = (E @ coef).astype(dtype)
            return PeriodicComb(one, n)
        # general comb: x[B*q + j] = sum_i E[j, i] * c_q[i] with
        # E[j, i] = exp(i*phi_i(j)) and c_q[i] = coef_i * exp(i*phi_i(B*q))
        B = block
        j = np.arange(B, dtype=np.uint64)
        E = np.exp(1j * _angle(np.multiply.outer(j, words))).astype(dtype)
        out = np.empty(n, dtype)
        Q = -(-n // B)
        qc = 1024
        for q0 in range(0, Q, qc):
            q = np.arange(q0, min(Q, q0 + qc), dtype=np.uint64)
            ph = np.multiply.outer(q * np.uint64(B), words)               # [q, tones]
            Cq = (np.exp(1j * _angle(ph)) * coef[None, :]).astype(dtype)  # [q, tones]
            blk = (Cq @ E.T).reshape(-1)                                  # [q*B]
            a = q0 * B
            b = min(n, a + blk.size)
            out[a:b] = blk[: b - a]
        return out


def quantise(z: np.ndarray, sigma: float, rng: np.random.Generator, scale: float = 1.0,
             chunk: int = 1 << 24) -> np.ndarray:
    """s*z + sigma*(gI + i gQ) -> int16 [n, 2], round half-even, clamp 14-bit."""
    n = z.shape[0]
    out = np.empty((n, 2), np.int16)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        re = z[a:b].real * scale
        im = z[a:b].imag * scale
        if sigma > 0:
            g = rng.standard_normal((b - a, 2))
            re = re + sigma * g[:, 0]
            im = im + sigma * g[:, 1]
        out[a:b, 0] = np.clip(np.rint(re), -FULL_SCALE - 1, FULL_SCALE)
        out[a:b, 1] = np.clip(np.rint(im), -FULL_SCALE - 1, FULL_SCALE)
    return out


def rms_scale(amps, sigma: float) -> float:
    """Scale for the 'rms' rule (per-component RMS of the composite = 8191/6)."""
    a = np.asarray(amps, np.float64)
    target = (FULL_SCALE / 6.0) ** 2 - sigma ** 2
    p = 0.5 * float(np.sum(a * a))
    return float(np.sqrt(max(target, 0.0) / p)) if p > 0 else 1.0


def distinct_bins(rng: np.random.Generator, n_chan: int, count: int, min_sep: int = 1) -> np.ndarray:
    """count distinct bins of an n_chan-bin PFB, pairwise circular separation
    >= min_sep (min_sep=2: no two tones in adjacent bins)."""
    if count * min_sep > n_chan:
        raise ValueError("too many tones for the requested separation")
    taken = np.zeros(n_chan, bool)
    chosen = []
    for c in rng.permutation(n_chan):
        if len(chosen) == count:
            break
        lo, hi = c - (min_sep - 1), c + (min_sep - 1)
        idx = np.arange(lo, hi + 1) % n_chan
        if not taken[idx].any():
            taken[c] = True
            chosen.append(int(c))
    if len(chosen) < count:
        raise ValueError("could not place the tones")
    return np.array(chosen, np.int64)


def bin_words(bins, n_chan: int) -> np.ndarray:
    """Bin-centred uint64 words c * 2^64 / N, rounded to the nearest integer
    (exact for N a power of two)."""
    n = int(n_chan)
    return np.array([((int(c) << 64) + n // 2) // n % 2 ** 64 for c in bins], np.uint64)


def random_words(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform random uint64 words (tones anywhere in +/- fs/2, off-bin)."""
    return rng.integers(0, 2 ** 64 - 1, size=count, dtype=np.uint64, endpoint=True)


# --------------------------------------------------------------------------
# Workload recipes (sizes, distributions and structure of the paper's use)
# --------------------------------------------------------------------------

def pfb_case(n: int, n_chan: int, n_tones: int, *, seed: int, amp=(500.0, 3000.0),
             sigma: float = 8.0, rule: str = "none", min_sep: int = 1):
    """Tones at distinct random bin centres of an n_chan-channel PFB.

    rule "none": A ~ U(amp) as given (clipping allowed);
    rule "sum":  A = a*U(0.5, 1) with a chosen so sum(A) + 4*sigma = 8191."""
    r = rng_for(seed)
    bins = distinct_bins(r, n_chan, n_tones, min_sep)
    words = bin_words(bins, n_chan)
    if rule == "sum":
        u = r.uniform(0.5, 1.0, n_tones)
        amps = u * (FULL_SCALE - 4.0 * sigma) / float(np.sum(u))
    else:
        amps = r.uniform(amp[0], amp[1], n_tones)
    th = r.uniform(0.0, 2 * np.pi, n_tones)
    z = tone_comb(n, words, amps, th)
    x = quantise(z, sigma, r)
    return {"x": x, "words": words, "bins": bins, "amps": amps, "phases": th,
            "sigma": sigma, "seed": seed}


def demod_case(n: int, n_tones: int, *, seed: int, amp=(100.0, 1000.0), sigma: float = 8.0,
               dtype=np.complex128):
    """Tones at uniform random (off-bin) words, scaled by the 'rms' rule."""
    r = rng_for(seed)
    words = random_words(r, n_tones)
    amps = r.uniform(amp[0], amp[1], n_tones)
    th = r.uniform(0.0, 2 * np.pi, n_tones)
    s = rms_scale(amps, sigma)
    z = tone_comb(n, words, amps, th, dtype=dtype)
    x = quantise(z, sigma, r, scale=s)
    return {"x": x, "words": words, "amps": amps * s, "phases": th, "sigma": sigma,
            "scale": s, "seed": seed}


# The five workloads (sizes from the benchmark definition).
C1 = dict(n=1 << 20, n_chan=64, taps=4, window="hann", beta=0.0, n_tones=16, sigma=8.0)
C2 = dict(n=1 << 28, n_chan=4096, taps=8, window="kaiser", beta=9.0, n_tones=1000, sigma=4.0)
C3 = dict(n=1 << 27, n_tones=2048, L=4096, D=2048, window="blackman", fc=40e3 / 200e6,
          sigma=8.0)


def c1(seed: int = SEED_BASE + 1, n: int | None = None):
    return pfb_case(n or C1["n"], C1["n_chan"], C1["n_tones"], seed=seed,
                    sigma=C1["sigma"], rule="none")


def c2(seed: int = SEED_BASE + 2, n: int | None = None):
    return pfb_case(n or C2["n"], C2["n_chan"], C2["n_tones"], seed=seed,
                    sigma=C2["sigma"], rule="sum", min_sep=2)


def c3(seed: int = SEED_BASE + 3, n: int | None = None, n_tones: int | None = None,
       dtype=np.complex64):
    return demod_case(n or C3["n"], n_tones or C3["n_tones"], seed=seed, sigma=C3["sigma"],
                      dtype=dtype)


def mixed_specs(count: int, seed: int, log2_n=(22.0, 26.0), round_to: int = 1024):
    """Stream specs of the batched workload: each stream is a PFB (p = 0.5;
    N in {256, 1024, 4096, 16384}, T in {4, 8, 16}, min(1000, N/4) tones at bin
    centres, Kaiser(9)) or a demodulation (2^U(6, 12) tones, L in {1024, 4096},
    D in {512, 2048}, Blackman 40 kHz), with 2^U(log2_n) samples rounded to a
    multiple of `round_to`."""
    r = rng_for(seed)
    specs = []
    for i in range(count):
        n = int(round(2.0 ** r.uniform(*log2_n)))
        n = max(round_to, n - n % round_to)
        if r.uniform() < 0.5:
            N = int(r.choice([256, 1024, 4096, 16384]))
            T = int(r.choice([4, 8, 16]))
            specs.append(dict(kind="pfb", N=N, T=T, tones=min(1000, N // 4), n=n, seed=seed * 100 + i))
        else:
            nt = int(round(2.0 ** r.uniform(6.0, 12.0)))
            L = int(r.choice([1024, 4096]))
            D = int(r.choice([512, 2048]))
            specs.append(dict(kind="demod", tones=nt, L=L, D=D, n=n, seed=seed * 100 + i))
    return specs


def spec_input(spec: dict, n: int | None = None):
    """Synthetic input of one mixed-workload stream (signal model as in the
    PFB and demodulation workloads)."""
    n = n or spec["n"]
    if spec["kind"] == "pfb":
        sep = 2 if 2 * spec["tones"] <= spec["N"] else 1
        return pfb_case(n, spec["N"], spec["tones"], seed=spec["seed"], sigma=4.0, rule="sum", min_sep=sep)
    return demod_case(n, spec["tones"], seed=spec["seed"], dtype=np.complex64)


def c4_specs(seed: int = SEED_BASE + 4):
    """24 streams of 2^22 .. 2^26 samples (log-uniform), PFB or demodulation."""
    return mixed_specs(24, seed)


def c5_specs(seed: int = SEED_BASE + 5):
    """32 readouts with plans drawn as in the batched workload."""
    return mixed_specs(32, seed)


def c5_buffer_samples(rng: np.random.Generator, count: int) -> np.ndarray:
    """Buffer sizes of the serving workload: log-uniform 1 .. 32 MB of complex
    int16 (4 bytes per sample), rounded to a multiple of 1024 samples."""
    b = np.exp(rng.uniform(np.log(1 << 20), np.log(32 << 20), count)) / 4.0
    return np.maximum(1024, (b // 1024).astype(np.int64) * 1024)
