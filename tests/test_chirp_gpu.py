"""Chirped readout (Sec. III.C, Eq. 1) on the GPU against the FP64 oracle:
synthesis of the transmit chirp (every int16 sample equal to the oracle's,
which rounds in FP64) and demodulation of a stream against chirps (relative
error <= 1e-5 per chirp; streamed = one-shot bit-exactly)."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FS = 200e6


def _chirps(n, seed):
    r = np.random.default_rng(seed)
    f0 = r.uniform(-80e6, 80e6, n)
    k = r.uniform(-5e13, 5e13, n)           # up to 50 MHz per ms
    s = [oracle.freq_to_word(f, FS) for f in f0]
    rw = [oracle.chirp_rate_word(kk, FS) for kk in k]
    return np.array(s, np.uint64), np.array(rw, np.uint64)


@pytest.mark.parametrize("amp,m0,n", [(8000.0, 0, 1 << 20), (32767.0, -12345, 300001), (123.456, 10 ** 9, 4097),
                                      (32767.0, 7, 1 << 22), (30000.3, -(1 << 40), 2049), (0.0, 0, 100), (1.5, 3, 1)])
def test_chirp_synthesis_matches_oracle(lib, amp, m0, n):
    s, r = _chirps(1, 3 + n)
    assert lib.chirp_rate_word(2.5e13, FS) == oracle.chirp_rate_word(2.5e13, FS)
    out = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    lib.chirp_synthesize(int(s[0]), int(r[0]), amp, m0, out)
    torch.cuda.synchronize()
    ref = oracle.chirp_synth(int(s[0]), int(r[0]), amp, m0, n)
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("L,D,nc,win,fc", [(1024, 512, 3, "rect", 0.0), (4096, 2048, 8, "blackman", 2e-4),
                                           (700, 1000, 2, "hann", 1e-3), (16384, 4096, 3, "blackman", 1e-4),
                                           (256, 64, 40, "hamming", 5e-3)])
def test_chirp_demod_parity(lib, L, D, nc, win, fc):
    s, r = _chirps(nc, 11 + L)
    n = D * 120 + 77
    # Rx: the chirps themselves (loop-back) plus a tone comb and noise
    tx = sum(oracle.chirp_synth(int(s[c]), int(r[c]), 900.0, 0, n).astype(np.int32) for c in range(nc))
    comb = siggen.demod_case(n, 50, seed=5)["x"].astype(np.int32)
    x = np.clip(tx + comb // 4, -8192, 8191).astype(np.int16)
    plan = lib.Plan.chirp(L, s, r, window=win, cutoff=fc, decimation=D)
    xt = torch.from_numpy(x).to(DEV)
    F = plan.frames_for(n)
    out = torch.zeros((nc, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(xt, tones=out) == F
    torch.cuda.synchronize()
    h = oracle.lowpass(win, L, fc)
    ref = oracle.chirp_demod(x, L, D, h, s, r)
    e = rel_rows(out.cpu().numpy(), ref)
    print(f"chirp L={L} D={D}: max rel err {e.max():.3e}")
    assert e.max() < TOL
    # streamed in random pieces = one shot, bit-exactly
    p2 = lib.Plan.chirp(L, s, r, window=win, cutoff=fc, decimation=D)
    out2 = torch.zeros((nc, F), dtype=torch.complex64, device=DEV)
    rng = np.random.default_rng(1)
    pos = off = 0
    while pos < n:
        cnt = int(min(n - pos, rng.integers(1, 7 * D)))
        off += p2.push_into(xt[pos:pos + cnt], tones=out2, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F and torch.equal(out, out2)


def test_chirp_loopback_through_the_gpu(lib):
    """Synthesise a chirp on the GPU, demodulate it against itself with a
    square window: a constant A (Sec. III.C: demodulate the Rx signal against
    the generated waveform)."""
    s, r = _chirps(1, 77)
    D = L = 256
    x = torch.empty((D * 64, 2), dtype=torch.int16, device=DEV)
    lib.chirp_synthesize(int(s[0]), int(r[0]), 5000.0, 0, x)
    plan = lib.Plan.chirp(L, s, r, window="rect", decimation=D)
    out = torch.zeros((1, 64), dtype=torch.complex64, device=DEV)
    plan.push_into(x, tones=out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()[0, 1:]
    assert np.all(np.abs(o - 5000.0) < 0.5)


def test_chirp_invalid(lib):
    s, r = _chirps(1, 1)
    with pytest.raises(lib.RfrError):
        lib.Plan.chirp(0, s, r, decimation=64)
    p = lib.Plan.chirp(64, s, r, decimation=64)
    with pytest.raises(lib.RfrError) as ei:
        p.plain_oneshot(torch.zeros((128, 2), dtype=torch.int16, device=DEV),
                        tones=torch.zeros((1, 2), dtype=torch.complex64, device=DEV))
    assert ei.value.status == lib.E_UNSUPPORTED
    with pytest.raises(lib.RfrError):
        lib.chirp_synthesize(int(s[0]), int(r[0]), 40000.0, 0, torch.zeros((8, 2), dtype=torch.int16, device=DEV))
