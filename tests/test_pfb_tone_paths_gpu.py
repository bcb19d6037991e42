"""Tone outputs of the N = 4096 PFB kernel (Sec. III.A: each tone's channel
is its bin of the frame spectrum) along every output path: tones held in
shared memory (whole output groups by 2-D TMA stores, partial groups and
unaligned rows by plain stores), tones beyond shared memory (gathered from
the spectrum), bins shared by several tones, any output frame offset and row
pitch, and streams split at any frame.  Each path must give, bit for bit, the
spectrum's own value at the tone's bin and the same values as one push."""
import numpy as np
import pytest

import siggen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
N, T = 4096, 8


def _words(nt, seed, dup=0):
    rng = siggen.rng_for(seed)
    bins = siggen.distinct_bins(rng, N, nt - dup)
    if dup:
        bins = np.concatenate([bins, bins[:dup]])      # tones sharing a bin
    return siggen.bin_words(bins, N)


def _x(n, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randint(-4000, 4000, (n, 2), dtype=torch.int16, generator=g).to(DEV)


@pytest.mark.parametrize("nt,dup", [(1000, 0), (37, 5), (1500, 0)])
def test_tones_equal_spectrum_columns(lib, nt, dup):
    """1000 tones (shared-memory tile), 37 with 5 repeated bins, 1500 (beyond
    the shared-memory tile: gathered from the spectrum)."""
    words = _words(nt, 300 + nt, dup)
    p = lib.Plan(N, T, window="kaiser", beta=9.0, words=words)
    F = 152 * 12 + 5
    x = _x(F * N, 7)      # zero history: one frame per N samples
    assert p.frames_for(x.shape[0]) == F
    full = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    tones = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert p.push_into(x, full, tones) == F
    torch.cuda.synchronize()
    bins = p.bins()
    f = full.cpu().numpy()
    assert np.array_equal(tones.cpu().numpy(), f[:, bins].T)


@pytest.mark.parametrize("offset,pad", [(0, 0), (5, 0), (5, 7), (2, 1), (3, 2)])
def test_tone_groups_any_offset_and_pitch(lib, offset, pad):
    """Output frame offsets that shift the 4-frame groups, and row pitches
    that are odd (no TMA) or even (TMA), give the values of an aligned push."""
    nt = 200
    words = _words(nt, 41)
    F = 152 * 8 + 3
    x = _x(F * N, 8)
    ref_p = lib.Plan(N, T, window="kaiser", beta=9.0, words=words, full=False)
    ref = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert ref_p.push_into(x, None, ref) == F
    p = lib.Plan(N, T, window="kaiser", beta=9.0, words=words, full=False)
    ld = offset + F + pad
    buf = torch.full((nt, ld), complex(7.0, -7.0), dtype=torch.complex64, device=DEV)
    assert p.push_into(x, None, buf, frame_offset=offset) == F
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    assert np.array_equal(b[:, offset:offset + F], ref.cpu().numpy())
    # nothing outside the frames written
    assert np.all(b[:, :offset] == np.complex64(complex(7.0, -7.0)))
    assert np.all(b[:, offset + F:] == np.complex64(complex(7.0, -7.0)))


def test_tone_groups_split_stream(lib):
    """A stream pushed in pieces ending at frames 1, 3, 7 and 600 (groups cut
    anywhere) gives the values of one push."""
    nt = 300
    words = _words(nt, 52, dup=3)
    F = 152 * 6 + 11
    x = _x(F * N, 9)
    one = lib.Plan(N, T, window="kaiser", beta=9.0, words=words)
    f1 = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    t1 = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert one.push_into(x, f1, t1) == F
    p = lib.Plan(N, T, window="kaiser", beta=9.0, words=words)
    f2 = torch.zeros_like(f1)
    t2 = torch.zeros_like(t1)
    k = 0
    for end_frame in (1, 3, 7, 600, F):
        k += p.push_into(x[k * N:end_frame * N], f2, t2, frame_offset=k)
    torch.cuda.synchronize()
    assert k == F
    assert np.array_equal(f2.cpu().numpy(), f1.cpu().numpy())
    assert np.array_equal(t2.cpu().numpy(), t1.cpu().numpy())
