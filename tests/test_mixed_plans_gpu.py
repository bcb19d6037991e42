"""Plans of every kind together, and the degenerate inputs.  A batch step
(one CUDA-graph launch) over any-N PFB plans (one pass and four-step),
power-of-two PFB, three- and four-product demodulation and chirp plans gives
each stream's frames bit for bit as the same stream pushed alone; empty
pushes, pushes shorter than a frame and zero-length synthesis are no-ops
that leave the stream state intact; the largest tone count gathers exactly
the spectrum's bins."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FC = 40e3 / 200e6


def _make(lib, kind, words):
    if kind == "pfb1000":
        return lib.Plan(1000, 4, window="hann", words=words, full=True, tones=True), 1000
    if kind == "pfb10000":
        return lib.Plan(10000, 4, window="kaiser", beta=9.0, words=words, full=True, tones=True), 10000
    if kind == "pfb256":
        return lib.Plan(256, 8, window="hann", words=words, full=True, tones=True), 256
    if kind in ("dem3", "dem4"):
        p = lib.Plan(0, 1024, window="blackman", cutoff=FC, words=words, decimation=512)
        p.set_demod_products(3 if kind == "dem3" else 4)
        return p, 0
    r = np.random.default_rng(4)
    sw = [lib.freq_to_word(f, 200e6) for f in r.uniform(-80e6, 80e6, len(words))]
    rw = [lib.chirp_rate_word(k, 200e6) for k in r.uniform(-5e13, 5e13, len(words))]
    return lib.Plan.chirp(1024, sw, rw, window="blackman", cutoff=FC, decimation=512), 0


KINDS = ["pfb1000", "pfb10000", "pfb256", "dem3", "dem4", "chirp"]


def _input(kind, seed):
    if kind.startswith("pfb"):
        N = int(kind[3:])
        return siggen.pfb_case(N * 40 + 123, N, 6, seed=seed)
    return siggen.demod_case(512 * 300 + 77, 6, seed=seed)


def _bufs(plan, N, nt, F):
    full = torch.zeros((F, N), dtype=torch.complex64, device=DEV) if N else None
    tones = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    return full, tones


def test_batch_of_every_plan_kind_equals_alone(lib):
    cases = [_input(k, 70 + i) for i, k in enumerate(KINDS)]
    made_b = [_make(lib, k, c["words"]) for k, c in zip(KINDS, cases)]
    made_a = [_make(lib, k, c["words"]) for k, c in zip(KINDS, cases)]
    xs = [torch.from_numpy(c["x"]).to(DEV) for c in cases]
    Fs = [p.frames_for(x.shape[0]) for (p, _), x in zip(made_a, xs)]
    out_b = [_bufs(p, N, 6, F) for (p, N), F in zip(made_b, Fs)]
    out_a = [_bufs(p, N, 6, F) for (p, N), F in zip(made_a, Fs)]
    rng = np.random.default_rng(2)
    splits = [np.sort(np.concatenate([[0, x.shape[0]], rng.integers(1, x.shape[0], 2)])) for x in xs]
    batch = lib.Batch([p for p, _ in made_b])
    offs = [0] * len(KINDS)
    for step in range(3):
        chunk = [x[sp[step]:sp[step + 1]] for x, sp in zip(xs, splits)]
        got = batch.push(chunk, [o[0] for o in out_b], [o[1] for o in out_b], offs)
        offs = [a + b for a, b in zip(offs, got)]
    for i, ((p, _), x, sp) in enumerate(zip(made_a, xs, splits)):
        off = 0
        for step in range(3):
            off += p.push_into(x[sp[step]:sp[step + 1]], out_a[i][0], out_a[i][1], frame_offset=off)
        assert off == offs[i] == Fs[i], KINDS[i]
    torch.cuda.synchronize()
    for k, ob, oa in zip(KINDS, out_b, out_a):
        if ob[0] is not None:
            assert torch.equal(ob[0], oa[0]), k
        assert torch.equal(ob[1], oa[1]), k
    # one stream of the batch against the oracle
    c = cases[1]
    _, h32 = oracle.pfb_prototype(10000, 4, "kaiser", 9.0)
    ref = oracle.pfb(c["x"], 10000, 4, h32.astype(np.float64), bins=made_b[1][0].bins(), want_full=False)
    assert rel_rows(out_b[1][1].cpu().numpy(), ref["tones"]).max() < TOL


@pytest.mark.parametrize("kind", KINDS)
def test_empty_and_short_pushes_keep_the_stream(lib, kind):
    c = _input(kind, 200)
    p1, N = _make(lib, kind, c["words"])
    p2, _ = _make(lib, kind, c["words"])
    x = torch.from_numpy(c["x"]).to(DEV)
    F = p1.frames_for(x.shape[0])
    a = _bufs(p1, N, 6, F)
    b = _bufs(p2, N, 6, F)
    assert p1.push_into(x, a[0], a[1]) == F
    hop = N if N else 512
    off = 0
    off += p2.push_into(x[:0], b[0], b[1], frame_offset=off)             # empty
    assert off == 0
    off += p2.push_into(x[:hop // 3], b[0], b[1], frame_offset=off)       # shorter than a frame
    off += p2.push_into(x[hop // 3:hop // 3], b[0], b[1], frame_offset=off)
    off += p2.push_into(x[hop // 3:], b[0], b[1], frame_offset=off)
    torch.cuda.synchronize()
    assert off == F
    if a[0] is not None:
        assert torch.equal(a[0], b[0])
    assert torch.equal(a[1], b[1])


def test_zero_length_synthesis(lib):
    out = torch.empty((0, 2), dtype=torch.int16, device=DEV)
    lib.chirp_synthesize(1 << 60, 12345, 1000.0, 0, out)
    tx = lib.Tx([1 << 60, 3 << 59], [10.0, 20.0])
    tx.synthesize(7, out)
    torch.cuda.synchronize()


def test_largest_tone_count_gathers_the_bins(lib):
    """65536 tones (the most a plan takes) on a 65536-channel PFB: every bin
    is a tone, so the tone rows are the spectrum transposed, exactly."""
    N, nt = 65536, 65536
    r = np.random.default_rng(9)
    words = siggen.bin_words(r.permutation(N)[:nt], N)
    x = torch.from_numpy(r.integers(-2000, 2000, size=(N * 5, 2)).astype(np.int16)).to(DEV)
    p = lib.Plan(N, 2, window="hann", words=words, full=True, tones=True)
    F = p.frames_for(x.shape[0])
    full = torch.empty((F, N), dtype=torch.complex64, device=DEV)
    tones = torch.empty((nt, F), dtype=torch.complex64, device=DEV)
    assert p.push_into(x, full, tones) == F
    torch.cuda.synchronize()
    bins = p.bins()
    assert np.array_equal(bins[:512], [oracle.word_to_bin(int(w), N) for w in words[:512]])
    assert torch.equal(tones, full[:, torch.from_numpy(bins.astype(np.int64)).to(DEV)].T)
