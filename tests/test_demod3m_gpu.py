"""GPU parity of the Gauss three-product form of the tensor-core
demodulation (Sec. III.B; rfr_plan_set_demod_products(plan, 3)) against the
FP64 oracle, through the C ABI: the same definition as the four-product
form with three real contractions per complex multiply-add, the same
tolerance (relative RMS error <= 1e-5 per tone)."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FC = 40e3 / 200e6


def _plan3(lib, L, D, words, win="blackman", fc=FC, beta=0.0):
    p = lib.Plan(0, L, window=win, beta=beta, cutoff=fc, words=words, decimation=D)
    p.set_demod_products(3)
    return p


def _run(plan, x_np, n_tones):
    x = torch.from_numpy(x_np).to(DEV)
    F = plan.frames_for(x.shape[0])
    out = torch.zeros((n_tones, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x, tones=out) == F
    torch.cuda.synchronize()
    return out.cpu().numpy()


SHAPES = [
    # L, D, tones, frames, window, cutoff
    (256, 64, 8, 200, "blackman", 0.01),
    (1000, 512, 130, 140, "hann", 0.002),       # L not a multiple of 64; 2 tone tiles
    (4096, 2048, 160, 130, "blackman", 2e-4),   # the workload's filter
    (4096, 512, 40, 150, "kaiser", 1e-3),       # L = 8 D
    (1024, 2048, 50, 160, "hamming", 1e-3),     # L < D
    (512, 512, 30, 260, "rect", 0.0),           # moving average, D = L
    (3000, 448, 300, 90, "hann", 1e-3),         # 3 tone tiles, D = 7 * 64
]


@pytest.mark.parametrize("L,D,nt,frames,win,fc", SHAPES)
def test_demod3m_parity_shapes(lib, L, D, nt, frames, win, fc):
    beta = 9.0 if win == "kaiser" else 0.0
    case = siggen.demod_case(frames * D + D // 3, nt, seed=3000 + L + D + nt)
    plan = _plan3(lib, L, D, case["words"], win, fc, beta)
    got = _run(plan, case["x"], nt)
    assert got.shape[1] == frames
    ref = oracle.demod(case["x"], L, D, oracle.lowpass(win, L, fc, beta), case["words"])
    e = rel_rows(got, ref)
    print(f"3M L={L} D={D} tones={nt}: max rel err {e.max():.3e}")
    assert e.max() < TOL


def test_demod3m_weak_tones_workload_statistics(lib):
    c = siggen.c3(n=1 << 21)
    L, D = 4096, 2048
    plan = _plan3(lib, L, D, c["words"])
    got = _run(plan, c["x"], 2048)
    h = oracle.lowpass("blackman", L, FC)
    sel = np.concatenate([np.argsort(c["amps"])[:8], np.random.default_rng(1).choice(2048, 8, replace=False)])
    frames = np.unique(np.linspace(0, got.shape[1] - 1, 64).astype(int))
    errs = []
    for s in sel:
        ref = np.concatenate([oracle.demod(c["x"], L, D, h, [c["words"][s]], k, k + 1)[0] for k in frames])
        errs.append(np.linalg.norm(got[s, frames] - ref) / np.linalg.norm(ref))
    errs = np.array(errs)
    print(f"3M weakest-tone rel err {errs[:8].max():.3e}, random {errs[8:].max():.3e}")
    assert errs.max() < TOL


def test_demod3m_c3_full_size_sampled(lib):
    c = siggen.c3()
    L, D = 4096, 2048
    plan = _plan3(lib, L, D, c["words"])
    got = _run(plan, c["x"], 2048)
    assert got.shape == (2048, 65536)
    h = oracle.lowpass("blackman", L, FC)
    sel = np.concatenate([np.argsort(c["amps"])[:4], [0, 1000, 2047]])
    for a, b in [(0, 8), (32760, 32768), (65528, 65536)]:
        ref = oracle.demod(c["x"], L, D, h, c["words"][sel], a, b)
        e = np.linalg.norm(got[sel, a:b] - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert e.max() < TOL, (a, e.max())


def test_demod3m_full_range_int16(lib):
    """Samples over the whole int16 range (xr + xi up to 65534, beyond the
    largest FP16 number without the halving of the sum)."""
    r = np.random.default_rng(17)
    L, D, nt, frames = 1024, 512, 40, 80
    x = r.integers(-32768, 32768, size=(frames * D, 2)).astype(np.int16)
    x[::7] = 32767
    x[3::11] = -32768
    words = siggen.random_words(r, nt)
    plan = _plan3(lib, L, D, words)
    got = _run(plan, x, nt)
    ref = oracle.demod(x, L, D, oracle.lowpass("blackman", L, FC), words)
    e = rel_rows(got, ref)
    print(f"3M full-range: max rel err {e.max():.3e}")
    assert np.isfinite(got).all() and e.max() < TOL


def test_demod3m_streamed_equals_one_shot_bit_exact(lib):
    L, D, nt = 1024, 512, 150
    case = siggen.demod_case(D * 400 + 77, nt, seed=31)
    ref = _run(_plan3(lib, L, D, case["words"]), case["x"], nt)
    st = _plan3(lib, L, D, case["words"])
    x = torch.from_numpy(case["x"]).to(DEV)
    F = ref.shape[1]
    out = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    rng = np.random.default_rng(8)
    pos = off = 0
    while pos < x.shape[0]:
        cnt = int(min(x.shape[0] - pos, rng.integers(1, 40 * D)))
        off += st.push_into(x[pos:pos + cnt], tones=out, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F and np.array_equal(out.cpu().numpy(), ref)


def test_demod3m_switching_forms(lib):
    """A fresh plan with D % 64 == 0 is in the three-product form; switching
    4 -> 3 -> 4 gives each form's results again bit for bit; D % 64 != 0 is
    refused for the three-product form."""
    L, D, nt = 1024, 512, 20
    case = siggen.demod_case(D * 50, nt, seed=5)
    p = lib.Plan(0, L, window="blackman", cutoff=FC, words=case["words"], decimation=D)
    default = _run(p, case["x"], nt)
    p.reset()
    p.set_demod_products(4)
    four = _run(p, case["x"], nt)
    p.reset()
    p.set_demod_products(3)
    three = _run(p, case["x"], nt)
    p.reset()
    p.set_demod_products(4)
    again = _run(p, case["x"], nt)
    assert np.array_equal(four, again)
    assert np.array_equal(three, default)
    assert rel_rows(three, four).max() < TOL
    q = lib.Plan(0, L, window="blackman", cutoff=FC, words=case["words"], decimation=96)
    with pytest.raises(lib.RfrError) as e:
        q.set_demod_products(3)
    assert e.value.status == -7


@pytest.mark.parametrize("L,D,nt", [(1024, 512, 20), (1000, 512, 130), (4096, 2048, 300), (1024, 2048, 70)])
def test_tone_tile_64_equals_128_and_oracle(lib, L, D, nt):
    """The tile shape is a launch choice: 64 tones per tile (tiles past the
    last tone skipped) gives, bit for bit, the frames of 128 tones per tile,
    and both match the oracle."""
    case = siggen.demod_case(D * 120 + 77, nt, seed=5100 + L + nt)
    a = _plan3(lib, L, D, case["words"], "hann", 1e-3)
    b = _plan3(lib, L, D, case["words"], "hann", 1e-3)
    b.set_tone_tile(64)
    assert a.tune()["tone_tile"] == 128 and b.tune()["tone_tile"] == 64
    ga = _run(a, case["x"], nt)
    gb = _run(b, case["x"], nt)
    assert np.array_equal(ga, gb)
    ref = oracle.demod(case["x"], L, D, oracle.lowpass("hann", L, 1e-3), case["words"])
    assert rel_rows(gb, ref).max() < TOL
    with pytest.raises(lib.RfrError):
        a.set_tone_tile(96)


def test_persistent_gemm_over_many_plans(lib):
    """A batched step with 19 demodulation plans (more than one persistent
    launch holds, both tile widths) and two PFB plans: every stream's frames
    equal the same stream pushed alone."""
    rng = np.random.default_rng(12)
    specs = []
    for i in range(19):
        L = int(rng.choice([256, 1024, 1000]))
        D = int(rng.choice([64, 512, 448]))
        specs.append(("demod", L, D, int(rng.integers(1, 300)), 64 if i % 3 == 0 else 128))
    specs += [("pfb", 1024, 8, 16, 0), ("pfb", 4096, 8, 24, 0)]
    plans_b, plans_a, xs, outs_b, outs_a = [], [], [], [], []
    for i, (kind, a1, a2, nt, bt) in enumerate(specs):
        if kind == "demod":
            c = siggen.demod_case(a2 * int(rng.integers(30, 80)) + int(rng.integers(0, a2)), nt, seed=6000 + i)
            mk = lambda: _plan3(lib, a1, a2, c["words"], "hann", 1e-3)
        else:
            c = siggen.pfb_case(a1 * 60 + 11, a1, nt, seed=6000 + i)
            mk = lambda: lib.Plan(a1, a2, window="hann", words=c["words"], full=False)
        pb, pa = mk(), mk()
        if kind == "demod":
            pb.set_tone_tile(bt)
            pa.set_tone_tile(bt)
        x = torch.from_numpy(c["x"]).to(DEV)
        F = pa.frames_for(x.shape[0])
        plans_b.append(pb)
        plans_a.append(pa)
        xs.append(x)
        outs_b.append(torch.zeros((nt, F), dtype=torch.complex64, device=DEV))
        outs_a.append(torch.zeros((nt, F), dtype=torch.complex64, device=DEV))
    batch = lib.Batch(plans_b)
    half = [x.shape[0] // 2 for x in xs]
    got = batch.push([x[:h] for x, h in zip(xs, half)], None, outs_b)
    batch.push([x[h:] for x, h in zip(xs, half)], None, outs_b, got)
    for p, x, o in zip(plans_a, xs, outs_a):
        p.push_into(x, tones=o)
    torch.cuda.synchronize()
    for i, (ob, oa) in enumerate(zip(outs_b, outs_a)):
        assert torch.equal(ob, oa), i
    batch.close()


FUSED_SHAPES = [
    # L, D, tones, window, cutoff, bt
    (1024, 512, 40, "hann", 1e-3, 128),
    (1000, 512, 130, "hann", 2e-3, 64),       # L not a multiple of 64
    (4096, 2048, 160, "blackman", 2e-4, 128),
    (1024, 2048, 50, "hamming", 1e-3, 128),   # L < D: the view skips D - L samples
    (3000, 448, 300, "hann", 1e-3, 64),
    (256, 64, 8, "blackman", 0.01, 128),
]


@pytest.mark.parametrize("L,D,nt,win,fc,bt", FUSED_SHAPES)
def test_fused_presplit_equals_two_kernels_and_oracle(lib, L, D, nt, win, fc, bt):
    """The FP16 split of the stream done by the GEMM's producer warps gives,
    bit for bit, the frames of the separate pre-split kernel: one push of a
    ragged buffer, then a stream pushed in odd-sized pieces (carry lengths and
    buffer addresses that are not multiples of 4 samples / 16 bytes take the
    per-sample path)."""
    case = siggen.demod_case(D * 90 + 37, nt, seed=7100 + L + nt)
    a = _plan3(lib, L, D, case["words"], win, fc)
    b = _plan3(lib, L, D, case["words"], win, fc)
    a.set_tone_tile(bt)
    b.set_tone_tile(bt)
    b.set_fused_presplit(True)
    assert b.tune()["fused_presplit"] == 1 and a.tune()["fused_presplit"] == 0
    ga = _run(a, case["x"], nt)
    gb = _run(b, case["x"], nt)
    assert np.array_equal(ga, gb)
    ref = oracle.demod(case["x"], L, D, oracle.lowpass(win, L, fc), case["words"])
    assert rel_rows(gb, ref).max() < TOL
    # streamed in odd pieces through the fused form = one push
    c = _plan3(lib, L, D, case["words"], win, fc)
    c.set_tone_tile(bt)
    c.set_fused_presplit(True)
    x = torch.from_numpy(case["x"]).to(DEV)
    F = ga.shape[1]
    out = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    rng = np.random.default_rng(L + D)
    pos, off = 0, 0
    while pos < x.shape[0]:
        cnt = min(int(rng.integers(1, 7 * D)), x.shape[0] - pos)
        off += c.push_into(x[pos:pos + cnt], tones=out, frame_offset=off)
        pos += cnt
    torch.cuda.synchronize()
    assert off == F
    assert np.array_equal(out.cpu().numpy(), ga)


def test_fused_presplit_far_origin_and_batch(lib):
    """The fused form at an absolute origin past 2^40 against the oracle, and
    in a batched step beside plans of the other forms (one persistent launch
    per form) equal to the streams alone."""
    L, D, nt = 2048, 512, 70
    halo = L - D
    S = (2 ** 40 + D - 1) // D * D + 3 * D
    case = siggen.demod_case(halo + D * 100 + 9, nt, seed=7301)
    p = _plan3(lib, L, D, case["words"], "blackman", 1e-3)
    p.set_fused_presplit(True)
    x = torch.from_numpy(case["x"]).to(DEV)
    p.seek(S, x[:halo])
    F = p.frames_for(x.shape[0] - halo)
    out = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert p.push_into(x[halo:], tones=out) == F
    torch.cuda.synchronize()
    h64, _ = p.taps_table()
    ref = oracle.demod(case["x"], L, D, h64, case["words"], S // D, S // D + F, m0=S - halo)
    assert rel_rows(out.cpu().numpy(), ref).max() < TOL
    # batch: fused/unfused x tile widths
    plans_b, plans_a, xs, ob, oa = [], [], [], [], []
    for i, (fused, bt) in enumerate([(1, 128), (0, 128), (1, 64), (0, 64), (1, 128)]):
        c = siggen.demod_case(D * 70 + 11 * i, 30 + 40 * i, seed=7400 + i)
        for lst in (plans_b, plans_a):
            q = _plan3(lib, 1024, D, c["words"], "hann", 1e-3)
            q.set_fused_presplit(bool(fused))
            q.set_tone_tile(bt)
            lst.append(q)
        xs.append(torch.from_numpy(c["x"]).to(DEV))
        Fi = plans_a[-1].frames_for(xs[-1].shape[0])
        ob.append(torch.zeros((30 + 40 * i, Fi), dtype=torch.complex64, device=DEV))
        oa.append(torch.zeros((30 + 40 * i, Fi), dtype=torch.complex64, device=DEV))
    batch = lib.Batch(plans_b)
    batch.push(xs, None, ob)
    for q, xx, o in zip(plans_a, xs, oa):
        q.push_into(xx, tones=o)
    torch.cuda.synchronize()
    for i, (u, v) in enumerate(zip(ob, oa)):
        assert torch.equal(u, v), i
    batch.close()


PAIR_SHAPES = [
    # L, D, tones, frames, tones per tile: odd and even tone-tile counts, ragged frame tiles
    (1024, 512, 20, 130, 128),     # one tone tile: the pair's second CTA works on zero taps
    (1000, 512, 130, 140, 128),    # two tiles, L not a multiple of 64
    (3000, 448, 300, 90, 128),     # three tiles
    (4096, 2048, 160, 129, 64),    # three 64-tone tiles, the workload's filter
    (1024, 2048, 50, 160, 64),     # L < D
    (256, 64, 8, 300, 128),
]


@pytest.mark.parametrize("L,D,nt,frames,bt", PAIR_SHAPES)
def test_pair_form_equals_single_cta_and_oracle(lib, L, D, nt, frames, bt):
    """Two-CTA clusters sharing each frame tile's operand tiles by TMA
    multicast give, bit for bit, the frames of one CTA per tile (the same
    MMAs in the same order), and match the oracle."""
    case = siggen.demod_case(frames * D + D // 5, nt, seed=7700 + L + nt + bt)
    a = _plan3(lib, L, D, case["words"], "hann", 1e-3)
    b = _plan3(lib, L, D, case["words"], "hann", 1e-3)
    for p in (a, b):
        p.set_tone_tile(bt)
    a.set_demod_pair(False)
    b.set_demod_pair(True)
    assert a.tune()["pair"] == 0 and b.tune()["pair"] == 1
    ga = _run(a, case["x"], nt)
    gb = _run(b, case["x"], nt)
    assert np.isfinite(gb).all()
    assert np.array_equal(ga, gb)
    ref = oracle.demod(case["x"], L, D, oracle.lowpass("hann", L, 1e-3), case["words"])
    e = rel_rows(gb, ref)
    print(f"pair form L={L} D={D} tones={nt} bt={bt}: bit-identical to one CTA per tile, max rel err {e.max():.3e}")
    assert e.max() < TOL
    # the fused pre-split has no pair form
    b.set_fused_presplit(True)
    assert b.tune()["pair"] == 0


def test_pair_form_in_batches_with_the_other_forms(lib):
    """A batched step mixing pair, single-CTA and fused plans of both tile
    widths (one persistent launch per form): every stream equals the same
    stream pushed alone in the single-CTA form."""
    D = 512
    forms = [(1, 0, 128), (0, 0, 128), (1, 0, 64), (0, 1, 128), (1, 0, 128), (0, 0, 64), (1, 0, 64)]
    plans_b, plans_a, xs, ob, oa = [], [], [], [], []
    for i, (pair, fused, bt) in enumerate(forms):
        nt = 25 + 61 * i
        c = siggen.demod_case(D * (60 + 7 * i) + 13 * i, nt, seed=7800 + i)
        q = _plan3(lib, 1024, D, c["words"], "hann", 1e-3)
        q.set_tone_tile(bt)
        q.set_demod_pair(bool(pair))
        q.set_fused_presplit(bool(fused))
        plans_b.append(q)
        r = _plan3(lib, 1024, D, c["words"], "hann", 1e-3)
        r.set_tone_tile(bt)
        r.set_demod_pair(False)
        plans_a.append(r)
        xs.append(torch.from_numpy(c["x"]).to(DEV))
        F = r.frames_for(xs[-1].shape[0])
        ob.append(torch.zeros((nt, F), dtype=torch.complex64, device=DEV))
        oa.append(torch.zeros((nt, F), dtype=torch.complex64, device=DEV))
    batch = lib.Batch(plans_b)
    half = [x.shape[0] // 2 for x in xs]
    got = batch.push([x[:h] for x, h in zip(xs, half)], None, ob)
    batch.push([x[h:] for x, h in zip(xs, half)], None, ob, got)
    for q, xx, o in zip(plans_a, xs, oa):
        q.push_into(xx, tones=o)
    torch.cuda.synchronize()
    for i, (u, v) in enumerate(zip(ob, oa)):
        assert torch.equal(u, v), i
    batch.close()
