"""Integer NCO phase bit-exactness far into a stream: plans positioned with
rfr_plan_seek at absolute sample indices past 2^31, 2^40 and 2^62 (a 200 Ms/s
stream passes 2^31 samples in 11 s and 2^40 in 1.7 hours), one ragged buffer
pushed, every output compared with the FP64 oracle evaluated at the same
absolute origin (Sec. III.B mixer, Sec. III.C chirps, Sec. III.A channels
keeping the phase of the time origin when the hop is below N).

The GPU forms the phase w*m (uint64) of the absolute sample index m exactly,
so its error at any origin is the same as at sample 0; a phase formed in
floating point or from a truncated index would fail here by orders of
magnitude."""
import numpy as np
import pytest

import oracle
import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
ORIGIN_BASES = [2 ** 31, 2 ** 40, 2 ** 62]


def _origin(base, hop, k):
    """A multiple of the hop just past `base`, k hops further."""
    return (base + hop - 1) // hop * hop + k * hop


@pytest.mark.parametrize("base", ORIGIN_BASES)
@pytest.mark.parametrize("L,D,nt,products", [(1024, 512, 48, 3), (1024, 512, 48, 4), (256, 512, 20, 3),
                                             (4096, 2048, 64, 3), (1024, 512, 300, "3-cluster")])
def test_demod_far_origin_matches_oracle(lib, base, L, D, nt, products):
    S = _origin(base, D, 3)
    halo = max(L - D, 0)
    n_push = D * 150 + 33                                  # ragged: a partial frame left over
    c = siggen.demod_case(halo + n_push, nt, seed=base % 1009 + L)
    plan = lib.Plan(0, L, window="blackman", cutoff=1e-3, words=c["words"], decimation=D)
    if products == 4:
        plan.set_demod_products(4)
    elif products == "3-cluster":
        plan.set_demod_pair(True)                       # two-CTA clusters, three tone tiles
    x = torch.from_numpy(c["x"]).to(DEV)
    plan.seek(S, x[:halo] if halo else None)
    info = plan.info()
    assert info["samples_consumed"] == S and info["frames_produced"] == S // D
    F = plan.frames_for(n_push)
    out = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x[halo:], tones=out) == F
    torch.cuda.synchronize()
    h64, _ = plan.taps_table()
    K0 = S // D
    ref = oracle.demod(c["x"], L, D, h64, c["words"], K0, K0 + F, m0=S - halo)
    e = rel_rows(out.cpu().numpy(), ref)
    print(f"demod origin 2^{int(np.log2(base))}+: L={L} D={D} {products} products, max rel err {e.max():.3e}")
    assert e.max() < TOL
    plan.close()


@pytest.mark.parametrize("base", ORIGIN_BASES)
def test_chirp_demod_far_origin_matches_oracle(lib, base):
    L, D, nc = 1024, 512, 4
    r = np.random.default_rng(base % 997)
    sw = np.array([oracle.freq_to_word(f, 200e6) for f in r.uniform(-80e6, 80e6, nc)], np.uint64)
    rw = np.array([oracle.chirp_rate_word(k, 200e6) for k in r.uniform(-5e13, 5e13, nc)], np.uint64)
    S = _origin(base, D, 5)
    halo = L - D
    n_push = D * 120 + 11
    x_np = siggen.demod_case(halo + n_push, 30, seed=base % 991)["x"]
    plan = lib.Plan.chirp(L, sw, rw, window="hann", cutoff=1e-3, decimation=D)
    x = torch.from_numpy(x_np).to(DEV)
    plan.seek(S, x[:halo])
    F = plan.frames_for(n_push)
    out = torch.zeros((nc, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x[halo:], tones=out) == F
    torch.cuda.synchronize()
    h = oracle.lowpass("hann", L, 1e-3)
    K0 = S // D
    ref = oracle.chirp_demod(x_np, L, D, h, sw, rw, K0, K0 + F, m0=S - halo)
    e = rel_rows(out.cpu().numpy(), ref)
    print(f"chirp demod origin 2^{int(np.log2(base))}+: max rel err {e.max():.3e}")
    assert e.max() < TOL
    plan.close()


@pytest.mark.parametrize("base", ORIGIN_BASES)
@pytest.mark.parametrize("N,T,hop", [(1000, 4, 250), (4096, 8, 1024), (4096, 8, 4096), (96, 4, 96)])
def test_pfb_far_origin_matches_oracle(lib, base, N, T, hop):
    """Oversampled plans (hop < N) rotate channel c by exp(-2 pi i c (A mod N)
    / N) with A the absolute first sample of the frame; critically sampled
    ones (hop = N) only index frames absolutely."""
    S = _origin(base, hop, 2)
    halo = N * T - hop
    n_push = hop * 40 + 5
    c = siggen.pfb_case(halo + n_push, N, 12, seed=base % 983 + N)
    plan = lib.Plan(N, T, window="kaiser", beta=9.0, words=c["words"], decimation=hop)
    x = torch.from_numpy(c["x"]).to(DEV)
    plan.seek(S, x[:halo])
    F = plan.frames_for(n_push)
    full = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    tones = torch.zeros((12, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x[halo:], full, tones) == F
    torch.cuda.synchronize()
    _, h32 = plan.taps_table()
    bins = plan.bins()
    K0 = S // hop
    ref = oracle.pfb_hop(c["x"], N, T, hop, h32.astype(np.float64), K0, K0 + F, bins=bins, m0=S - halo)
    et = rel_rows(tones.cpu().numpy(), ref["tones"])
    g = full.cpu().numpy()
    # full spectrum: every channel against max(own norm, RMS channel norm)
    num = np.linalg.norm(g - ref["full"], axis=0)
    own = np.linalg.norm(ref["full"], axis=0)
    ef = num / np.maximum(own, np.sqrt(np.mean(own ** 2)))
    print(f"PFB N={N} hop={hop} origin 2^{int(np.log2(base))}+: tones {et.max():.3e}, full {ef.max():.3e}")
    assert et.max() < TOL and ef.max() < TOL
    plan.close()


@pytest.mark.parametrize("base", ORIGIN_BASES)
def test_chirp_synthesis_far_origin_is_exact(lib, base):
    r = np.random.default_rng(base % 1013)
    s = oracle.freq_to_word(r.uniform(-80e6, 80e6), 200e6)
    q = oracle.chirp_rate_word(r.uniform(-5e13, 5e13), 200e6)
    m0, n = base + 12345, 40001
    out = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    lib.chirp_synthesize(s, q, 20000.0, m0, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.chirp_synth(s, q, 20000.0, m0, n))


@pytest.mark.parametrize("base", ORIGIN_BASES)
def test_tx_far_origin_matches_oracle(lib, base):
    r = siggen.rng_for(base % 1019)
    words = siggen.random_words(r, 64)
    amps = r.uniform(0.5, 1.0, 64)
    amps *= 8000.0 / amps.sum()
    m0, n = base + 777, 8192
    tx = lib.Tx(words, amps)
    e = tx.error_bound
    out = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    tx.synthesize(m0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    val, iq = oracle.tones_synth(words, amps, m0, n)
    v = np.stack([val.real, val.imag], axis=1)
    unique = np.abs(np.abs(v - np.floor(v)) - 0.5) > e
    assert np.array_equal(got[unique], iq.astype(np.int64)[unique])
    amb = ~unique
    assert ((got[amb] == np.floor(v[amb])) | (got[amb] == np.ceil(v[amb]))).all()
    tx.close()


@pytest.mark.parametrize("base", [2 ** 40, 2 ** 62])
def test_cluster_pfb_far_origin_matches_oracle(lib, base):
    """N = 16384, T = 8 on the cluster kernel, seeked past 2^40 and 2^62 with
    its history: frames against the oracle at the same absolute origin."""
    N, T, nt = 16384, 8, 40
    S = _origin(base, N, 2)
    halo = (T - 1) * N
    n_push = N * 12 + 321
    c = siggen.pfb_case(halo + n_push, N, nt, seed=base % 983, amp=(200.0, 1500.0))
    plan = lib.Plan(N, T, window="kaiser", beta=9.0, words=c["words"])
    plan.set_pfb_cluster(True)
    x = torch.from_numpy(c["x"]).to(DEV)
    plan.seek(S, x[:halo])
    F = plan.frames_for(n_push)
    full = torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    tones = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    assert plan.push_into(x[halo:], full, tones) == F
    torch.cuda.synchronize()
    _, h32 = oracle.pfb_prototype(N, T, "kaiser", 9.0)
    K0 = S // N
    ref = oracle.pfb_hop(c["x"], N, T, N, h32.astype(np.float64), k_begin=K0, k_end=K0 + F,
                         bins=plan.bins(), m0=S - halo)
    e = rel_rows(tones.cpu().numpy(), ref["tones"])
    print(f"cluster PFB origin 2^{int(np.log2(base))}+: max tone rel err {e.max():.3e}")
    assert e.max() < TOL
    assert np.array_equal(tones.cpu().numpy(), full.cpu().numpy()[:, plan.bins()].T)
    plan.close()
