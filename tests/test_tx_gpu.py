"""GPU transmit-buffer synthesis (Sec. III: the GPU generates the
transmission buffer from the readout tones) against the FP64 oracle, through
the C ABI.  Every component whose exact value lies farther than the stated
error bound from a rounding tie must equal the oracle's rounding bit for bit;
the few within the bound of a tie must be one of the two neighbours (both
are correct roundings of a value within the bound)."""
import numpy as np
import pytest

import oracle
import siggen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _check(lib, words, amps, m0, n, phases=None):
    tx = lib.Tx(words, amps, phases)
    e = tx.error_bound
    assert 0.0 < e < 0.05 * max(1.0, sum(amps) / 8191.0)
    out = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    tx.synthesize(m0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    val, iq = oracle.tones_synth(words, amps, m0, n, phases)
    v = np.stack([val.real, val.imag], axis=1)
    dist = np.abs(np.abs(v - np.floor(v)) - 0.5)          # distance to the nearest tie
    unique = dist > e
    assert np.array_equal(got[unique], iq.astype(np.int64)[unique])
    amb = ~unique
    ok = (got[amb] == np.floor(v[amb])) | (got[amb] == np.ceil(v[amb]))
    assert ok.all()
    print(f"n={n} tones={len(words)}: bound {e:.2e}, {amb.mean() * 100:.3f}% of components near a tie, "
          f"{(got[amb] != iq.astype(np.int64)[amb]).sum()} of them differ from the oracle")
    return out, tx


@pytest.mark.parametrize("n_tones,n,m0", [(1000, 1 << 15, 123456789), (16, 1 << 16, 0), (1, 4097, -5),
                                          (300, 1, 7), (257, 5000, -(1 << 40))])
def test_tx_matches_oracle(lib, n_tones, n, m0):
    r = siggen.rng_for(77 + n_tones)
    words = siggen.random_words(r, n_tones)
    amps = r.uniform(0.5, 1.0, n_tones)
    amps *= (8191.0 - 32.0) / amps.sum()                     # full scale with 4-sigma room
    phases = siggen.random_words(r, n_tones)
    _check(lib, words, amps, m0, n, phases)


def test_tx_grid_tones_full_amplitude(lib):
    """One bin-centred tone at the int16 limit (bound ~1e-2 LSB)."""
    words = siggen.bin_words([37], 4096)
    out, _ = _check(lib, words, [32767.0], 0, 1 << 14)


def test_tx_any_split_is_the_same_buffer(lib):
    r = siggen.rng_for(3)
    words = siggen.random_words(r, 100)
    amps = np.full(100, 80.0)
    tx = lib.Tx(words, amps)
    n = 10000
    one = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    tx.synthesize(1000, one)
    parts = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    for a, b in [(0, 1), (1, 1500), (1500, 1501), (1501, 7777), (7777, n)]:
        tx.synthesize(1000 + a, parts[a:b])
    torch.cuda.synchronize()
    assert torch.equal(one, parts)


def test_tx_loopback_through_the_demodulator(lib):
    """Transmit 8 tones, demodulate the int16 buffer with a demodulation plan
    at the same words: each channel returns A_t e^{i 2 pi p_t / 2^64} (a
    Blackman low-pass of unit DC gain, 200 kHz cut-off, rejects the other
    tones)."""
    r = siggen.rng_for(9)
    fs = 200e6
    words = np.array([lib.freq_to_word(f, fs) for f in r.uniform(-90e6, 90e6, 8)], np.uint64)
    amps = np.full(8, 1000.0)
    phases = siggen.random_words(r, 8)
    L = D = 8192
    n = D * 64
    tx = lib.Tx(words, amps, phases)
    x = torch.empty((n, 2), dtype=torch.int16, device=DEV)
    tx.synthesize(0, x)
    plan = lib.Plan(0, L, window="blackman", cutoff=1e-3, words=words, decimation=D)
    F = plan.frames_for(n)
    out = torch.zeros((8, F), dtype=torch.complex64, device=DEV)
    plan.push_into(x, tones=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()[:, 1:]
    ang = np.array([((int(p) + 2 ** 63) % 2 ** 64 - 2 ** 63) / 2 ** 64 for p in phases]) * 2 * np.pi
    want = amps * np.exp(1j * ang)
    err = np.abs(got - want[:, None]).max() / amps[0]
    print(f"loop-back max error {err:.2e} of the amplitude")
    assert err < 5e-3


def test_tx_rejects_bad_arguments(lib):
    with pytest.raises(lib.RfrError):
        lib.Tx([1, 2], [1.0, -1.0])
    with pytest.raises(lib.RfrError):
        lib.Tx([], [])
