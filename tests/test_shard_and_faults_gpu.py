"""Time-axis sharding with a halo (how one stream splits across plans or
GPUs), reset, and the bounded device-side waits (failure detection without
faulting the GPU)."""
import numpy as np
import pytest

import siggen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.mark.parametrize("kind", ["pfb", "pfb_padded", "pfb_oversampled", "demod", "demod_short"])
def test_two_shards_concatenate_to_one_shot(lib, kind):
    if kind.startswith("pfb"):
        N, T = {"pfb": (1024, 8), "pfb_padded": (512, 3), "pfb_oversampled": (1000, 4)}[kind]
        hop = N // 4 if kind == "pfb_oversampled" else N      # T=3 runs with zero-padded taps
        c = siggen.pfb_case(N * 300 + 17, N, 12, seed=81)
        mk = lambda: lib.Plan(N, T, window="hann", words=c["words"], decimation=hop)
        halo = T * N - hop
    else:
        L, D = (4096, 1024) if kind == "demod" else (1024, 2048)
        c = siggen.demod_case(D * 200 + 33, 90, seed=82)
        mk = lambda: lib.Plan(0, L, window="blackman", cutoff=1e-3, words=c["words"], decimation=D)
        hop, halo = D, max(L - D, 0)
    x = torch.from_numpy(c["x"]).to(DEV)
    one = mk()
    F = one.frames_for(x.shape[0])
    nt = one.n_tones
    ref = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    one.push_into(x, tones=ref) if kind.startswith("demod") else one.push_into(
        x, torch.zeros((F, N), dtype=torch.complex64, device=DEV), ref)
    cut = (x.shape[0] // 2) // hop * hop                       # frame-aligned shard boundary
    a, b = mk(), mk()
    out = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
    full = None if kind.startswith("demod") else torch.zeros((F, N), dtype=torch.complex64, device=DEV)
    fa = a.push_into(x[:cut], full, out)
    b.seek(cut, x[cut - min(halo, cut):cut] if halo > 0 else None)
    assert b.info()["frames_produced"] == cut // hop == fa
    fb = b.push_into(x[cut:], full, out, frame_offset=fa)
    torch.cuda.synchronize()
    assert fa + fb == F
    assert torch.equal(out, ref)


def test_seek_rejects_misaligned_or_short_history(lib):
    c = siggen.pfb_case(64 * 20, 64, 4, seed=1)
    p = lib.Plan(64, 4, window="hann", words=c["words"])
    x = torch.from_numpy(c["x"]).to(DEV)
    with pytest.raises(lib.RfrError):
        p.seek(100, x[:100])                # not a multiple of the hop
    with pytest.raises(lib.RfrError):
        p.seek(640, x[:10])                 # history must be (T-1)*N samples
    p.seek(640, x[640 - 192:640])
    assert p.info()["samples_consumed"] == 640


def test_reset_restarts_the_stream(lib):
    c = siggen.pfb_case(256 * 40, 256, 8, seed=2)
    x = torch.from_numpy(c["x"]).to(DEV)
    p = lib.Plan(256, 8, window="hann", words=c["words"], full=False)
    t1 = torch.zeros((8, 40), dtype=torch.complex64, device=DEV)
    t2 = torch.zeros((8, 40), dtype=torch.complex64, device=DEV)
    p.push_into(x, tones=t1)
    p.reset()
    assert p.info()["samples_consumed"] == 0
    p.push_into(x, tones=t2)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2)


def test_bounded_device_wait_reports_timeout(lib):
    st, dev_status = lib.wait_selftest(20_000_000)      # 20 ms
    assert st == lib.E_TIMEOUT and dev_status == 1
    # the context is still usable afterwards
    x = torch.ones(1024, device=DEV)
    assert float(x.sum()) == 1024.0
    with pytest.raises(Exception):
        raise lib.RfrError(lib.E_TIMEOUT, "status string check")
