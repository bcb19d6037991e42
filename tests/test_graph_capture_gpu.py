"""Pushes inside CUDA stream capture (a caller building its own CUDA graph
around the plan's kernels): a push whose size would make the plan grow its
device scratch is refused with RFR_E_INVALID before anything is enqueued
(growth would synchronise the device and break the capture); a push of a
size the plan has already served is captured, and the replayed graph writes
the same frames as the same push made directly."""
import numpy as np
import pytest

import siggen

torch = pytest.importorskip("torch")
# the refused push leaves the first capture empty, which torch reports as a warning
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")]

DEV = "cuda:0"


def _capture(stream, fn):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        fn()
    return g


def _check_refused_then_captured(lib, make, n_small, n_big, out_shape):
    """make(): a fresh plan; out_shape(plan, n): (tones shape, full shape or None)."""
    c = make.case
    x = torch.from_numpy(c["x"]).to(DEV)
    s = torch.cuda.Stream()
    # plan A: warm with a small push, then a bigger push inside capture is refused
    a = make()
    ts, fs = out_shape(a, n_small)
    a.push_into(x[:n_small], *make.outs(ts, fs))
    torch.cuda.synchronize()
    ts, fs = out_shape(a, n_big)
    big_outs = make.outs(ts, fs)
    with pytest.raises(lib.RfrError) as ei:
        _capture(s, lambda: a.push_into(x[n_small:n_small + n_big], *big_outs, stream=s))
    assert ei.value.status == lib.E_INVALID
    torch.cuda.synchronize()
    # plan B: the same warm push, then a push of the served size captured and replayed
    b = make()
    ref = make()
    ts, fs = out_shape(b, n_small)
    b.push_into(x[:n_small], *make.outs(ts, fs))
    ref.push_into(x[:n_small], *make.outs(ts, fs))
    torch.cuda.synchronize()
    ts, fs = out_shape(b, n_small)
    got = make.outs(ts, fs)
    want = make.outs(ts, fs)
    xin = x[n_small:2 * n_small].clone()
    g = _capture(s, lambda: b.push_into(xin, *got, stream=s))
    g.replay()
    ref.push_into(x[n_small:2 * n_small], *want)
    torch.cuda.synchronize()
    for u, v in zip(got, want):
        if u is not None:
            assert torch.equal(u, v)
    for p in (a, b, ref):
        p.close()


class _Maker:
    def __init__(self, fn, case, outs):
        self.fn, self.case, self.outs = fn, case, outs

    def __call__(self):
        return self.fn()


def test_demodulation_push_in_capture(lib):
    L, D, nt = 1024, 512, 100
    case = siggen.demod_case(D * 400, nt, seed=9101)
    mk = _Maker(lambda: lib.Plan(0, L, window="blackman", cutoff=1e-3, words=case["words"], decimation=D),
                case, lambda ts, fs: (None, torch.full(ts, float("nan"), dtype=torch.complex64, device=DEV)))
    _check_refused_then_captured(lib, mk, D * 60, D * 200,
                                 lambda p, n: ((nt, p.frames_for(n)), None))


def test_oversampled_pfb_push_in_capture(lib):
    N, T, hop, nt = 4096, 8, 1024, 30
    case = siggen.pfb_case(hop * 300 + N * T, N, nt, seed=9102)
    mk = _Maker(lambda: lib.Plan(N, T, window="kaiser", beta=9.0, words=case["words"], decimation=hop),
                case, lambda ts, fs: (torch.full(fs, float("nan"), dtype=torch.complex64, device=DEV),
                                      torch.full(ts, float("nan"), dtype=torch.complex64, device=DEV)))
    _check_refused_then_captured(lib, mk, hop * 40 + N * T, hop * 200,
                                 lambda p, n: ((nt, p.frames_for(n)), (p.frames_for(n), N)))


def test_16_tap_pfb_push_in_capture(lib):
    """N = 4096 with 16 taps: the first-half FIR rows are plan scratch too."""
    N, T, nt = 4096, 16, 30
    case = siggen.pfb_case(N * 300, N, nt, seed=9103)
    mk = _Maker(lambda: lib.Plan(N, T, window="kaiser", beta=9.0, words=case["words"]),
                case, lambda ts, fs: (torch.full(fs, float("nan"), dtype=torch.complex64, device=DEV),
                                      torch.full(ts, float("nan"), dtype=torch.complex64, device=DEV)))
    _check_refused_then_captured(lib, mk, N * 56, N * 200,
                                 lambda p, n: ((nt, p.frames_for(n)), (p.frames_for(n), N)))
