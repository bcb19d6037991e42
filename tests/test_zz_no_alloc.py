"""The allocation-free demodulation entry point (rfr_demod_noalloc), for
callers that cannot allocate device memory while running (e.g. a real-time
processing thread), checked through the C ABI against the regular plan path
(rfr_plan_create + rfr_push_into on a fresh plan) on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import siggen
from helpers import TOL, rel_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _noalloc(lib):
    f = lib._lib.rfr_demod_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                  C.c_void_p, C.c_int64, C.c_void_p]
    return f


def test_noalloc_matches_plan_path_two_calls(lib):
    f = _noalloc(lib)
    L, D = 1024, 512
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, nt, seed) in enumerate([((1 << 18) - 77, 200, 71), (150 * 512 + 3, 37, 72)]):
        case = siggen.demod_case(n, nt, seed=seed)
        plan = lib.Plan(0, L, window="blackman", cutoff=1e-3, words=case["words"], decimation=D)
        x = torch.from_numpy(case["x"]).to(DEV)
        F = plan.frames_for(n)
        assert F == n // D
        ref = torch.zeros((nt, F), dtype=torch.complex64, device=DEV)
        plan.push_into(x, tones=ref)
        h64, _ = plan.taps_table()
        words = np.ascontiguousarray(case["words"], np.uint64)
        got = torch.full((nt, F), float("nan"), dtype=torch.complex64, device=DEV)
        st = f(x.data_ptr(), n, h64.ctypes.data, L, D, words.ctypes.data, nt, got.data_ptr(), F, stream)
        assert st == lib.OK, (call, st)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        e = rel_rows(g, r)
        print(f"call {call}: max rel diff vs plan path {e.max():.3e}, identical={np.array_equal(g, r)}")
        assert np.isfinite(g).all()
        assert e.max() < TOL
        plan.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    f = _noalloc(lib)
    h = np.full(64, 1.0 / 64)
    w = np.array([1 << 60], np.uint64)
    out = torch.zeros((1, 8), dtype=torch.complex64, device=DEV)
    x = torch.zeros((512 * 8, 2), dtype=torch.int16, device=DEV)
    big = [((1 << 18) + 1, 64, 512, 1), (4096, 2048, 512, 1), (4096, 64, 512, 257), (4096, 64, 100, 1)]
    for n, L, D, nt in big:
        hh = np.full(L, 1.0 / L)
        ww = np.full(nt, 1 << 60, np.uint64)
        st = f(x.data_ptr(), n, hh.ctypes.data, L, D, ww.ctypes.data, nt, out.data_ptr(), 8, None)
        assert st == lib.E_INVALID
    assert f(x.data_ptr(), 4096, h.ctypes.data, 64, 512, w.ctypes.data, 1, out.data_ptr(), 8, None) == lib.OK
    torch.cuda.synchronize()
