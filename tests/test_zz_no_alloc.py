"""The allocation-free demodulation entry point (rfr_demod_noalloc), for
callers that cannot allocate device memory while running (e.g. a real-time
processing thread), checked through the C ABI against the regular plan path
(rfr_plan_create + rfr_push_into on a fresh plan) and against the FP64
oracle, on calls in a row: L > D, L < D (the stream view then skips D - L
samples before the first frame), and the largest buffer with a small D (the
split stream reaching the end of its static region).  After each call the
shared status word is read back through rfr_demod_noalloc_status.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

import oracle
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


def _status(lib, stream):
    g = lib._lib.rfr_demod_noalloc_status
    g.restype = C.c_int
    g.argtypes = [C.c_void_p, C.POINTER(C.c_int32)]
    v = C.c_int32(-1)
    st = g(stream, C.byref(v))
    return st, v.value


# (n, L, D, tones, seed, tones checked against the oracle)
CALLS = [((1 << 18) - 77, 1024, 512, 200, 71, 12),
         (150 * 512 + 3, 1024, 512, 37, 72, 37),
         ((1 << 18), 256, 2048, 37, 73, 37),          # L < D
         ((1 << 18), 1024, 32, 20, 74, 6)]            # 8192 frames, split rows up to the region's end


def test_noalloc_matches_plan_path_and_oracle(lib):
    f = _noalloc(lib)
    stream = torch.cuda.current_stream().cuda_stream
    for call, (n, L, D, nt, seed, n_chk) in enumerate(CALLS):
        case = siggen.demod_case(n, nt, seed=seed)
        plan = lib.Plan(0, L, window="blackman", cutoff=1e-3, words=case["words"], decimation=D)
        plan.set_demod_products(4)            # the form the allocation-free call runs
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
        assert _status(lib, stream) == (lib.OK, 0)
        torch.cuda.synchronize()
        g, r = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(g).all()
        assert np.array_equal(g, r), call      # same kernels, same order: bit-identical
        sel = np.linspace(0, nt - 1, n_chk).astype(int)
        orc = oracle.demod(case["x"], L, D, h64, case["words"][sel])
        e = rel_rows(g[sel], orc)
        print(f"call {call} (n={n}, L={L}, D={D}): bit-identical to the plan path, "
              f"max rel err vs oracle {e.max():.3e} over {n_chk} tones")
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
    assert _status(lib, None) == (lib.OK, 0)
    torch.cuda.synchronize()
