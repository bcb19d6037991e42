"""Thin Python binding of the C ABI in include/rfr.h (argument marshalling
only; every step of the computation runs in the library's CUDA kernels).

Device memory and streams come from PyTorch tensors (``data_ptr()``,
``torch.cuda.current_stream().cuda_stream``).  The library must have been
built (``paper_1812_02200_gb300.build.build()``); importing this module
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"librfr.so not found at {LIB_PATH}: build it first with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (nvcc, sm_103a)")

_lib = C.CDLL(LIB_PATH)

OK, E_INVALID, E_NOMEM, E_CUDA, E_TIMEOUT, E_SHORT, E_BUSY, E_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
PLAIN_DEFAULT, PLAIN_CGEMM = 0, 1
WIN = {"rect": 0, "hann": 1, "hamming": 2, "blackman": 3, "kaiser": 4}
OUT_FULL, OUT_TONES = 1, 2
MODE_PFB, MODE_DEMOD = 1, 2


class Window(C.Structure):
    _fields_ = [("kind", C.c_int32), ("beta", C.c_double), ("cutoff", C.c_double)]


class Tones(C.Structure):
    _fields_ = [("words", C.POINTER(C.c_uint64)), ("count", C.c_int32)]


class Output(C.Structure):
    _fields_ = [("full", C.c_void_p), ("full_ld", C.c_int64), ("full_cap", C.c_int64),
                ("tones", C.c_void_p), ("tones_ld", C.c_int64), ("tones_cap", C.c_int64),
                ("frame_offset", C.c_int64), ("frames", C.c_int64)]


class PlanInfo(C.Structure):
    _fields_ = [("mode", C.c_int32), ("channels", C.c_int32), ("taps", C.c_int32),
                ("decimation", C.c_int32), ("n_tones", C.c_int32), ("out_flags", C.c_uint32),
                ("samples_consumed", C.c_int64), ("frames_produced", C.c_int64),
                ("frames_pending", C.c_int64), ("tap_scale", C.c_double)]


class Completion(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("readout", C.c_int32), ("status", C.c_int32),
                ("frames", C.c_int64), ("samples", C.c_int64), ("t_submit_us", C.c_double),
                ("t_admit_us", C.c_double), ("t_done_us", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("queued", C.c_int64), ("in_flight", C.c_int64), ("budget_bytes", C.c_int64),
                ("peak_bytes", C.c_int64)]


_P = C.c_void_p
_SIGS = {
    "rfr_plan_create": (C.c_int, [C.POINTER(_P), C.c_int32, C.c_int32, C.POINTER(Window),
                                  C.POINTER(Tones), C.c_int32, C.c_uint32]),
    "rfr_plan_destroy": (None, [_P]),
    "rfr_plan_get_info": (C.c_int, [_P, C.POINTER(PlanInfo)]),
    "rfr_frames_for": (C.c_int, [_P, C.c_int64, C.POINTER(C.c_int64)]),
    "rfr_push_into": (C.c_int, [_P, _P, C.c_int64, C.POINTER(Output), _P]),
    "rfr_push": (C.c_int, [_P, _P, C.c_int64, _P]),
    "rfr_pull": (C.c_int, [_P, C.POINTER(Output)]),
    "rfr_process_host": (C.c_int, [_P, _P, C.c_int64, C.POINTER(Output)]),
    "rfr_reset": (C.c_int, [_P]),
    "rfr_state_export": (C.c_int, [_P, _P, C.POINTER(C.c_size_t)]),
    "rfr_state_import": (C.c_int, [_P, _P, C.c_size_t]),
    "rfr_plan_get_taps": (C.c_int, [_P, _P, _P, C.POINTER(C.c_int64)]),
    "rfr_plan_get_bins": (C.c_int, [_P, _P, C.POINTER(C.c_int32)]),
    "rfr_plain_oneshot": (C.c_int, [_P, _P, C.c_int64, C.POINTER(Output), _P]),
    "rfr_plain_oneshot_form": (C.c_int, [_P, C.c_int32, _P, C.c_int64, C.POINTER(Output), _P]),
    "rfr_freq_to_word": (C.c_uint64, [C.c_double, C.c_double]),
    "rfr_word_to_bin": (C.c_int32, [C.c_uint64, C.c_int32]),
    "rfr_status_string": (C.c_char_p, [C.c_int]),
    "rfr_last_error": (C.c_char_p, [_P]),
    "rfr_version": (C.c_char_p, []),
    "rfr_batch_create": (C.c_int, [C.POINTER(_P), C.POINTER(_P), C.c_int32]),
    "rfr_batch_destroy": (None, [_P]),
    "rfr_batch_push": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_int64), C.POINTER(Output), _P]),
    "rfr_batch_stats": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "rfr_batch_last_error": (C.c_char_p, [_P]),
    "rfr_plan_autotune": (C.c_int, [_P, C.c_int64, C.c_int32, C.POINTER(C.c_double)]),
    "rfr_plan_get_tune": (C.c_int, [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "rfr_server_create": (C.c_int, [C.POINTER(_P), C.POINTER(_P), C.c_int32, C.c_size_t, C.c_int64]),
    "rfr_server_submit": (C.c_int, [_P, C.c_int32, _P, C.c_int64, C.POINTER(Output), C.c_uint64]),
    "rfr_server_poll": (C.c_int, [_P, C.POINTER(Completion), C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "rfr_server_get_stats": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "rfr_server_destroy": (None, [_P]),
    "rfr_now_us": (C.c_double, []),
    "rfr_plan_seek": (C.c_int, [_P, C.c_int64, _P, C.c_int64]),
    "rfr_plan_set_accum_chunk": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_set_demod_products": (C.c_int, [_P, C.c_int32]),
    "rfr_wait_selftest": (C.c_int, [C.c_int64, C.POINTER(C.c_int32)]),
    "rfr_plan_create_chirp": (C.c_int, [C.POINTER(_P), C.c_int32, C.POINTER(Window), _P, _P, C.c_int32,
                                        C.c_int32]),
    "rfr_chirp_rate_word": (C.c_uint64, [C.c_double, C.c_double]),
    "rfr_chirp_synthesize": (C.c_int, [C.c_uint64, C.c_uint64, C.c_double, C.c_int64, C.c_int64, _P, _P]),
    "rfr_tx_create": (C.c_int, [C.POINTER(_P), _P, _P, _P, C.c_int32]),
    "rfr_tx_synthesize": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P]),
    "rfr_tx_error_bound": (C.c_double, [_P]),
    "rfr_tx_destroy": (None, [_P]),
    "rfr_demod_noalloc": (C.c_int, [_P, C.c_int64, _P, C.c_int32, C.c_int32, _P, C.c_int32, _P, C.c_int64, _P]),
    "rfr_demod_noalloc_status": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "rfr_plan_inject_device_status": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_get_tone_tile": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "rfr_plan_set_tone_tile": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_set_fused_presplit": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_get_fused_presplit": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "rfr_plan_set_demod_pair": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_get_demod_pair": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "rfr_plan_set_pfb_cluster": (C.c_int, [_P, C.c_int32]),
    "rfr_plan_get_pfb_cluster": (C.c_int, [_P, C.POINTER(C.c_int32)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype, _f.argtypes = _res, _args


class RfrError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{_lib.rfr_status_string(status).decode()} ({status}): {msg}")


def version() -> str:
    return _lib.rfr_version().decode()


def freq_to_word(f_hz: float, fs_hz: float) -> int:
    return int(_lib.rfr_freq_to_word(float(f_hz), float(fs_hz)))


def word_to_bin(word: int, n: int) -> int:
    return int(_lib.rfr_word_to_bin(int(word) & (2 ** 64 - 1), int(n)))


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t):
    return None if t is None else t.data_ptr()


def chirp_rate_word(k_hz_per_s: float, fs_hz: float) -> int:
    return int(_lib.rfr_chirp_rate_word(float(k_hz_per_s), float(fs_hz)))


def chirp_synthesize(start_word: int, rate_word: int, amplitude: float, m0: int, out, stream=None):
    """Chirp transmit buffer (Sec. III.C) into the int16 [n, 2] device tensor `out`."""
    st = _lib.rfr_chirp_synthesize(int(start_word) & (2 ** 64 - 1), int(rate_word) & (2 ** 64 - 1),
                                   float(amplitude), int(m0), out.shape[0], out.data_ptr(), _stream_ptr(stream))
    if st != OK:
        raise RfrError(st, "rfr_chirp_synthesize")


class Tx:
    """Multi-tone transmit buffer generator (rfr_tx_*): int16 [n, 2] samples of
    sum_t A_t exp(+i 2 pi (w_t m + p_t) / 2^64)."""

    def __init__(self, words, amplitudes, phase_words=None):
        w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
        a = np.ascontiguousarray(np.asarray(amplitudes, dtype=np.float64))
        p = None if phase_words is None else np.ascontiguousarray(np.asarray(phase_words, dtype=np.uint64))
        h = _P()
        st = _lib.rfr_tx_create(C.byref(h), w.ctypes.data, None if p is None else p.ctypes.data,
                                a.ctypes.data, len(w))
        if st != OK:
            raise RfrError(st, "rfr_tx_create")
        self._h = h

    @property
    def error_bound(self) -> float:
        return float(_lib.rfr_tx_error_bound(self._h))

    def synthesize(self, m0: int, out, stream=None):
        st = _lib.rfr_tx_synthesize(self._h, int(m0), out.shape[0], out.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise RfrError(st, "rfr_tx_synthesize")

    def close(self):
        if getattr(self, "_h", None):
            _lib.rfr_tx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A PFB (channels > 0) or direct-demodulation (channels == 0) plan; a
    chirp-demodulation plan with Plan.chirp(...)."""

    @classmethod
    def chirp(cls, taps: int, start_words, rate_words, *, window: str = "rect", beta: float = 0.0,
              cutoff: float = 0.0, decimation: int):
        self = cls.__new__(cls)
        sw = np.ascontiguousarray(np.asarray(start_words, dtype=np.uint64))
        rw = np.ascontiguousarray(np.asarray(rate_words, dtype=np.uint64))
        w = Window(WIN[window], float(beta), float(cutoff))
        h = _P()
        st = _lib.rfr_plan_create_chirp(C.byref(h), int(taps), C.byref(w), sw.ctypes.data, rw.ctypes.data,
                                        len(sw), int(decimation))
        if st != OK:
            raise RfrError(st, "rfr_plan_create_chirp")
        self._h = h
        self.words, self.rates = sw, rw
        self.channels, self.taps, self.decimation = 0, taps, decimation
        self.out_flags, self.n_tones = OUT_TONES, len(sw)
        return self

    def __init__(self, channels: int, taps: int, *, window: str = "hann", beta: float = 0.0,
                 cutoff: float = 0.0, words=None, decimation: int | None = None,
                 full: bool = True, tones: bool = True):
        words = np.ascontiguousarray(np.asarray([] if words is None else words, dtype=np.uint64))
        self.words = words
        self.channels = channels
        if channels > 0:
            flags = (OUT_FULL if full else 0) | (OUT_TONES if (tones and len(words)) else 0)
            dec = channels if decimation is None else decimation
        else:
            flags = OUT_TONES
            dec = decimation
        w = Window(WIN[window], float(beta), float(cutoff))
        tn = Tones(words.ctypes.data_as(C.POINTER(C.c_uint64)) if len(words) else None, len(words))
        h = _P()
        st = _lib.rfr_plan_create(C.byref(h), int(channels), int(taps), C.byref(w), C.byref(tn),
                                  int(dec), flags)
        if st != OK:
            raise RfrError(st, "rfr_plan_create")
        self._h = h
        self.taps = taps
        self.decimation = dec
        self.out_flags = flags
        self.n_tones = len(words)

    # --------------------------------------------------------------- utils
    def close(self):
        if getattr(self, "_h", None):
            _lib.rfr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != OK:
            raise RfrError(st, f"{what}: {_lib.rfr_last_error(self._h).decode()}")

    def info(self) -> dict:
        i = PlanInfo()
        self._check(_lib.rfr_plan_get_info(self._h, C.byref(i)), "info")
        return {f: getattr(i, f) for f, _ in PlanInfo._fields_}

    def frames_for(self, n: int) -> int:
        f = C.c_int64()
        self._check(_lib.rfr_frames_for(self._h, int(n), C.byref(f)), "frames_for")
        return f.value

    def taps_table(self):
        n = C.c_int64()
        self._check(_lib.rfr_plan_get_taps(self._h, None, None, C.byref(n)), "taps")
        h64 = np.empty(n.value, np.float64)
        h32 = np.empty(n.value, np.float32)
        self._check(_lib.rfr_plan_get_taps(self._h, h64.ctypes.data, h32.ctypes.data, C.byref(n)), "taps")
        return h64, h32

    def bins(self):
        c = C.c_int32()
        self._check(_lib.rfr_plan_get_bins(self._h, None, C.byref(c)), "bins")
        b = np.empty(c.value, np.int32)
        if c.value:
            self._check(_lib.rfr_plan_get_bins(self._h, b.ctypes.data, C.byref(c)), "bins")
        return b

    @staticmethod
    def _out(full, tones, frame_offset):
        o = Output()
        if full is not None:
            o.full, o.full_ld, o.full_cap = full.data_ptr(), full.shape[1], full.shape[0]
        if tones is not None:
            o.tones, o.tones_ld, o.tones_cap = tones.data_ptr(), tones.shape[1], tones.shape[1]
        o.frame_offset = frame_offset
        return o

    # ---------------------------------------------------------------- work
    def push_into(self, x, full=None, tones=None, frame_offset: int = 0, stream=None) -> int:
        """x: int16 [n, 2] device tensor; full: complex64 [cap, >=N]; tones:
        complex64 [n_tones, cap] (device).  Returns frames written."""
        o = self._out(full, tones, frame_offset)
        n = 0 if x is None else x.shape[0]
        self._check(_lib.rfr_push_into(self._h, _ptr(x), n, C.byref(o), _stream_ptr(stream)),
                    "push_into")
        return o.frames

    def push(self, x, stream=None):
        self._check(_lib.rfr_push(self._h, _ptr(x), x.shape[0], _stream_ptr(stream)), "push")

    def pull(self, full=None, tones=None, frame_offset: int = 0) -> int:
        o = self._out(full, tones, frame_offset)
        self._check(_lib.rfr_pull(self._h, C.byref(o)), "pull")
        return o.frames

    def process_host(self, x, full=None, tones=None, frame_offset: int = 0) -> int:
        """Host (ideally pinned) int16 [n, 2] in, host outputs."""
        o = self._out(full, tones, frame_offset)
        self._check(_lib.rfr_process_host(self._h, _ptr(x), x.shape[0], C.byref(o)), "process_host")
        return o.frames

    def plain_oneshot(self, x, full=None, tones=None, stream=None, form: int = 0) -> int:
        """The plain FP32 comparison form; form PLAIN_CGEMM (demodulation
        only) runs cublasCgemm on the materialised Toeplitz matrix."""
        o = self._out(full, tones, 0)
        if form == PLAIN_DEFAULT:
            st = _lib.rfr_plain_oneshot(self._h, _ptr(x), x.shape[0], C.byref(o), _stream_ptr(stream))
        else:
            st = _lib.rfr_plain_oneshot_form(self._h, form, _ptr(x), x.shape[0], C.byref(o), _stream_ptr(stream))
        self._check(st, "plain_oneshot")
        return o.frames

    def reset(self):
        self._check(_lib.rfr_reset(self._h), "reset")

    def set_accum_chunk(self, k_blocks: int):
        self._check(_lib.rfr_plan_set_accum_chunk(self._h, int(k_blocks)), "set_accum_chunk")

    def set_demod_products(self, products: int):
        """Demodulation GEMM form: 3 (Gauss; the default where D % 64 == 0) or
        4 (real embedding of the complex product)."""
        self._check(_lib.rfr_plan_set_demod_products(self._h, int(products)), "set_demod_products")

    def seek(self, start_sample: int, history=None):
        """Start at absolute sample `start_sample` (a multiple of the hop) with
        `history` = the samples just before it (int16 [n, 2] tensor)."""
        n = 0 if history is None else history.shape[0]
        self._check(_lib.rfr_plan_seek(self._h, int(start_sample), _ptr(history), n), "seek")

    def set_tone_tile(self, tones_per_tile: int):
        """Three-product demodulation: tones per GEMM tile (128 or 64);
        result-neutral, normally chosen by autotune()."""
        self._check(_lib.rfr_plan_set_tone_tile(self._h, int(tones_per_tile)), "set_tone_tile")

    def set_fused_presplit(self, on: bool):
        """Three-product demodulation: the FP16 split of the stream inside the
        GEMM's producers (True) or as its own kernel (False); result-neutral,
        normally chosen by autotune()."""
        self._check(_lib.rfr_plan_set_fused_presplit(self._h, 1 if on else 0), "set_fused_presplit")

    def set_demod_pair(self, on: bool):
        """Three-product demodulation: the GEMM in clusters of two CTAs that
        share each frame tile by TMA multicast (True) or one CTA per tile
        (False, the default); result-neutral, normally chosen by autotune()."""
        self._check(_lib.rfr_plan_set_demod_pair(self._h, 1 if on else 0), "set_demod_pair")

    def set_pfb_cluster(self, on: bool):
        """PFB N = 8192 or 16384 with T <= 8: the cluster kernel (True) or the
        direct kernel (False, the default); set before the first push."""
        self._check(_lib.rfr_plan_set_pfb_cluster(self._h, 1 if on else 0), "set_pfb_cluster")

    def inject_device_status(self, status: int):
        """Write the plan's device status word as a timed-out kernel would
        (1), or clear it (0): host-side failure injection for tests."""
        self._check(_lib.rfr_plan_inject_device_status(self._h, int(status)), "inject_device_status")

    def autotune(self, n_samples: int, use_cache: bool = True) -> float:
        ms = C.c_double()
        self._check(_lib.rfr_plan_autotune(self._h, int(n_samples), 1 if use_cache else 0,
                                           C.byref(ms)), "autotune")
        return ms.value

    def tune(self) -> dict:
        a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(_lib.rfr_plan_get_tune(self._h, C.byref(a), C.byref(b), C.byref(c)), "tune")
        t, f, pr, cl = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        self._check(_lib.rfr_plan_get_tone_tile(self._h, C.byref(t)), "tone tile")
        self._check(_lib.rfr_plan_get_fused_presplit(self._h, C.byref(f)), "fused pre-split")
        self._check(_lib.rfr_plan_get_demod_pair(self._h, C.byref(pr)), "pair")
        self._check(_lib.rfr_plan_get_pfb_cluster(self._h, C.byref(cl)), "cluster")
        return {"pfb_lookahead": a.value, "demod_raster": b.value, "tone_tile": t.value,
                "fused_presplit": f.value, "pair": pr.value, "pfb_cluster": cl.value, "tuned": bool(c.value)}

    def state_export(self) -> bytes:
        n = C.c_size_t()
        self._check(_lib.rfr_state_export(self._h, None, C.byref(n)), "state_export")
        buf = C.create_string_buffer(n.value)
        self._check(_lib.rfr_state_export(self._h, buf, C.byref(n)), "state_export")
        return buf.raw[: n.value]

    def state_import(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(_lib.rfr_state_import(self._h, buf, len(blob)), "state_import")


class Batch:
    """Plans that advance together; one step = one CUDA-graph launch."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (_P * len(self.plans))(*[p._h for p in self.plans])
        h = _P()
        st = _lib.rfr_batch_create(C.byref(h), arr, len(self.plans))
        if st != OK:
            raise RfrError(st, "rfr_batch_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.rfr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def push(self, xs, fulls=None, tones=None, frame_offsets=None, stream=None):
        """xs: list of int16 [n_i, 2] device tensors; fulls/tones: lists of
        output tensors (or None) per plan.  Returns frames per plan."""
        n = len(self.plans)
        fulls = fulls or [None] * n
        tones = tones or [None] * n
        frame_offsets = frame_offsets or [0] * n
        bufs = (_P * n)(*[x.data_ptr() if x is not None and x.shape[0] else None for x in xs])
        ns = (C.c_int64 * n)(*[0 if x is None else x.shape[0] for x in xs])
        outs = (Output * n)(*[Plan._out(f, t, o) for f, t, o in zip(fulls, tones, frame_offsets)])
        st = _lib.rfr_batch_push(self._h, bufs, ns, outs, _stream_ptr(stream))
        if st != OK:
            raise RfrError(st, _lib.rfr_batch_last_error(self._h).decode())
        return [outs[i].frames for i in range(n)]

    def stats(self) -> dict:
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        _lib.rfr_batch_stats(self._h, C.byref(a), C.byref(b), C.byref(c))
        return {"steps": a.value, "graph_updates": b.value, "graph_instantiations": c.value}


def wait_selftest(limit_ns: int = 20_000_000):
    """Returns (status, device_status) of the bounded-wait self-test."""
    d = C.c_int32()
    st = _lib.rfr_wait_selftest(int(limit_ns), C.byref(d))
    return st, d.value


def now_us() -> float:
    return float(_lib.rfr_now_us())


class Server:
    """Serving loop over readouts (plans[i] serves readout i)."""

    def __init__(self, plans, mem_budget_bytes: int, max_buffer_samples: int):
        self.plans = list(plans)
        arr = (_P * len(self.plans))(*[p._h for p in self.plans])
        h = _P()
        st = _lib.rfr_server_create(C.byref(h), arr, len(self.plans), int(mem_budget_bytes),
                                    int(max_buffer_samples))
        if st != OK:
            raise RfrError(st, "rfr_server_create")
        self._h = h
        self._keep = {}

    def submit(self, readout: int, x, full=None, tones=None, frame_offset: int = 0, tag: int = 0):
        o = Plan._out(full, tones, frame_offset)
        st = _lib.rfr_server_submit(self._h, int(readout), _ptr(x), 0 if x is None else x.shape[0],
                                    C.byref(o), int(tag))
        if st != OK:
            raise RfrError(st, "rfr_server_submit")

    def poll(self, cap: int = 256, wait_ms: int = 0):
        buf = (Completion * cap)()
        n = C.c_int32()
        st = _lib.rfr_server_poll(self._h, buf, cap, C.byref(n), int(wait_ms))
        if st != OK:
            raise RfrError(st, "rfr_server_poll")
        return [{f: getattr(buf[i], f) for f, _ in Completion._fields_} for i in range(n.value)]

    def stats(self) -> dict:
        s = ServerStats()
        _lib.rfr_server_get_stats(self._h, C.byref(s))
        return {f: getattr(s, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.rfr_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
