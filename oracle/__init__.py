"""FP64 oracle of the readout DSP stage (PFB of Sec. III.A, direct demodulation
of Sec. III.B of arXiv:1812.02200).

TEST INFRASTRUCTURE ONLY: the product package never imports this module.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  The C source (``oracle.c``) is plain single-threaded
FP64 and shares no code with the CUDA path.

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(brute-force DFT and library FFT for power-of-two and mixed-radix lengths,
library windows and Bessel function, closed forms for pure tones and the
Dirichlet kernel, Parseval, linearity, shift, the PFB/demod identity for
bin-centred tones, integer phase and bin rules for any N, the paper's -6 dB
cross-over of adjacent channels from the prototype and from a whole PFB run at
Fig. 3's N = 10^5, Eq. 1's chirp phase checked with Python
integers and against its FP64 formula, the zero-rate chirp equal to the NCO
demodulator, a chirp demodulated against itself, the multi-tone transmit
buffer against the library inverse FFT and its own demodulation).  No function is "parity
unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

WINDOWS = {"rect": 0, "hann": 1, "hamming": 2, "blackman": 3, "kaiser": 4}


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc -O2 (no fast-math) into _build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-Wall",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P = C.c_void_p
        i32, i64, u64, dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "orc_bessel_i0": (dbl, [dbl]),
            "orc_window": (C.c_int, [C.c_int, dbl, i64, P]),
            "orc_lowpass": (C.c_int, [C.c_int, dbl, dbl, i64, P]),
            "orc_pfb_prototype": (C.c_int, [i32, i32, C.c_int, dbl, dbl, P, P]),
            "orc_freq_to_word": (u64, [dbl, dbl]),
            "orc_word_to_bin": (i32, [u64, i32]),
            "orc_nco_phase": (u64, [u64, u64]),
            "orc_dft": (C.c_int, [i32, P, P]),
            "orc_fft": (C.c_int, [i32, P]),
            "orc_pfb_f64": (C.c_int, [P, i64, i32, i32, P, i64, i64, P, P, P, i32, P]),
            "orc_pfb_i16": (C.c_int, [P, i64, i32, i32, P, i64, i64, P, P, i32, P]),
            "orc_demod_f64": (C.c_int, [P, i64, i32, i32, P, P, i32, i64, i64, P]),
            "orc_demod_i16": (C.c_int, [P, i64, i64, i32, i32, P, P, i32, i64, i64, P]),
            "orc_chirp_phase": (u64, [u64, u64, i64]),
            "orc_chirp_rate_word": (u64, [dbl, dbl]),
            "orc_chirp_synth": (C.c_int, [u64, u64, dbl, i64, i64, P]),
            "orc_chirp_demod_i16": (C.c_int, [P, i64, i64, i32, i32, P, P, P, i32, i64, i64, P]),
            "orc_tones_synth": (C.c_int, [P, P, P, i32, i64, i64, P, P]),
            "orc_pfb_hop_i16": (C.c_int, [P, i64, i64, i32, i32, i32, P, i64, i64, P, P, i32, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def bessel_i0(x: float) -> float:
    return _load().orc_bessel_i0(float(x))


def window(kind: str, m: int, beta: float = 0.0) -> np.ndarray:
    w = np.empty(m, np.float64)
    _check(_load().orc_window(WINDOWS[kind], float(beta), int(m), _ptr(w)), "window")
    return w


def lowpass(kind: str, m: int, fc: float, beta: float = 0.0) -> np.ndarray:
    """Windowed sinc with sum 1 (fc <= 0: pure window)."""
    h = np.empty(m, np.float64)
    _check(_load().orc_lowpass(WINDOWS[kind], float(beta), float(fc), int(m), _ptr(h)), "lowpass")
    return h


def pfb_prototype(n_chan: int, taps: int, kind: str, beta: float = 0.0, fc: float = 0.0):
    """Returns (h64, h32) of length n_chan*taps."""
    m = n_chan * taps
    h64 = np.empty(m, np.float64)
    h32 = np.empty(m, np.float32)
    _check(_load().orc_pfb_prototype(int(n_chan), int(taps), WINDOWS[kind], float(beta),
                                     float(fc), _ptr(h64), _ptr(h32)), "pfb_prototype")
    return h64, h32


def freq_to_word(f: float, fs: float) -> int:
    return int(_load().orc_freq_to_word(float(f), float(fs)))


def word_to_bin(word: int, n_chan: int) -> int:
    return int(_load().orc_word_to_bin(int(word) & (2**64 - 1), int(n_chan)))


def nco_phase(word: int, m: int) -> int:
    return int(_load().orc_nco_phase(int(word) & (2**64 - 1), int(m) & (2**64 - 1)))


def dft(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.complex128)
    y = np.empty_like(x)
    _check(_load().orc_dft(len(x), _ptr(x), _ptr(y)), "dft")
    return y


def fft(x: np.ndarray) -> np.ndarray:
    y = np.array(x, np.complex128, copy=True)
    _check(_load().orc_fft(len(y), _ptr(y)), "fft")
    return y


def pfb(x: np.ndarray, n_chan: int, taps: int, h: np.ndarray, k_begin: int = 0,
        k_end: int | None = None, bins=None, want_full: bool = True, want_v: bool = False):
    """PFB over a complex stream.

    x: complex128 [n] (FP64 stream) or int16 [n, 2] (I, Q).  Returns a dict with
    'full' [nk, N] complex128, 'tones' [n_bins, nk], and 'v' [nk, N] (FP64
    input only)."""
    lib = _load()
    h = np.ascontiguousarray(h, np.float64)
    is_i16 = x.dtype == np.int16
    n = x.shape[0]
    if k_end is None:
        k_end = n // n_chan
    nk = k_end - k_begin
    bins_a = None if bins is None else np.ascontiguousarray(bins, np.int32)
    nb = 0 if bins_a is None else len(bins_a)
    full = np.empty((nk, n_chan), np.complex128) if want_full else None
    tones = np.empty((nb, nk), np.complex128) if nb else None
    out = {}
    if is_i16:
        xi = np.ascontiguousarray(x)
        rc = lib.orc_pfb_i16(_ptr(xi), n, n_chan, taps, _ptr(h), k_begin, k_end,
                             _ptr(full), _ptr(bins_a), nb, _ptr(tones))
    else:
        xc = np.ascontiguousarray(x, np.complex128)
        v = np.empty((nk, n_chan), np.complex128) if want_v else None
        rc = lib.orc_pfb_f64(_ptr(xc), n, n_chan, taps, _ptr(h), k_begin, k_end,
                             _ptr(v), _ptr(full), _ptr(bins_a), nb, _ptr(tones))
        if want_v:
            out["v"] = v
    _check(rc, "pfb")
    if want_full:
        out["full"] = full
    if nb:
        out["tones"] = tones
    return out


def pfb_hop(x: np.ndarray, n_chan: int, taps: int, hop: int, h: np.ndarray, k_begin: int = 0,
            k_end: int | None = None, bins=None, want_full: bool = True, m0: int = 0):
    """PFB with `hop` samples between frames on an int16 [n, 2] stream (frames
    end at (k+1)*hop - 1; channels keep the absolute time origin's phase).
    x[i] is the sample at absolute index m0 + i (earlier samples are zero) and
    k_begin, k_end are absolute frame indices.
    Returns a dict with 'full' [nk, N] and 'tones' [n_bins, nk]."""
    h = np.ascontiguousarray(h, np.float64)
    xi = np.ascontiguousarray(x, np.int16)
    n = xi.shape[0]
    if k_end is None:
        k_end = (m0 + n) // hop
    nk = k_end - k_begin
    bins_a = None if bins is None else np.ascontiguousarray(bins, np.int32)
    nb = 0 if bins_a is None else len(bins_a)
    full = np.empty((nk, n_chan), np.complex128) if want_full else None
    tones = np.empty((nb, nk), np.complex128) if nb else None
    _check(_load().orc_pfb_hop_i16(_ptr(xi), n, int(m0), n_chan, taps, hop, _ptr(h), k_begin, k_end, _ptr(full),
                                   _ptr(bins_a), nb, _ptr(tones)), "pfb_hop")
    out = {}
    if want_full:
        out["full"] = full
    if nb:
        out["tones"] = tones
    return out


def demod(x: np.ndarray, L: int, D: int, h: np.ndarray, words, k_begin: int = 0,
          k_end: int | None = None, m0: int = 0) -> np.ndarray:
    """Direct demodulation; returns complex128 [n_words, nk].  For an int16
    stream, x[i] is the sample at absolute index m0 + i (earlier samples are
    zero) and k_begin, k_end are absolute frame indices."""
    lib = _load()
    h = np.ascontiguousarray(h, np.float64)
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    n = x.shape[0]
    if m0 and x.dtype != np.int16:
        raise ValueError("an absolute origin m0 is supported for int16 streams")
    if k_end is None:
        k_end = (m0 + n) // D
    nk = k_end - k_begin
    out = np.empty((len(w), nk), np.complex128)
    if x.dtype == np.int16:
        xi = np.ascontiguousarray(x)
        rc = lib.orc_demod_i16(_ptr(xi), n, int(m0), L, D, _ptr(h), _ptr(w), len(w), k_begin, k_end, _ptr(out))
    else:
        xc = np.ascontiguousarray(x, np.complex128)
        rc = lib.orc_demod_f64(_ptr(xc), n, L, D, _ptr(h), _ptr(w), len(w), k_begin, k_end, _ptr(out))
    _check(rc, "demod")
    return out


def chirp_phase(start_word: int, rate_word: int, m: int) -> int:
    """Eq. 1 in sample units: start*m + rate*m^2 mod 2^64."""
    return int(_load().orc_chirp_phase(int(start_word) & (2 ** 64 - 1), int(rate_word) & (2 ** 64 - 1), int(m)))


def chirp_rate_word(k_hz_per_s: float, fs: float) -> int:
    return int(_load().orc_chirp_rate_word(float(k_hz_per_s), float(fs)))


def chirp_synth(start_word: int, rate_word: int, amp: float, m0: int, n: int) -> np.ndarray:
    out = np.empty((n, 2), np.int16)
    _check(_load().orc_chirp_synth(int(start_word) & (2 ** 64 - 1), int(rate_word) & (2 ** 64 - 1),
                                   float(amp), int(m0), int(n), _ptr(out)), "chirp_synth")
    return out


def chirp_demod(x: np.ndarray, L: int, D: int, h: np.ndarray, start_words, rate_words,
                k_begin: int = 0, k_end: int | None = None, m0: int = 0) -> np.ndarray:
    """Demodulation against chirps; x int16 [n, 2], x[i] the sample at absolute
    index m0 + i (earlier samples zero), absolute frame indices; returns
    complex128 [n_chirps, nk]."""
    lib = _load()
    h = np.ascontiguousarray(h, np.float64)
    sw = np.ascontiguousarray(np.asarray(start_words, dtype=np.uint64))
    rw = np.ascontiguousarray(np.asarray(rate_words, dtype=np.uint64))
    n = x.shape[0]
    if k_end is None:
        k_end = (m0 + n) // D
    out = np.empty((len(sw), k_end - k_begin), np.complex128)
    xi = np.ascontiguousarray(x, np.int16)
    _check(lib.orc_chirp_demod_i16(_ptr(xi), n, int(m0), L, D, _ptr(h), _ptr(sw), _ptr(rw), len(sw), k_begin,
                                   k_end, _ptr(out)), "chirp_demod")
    return out


def tones_synth(words, amps, m0: int, n: int, phase_words=None):
    """Multi-tone transmit samples: returns (values complex128 [n], iq int16 [n, 2])."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    a = np.ascontiguousarray(np.asarray(amps, dtype=np.float64))
    p = None if phase_words is None else np.ascontiguousarray(np.asarray(phase_words, dtype=np.uint64))
    val = np.empty(n, np.complex128)
    iq = np.empty((n, 2), np.int16)
    _check(_load().orc_tones_synth(_ptr(w), _ptr(p), _ptr(a), len(w), int(m0), int(n), _ptr(val), _ptr(iq)),
           "tones_synth")
    return val, iq
