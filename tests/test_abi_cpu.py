"""CPU checks of the boundary: the library builds, loads and exports every
function include/rfr.h declares; its host-only integer rules agree with the
oracle; no compute call is made (no GPU here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rfr.h")


@pytest.fixture(scope="module")
def so():
    from paper_1812_02200_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(rfr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_core_calls():
    names = declared_functions()
    for n in ("rfr_plan_create", "rfr_push", "rfr_pull", "rfr_push_into", "rfr_reset",
              "rfr_state_export", "rfr_state_import", "rfr_plan_get_taps", "rfr_freq_to_word",
              "rfr_word_to_bin", "rfr_status_string", "rfr_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_loads():
    from paper_1812_02200_gb300 import rfr
    assert rfr.version().startswith("rfr")


def test_host_word_and_bin_rules_match_oracle():
    from paper_1812_02200_gb300 import rfr
    r = np.random.default_rng(2)
    fs = 200e6
    for f in list(r.uniform(-1.5 * fs, 1.5 * fs, 200)) + [0.0, fs / 4, -fs / 2, 40e3, 99.99e6]:
        assert rfr.freq_to_word(f, fs) == oracle.freq_to_word(f, fs)
    for n in (2, 3, 16, 64, 100, 4096, 16384, 10 ** 5, 10 ** 7, 2 ** 24):
        for w in r.integers(0, 2 ** 64, 300, dtype=np.uint64):
            assert rfr.word_to_bin(int(w), n) == oracle.word_to_bin(int(w), n)
    assert rfr.word_to_bin(123, 1) == -1


def test_status_strings(so):
    so.rfr_status_string.restype = ctypes.c_char_p
    for s in range(-7, 1):
        assert so.rfr_status_string(s)
