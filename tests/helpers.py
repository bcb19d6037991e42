"""Shared test helpers: error metrics and device round trips."""
import numpy as np


def rel_rows(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-row relative RMS error ||got_r - ref_r|| / ||ref_r||."""
    num = np.linalg.norm(got - ref, axis=-1)
    den = np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)
    return num / den


def rel_channels_vs_rms(got_full: np.ndarray, ref_full: np.ndarray) -> np.ndarray:
    """Full-spectrum channels [frames, N]: per channel ||got_c - ref_c|| divided
    by max(||ref_c||, RMS over channels of ||ref_c||): the relative error of
    every channel at or above the RMS channel norm (the tone channels), and
    the error against the RMS norm for the weaker, noise-only channels (their
    strict ratio is not meaningful in FP32 at ~1e-3 of the tone power)."""
    num = np.linalg.norm(got_full - ref_full, axis=0)
    own = np.linalg.norm(ref_full, axis=0)
    rms = np.sqrt(np.mean(own ** 2))
    return num / np.maximum(own, rms)


TOL = 1e-5   # relative RMS error bar per readout channel (FP32 path vs FP64 oracle)
