"""Helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def random_qbar(p, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    return p.X0.ravel() + amp * rng.standard_normal(p.n)


def round_bf16(a):
    """float32 values rounded to the nearest BF16 (ties to even), as float32:
    the weights the BF16 form stores, for building the matching oracle."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32)


def elementwise_ratio(a, b, tol, floor=1e-3):
    """Largest |a_i - b_i| / (tol (|b_i| + floor max|b|)): at most 1 when every
    entry agrees to `tol` relative to its own size, with a floor of `floor`
    times the largest entry for entries near zero."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    if b.size == 0:
        return 0.0
    scale = np.abs(b) + floor * max(float(np.max(np.abs(b))), 1e-300)
    return float(np.max(np.abs(a - b) / (tol * scale)))


def close_elementwise(a, b, tol, floor=1e-3):
    """True when every entry of a matches b to `tol` (see elementwise_ratio)."""
    return elementwise_ratio(a, b, tol, floor) <= 1.0
