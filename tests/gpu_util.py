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
