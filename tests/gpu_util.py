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
