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


# unit roundoff of the arithmetic that rounds each form's results: FP64; FP32
# element and decoder math (the BF16 form too, apart from its Gram operands);
# TF32 operands (11 significant bits); BF16 operands (8 significant bits)
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "bf16": 2.0 ** -24, "tf32": 2.0 ** -11,
                 "bf16_operands": 2.0 ** -9}


def assert_close(a, b, tol, u=2.0 ** -24, floor=None):
    """Norm-wise rel(a, b) < tol and element-wise agreement:
    |a_i - b_i| <= tol (|b_i| + floor max|b|).  The floor gives entries near
    zero (sums that cancel) the rounding error of the largest entry, 256 units
    of roundoff u of the arithmetic: floor = min(1, max(1e-3, 256 u / tol));
    at floor = 1 this is a sup-norm check, which still catches one wrong entry
    that the 2-norm hides.  The message names the worst entry."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if floor is None:
        floor = min(1.0, max(1e-3, 256.0 * u / tol))
    r = rel(a, b)
    e = elementwise_ratio(a, b, tol, floor)
    if not (r < tol and e <= 1.0):
        af, bf = a.ravel(), b.ravel()
        scale = np.abs(bf) + floor * max(float(np.max(np.abs(bf))), 1e-300)
        i = int(np.argmax(np.abs(af - bf) / scale))
        raise AssertionError(f"norm-wise {r:.3e} (tol {tol:g}); element-wise ratio {e:.3f} "
                             f"(floor {floor:.3g}) at flat index {i}: {af[i]!r} vs {bf[i]!r} "
                             f"(max |b| {np.max(np.abs(bf)):.3e})")
