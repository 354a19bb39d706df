"""Seeded decoder weights (inputs only).

Xavier-uniform weights U(-a, a) with a = sqrt(6 / (fan_in + fan_out)) and
zero biases, drawn with numpy's PCG64 generator from a stated seed.  The
weights are rounded to float32 once here so that the CPU oracle (which
promotes them exactly to float64) and the CUDA path see identical values.
With zero biases and ELU(0) = 0 the decoder maps z = 0 to zero output, so
z = 0 is the rest shape.
"""
import numpy as np


def xavier_decoder(widths, seed):
    """widths = [r, H1, ..., n]; returns (Ws, bs) lists, W_l of shape (out, in)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, bs = [], []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        W = rng.uniform(-a, a, size=(fan_out, fan_in)).astype(np.float32)
        Ws.append(W)
        bs.append(np.zeros(fan_out, dtype=np.float32))
    return Ws, bs
