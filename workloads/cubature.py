"""Uniform seeded cubature draw (inputs only).

S distinct tets drawn uniformly without replacement, each with the same
non-negative weight E / S so that the weights sum to the tet count.
S = 0 (or S >= E) selects every tet with weight 1.
"""
import numpy as np


def draw_cubature(ne, s, seed):
    if s <= 0 or s >= ne:
        return np.arange(ne, dtype=np.int32), np.ones(ne, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.sort(rng.choice(ne, size=s, replace=False)).astype(np.int32)
    return idx, np.full(s, ne / s, dtype=np.float64)
