"""Voxel tetrahedral meshes of a solid torus (inputs only).

The torus of major radius R and minor radius a, axis z, centred at `center`,
is voxelised on a grid of spacing h: a hex cell of the grid belongs to the
mesh when its centre lies inside the torus, (sqrt(x^2 + y^2) - R)^2 + z^2 <=
a^2 in coordinates relative to the centre.  Every kept cell is split into
the same six Kuhn/Freudenthal tetrahedra as the bar meshes (walks 000 ->
+e_a -> +e_a+e_b -> 111 along the cell's main diagonal, odd axis orderings
with their middle vertices swapped for positive orientation), so the mesh is
conforming.  Only the grid nodes that some kept cell uses become vertices,
numbered in grid order.
"""
from dataclasses import dataclass
import itertools
import numpy as np

from .bar import _PERMS


@dataclass
class TorusMesh:
    X0: np.ndarray        # (nv, 3) float64 rest positions
    tets: np.ndarray      # (ne, 4) int32 vertex indices
    h: float

    @property
    def nv(self):
        return self.X0.shape[0]

    @property
    def ne(self):
        return self.tets.shape[0]


def make_torus(R, a, h, center=(0.0, 0.0, 0.0)):
    center = np.asarray(center, dtype=np.float64)
    half = np.array([R + a, R + a, a])
    nc = np.ceil(2 * half / h).astype(int)            # cells per axis
    origin = center - 0.5 * nc * h                    # grid symmetric about the centre
    ci, cj, ck = np.meshgrid(*(np.arange(m) for m in nc), indexing="ij")
    cx = origin[0] + (ci + 0.5) * h - center[0]
    cy = origin[1] + (cj + 0.5) * h - center[1]
    cz = origin[2] + (ck + 0.5) * h - center[2]
    inside = (np.sqrt(cx * cx + cy * cy) - R) ** 2 + cz * cz <= a * a
    cells = np.argwhere(inside)                       # grid order
    ny, nz = nc[1] + 1, nc[2] + 1

    def node(i, j, k):
        return (i * ny + j) * nz + k

    walks = []
    for perm, parity in _PERMS:
        w = [np.zeros(3, dtype=int)]
        c = np.zeros(3, dtype=int)
        for ax in perm:
            c = c.copy()
            c[ax] += 1
            w.append(c)
        if parity < 0:
            w[1], w[2] = w[2], w[1]
        walks.append(np.array(w))
    tets = np.empty((cells.shape[0] * 6, 4), dtype=np.int64)
    for s, w in enumerate(walks):
        for v in range(4):
            p = cells + w[v]
            tets[s::6, v] = node(p[:, 0], p[:, 1], p[:, 2])
    used, inv = np.unique(tets, return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int32)
    k = used % nz
    j = (used // nz) % ny
    i = used // (ny * nz)
    X0 = origin + np.stack([i, j, k], axis=1) * h
    return TorusMesh(X0=X0.astype(np.float64), tets=tets, h=float(h))
