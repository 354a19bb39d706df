"""Structured tetrahedral bar meshes (inputs only).

A node grid of nx x ny x nz nodes with spacing h; the long axis is x.  Node
(i, j, k) sits at (i h, j h, k h) and has index (i*ny + j)*nz + k.  Every hex
cell is split into the six tetrahedra that share the cell's main diagonal
(the Kuhn/Freudenthal split): for each ordering (a, b, c) of the three axes,
the tet walks 000 -> +e_a -> +e_a+e_b -> 111.  Using the same split in every
cell makes the mesh conforming.  Vertex order is chosen so that the rest
edge matrix [X1-X0, X2-X0, X3-X0] has positive determinant: the determinant
of the walk is the sign of the axis permutation, so odd permutations swap
their second and third vertices.
"""
from dataclasses import dataclass
import itertools
import numpy as np

# the six axis orderings with their permutation parity
_PERMS = [(p, 1 if _even else -1) for p, _even in
          [((0, 1, 2), True), ((1, 2, 0), True), ((2, 0, 1), True),
           ((1, 0, 2), False), ((0, 2, 1), False), ((2, 1, 0), False)]]


@dataclass
class BarMesh:
    X0: np.ndarray        # (nv, 3) float64 rest positions
    tets: np.ndarray      # (ne, 4) int32 vertex indices
    dims: tuple           # (nx, ny, nz) nodes
    h: float              # node spacing

    @property
    def nv(self):
        return self.X0.shape[0]

    @property
    def ne(self):
        return self.tets.shape[0]


def _node(i, j, k, ny, nz):
    return (i * ny + j) * nz + k


def make_bar(nx, ny, nz, h):
    """Bar of nx*ny*nz nodes (x is the long axis), 6 tets per hex cell."""
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    X0 = np.stack([ii.ravel() * h, jj.ravel() * h, kk.ravel() * h],
                  axis=1).astype(np.float64)
    tets = []
    for i, j, k in itertools.product(range(nx - 1), range(ny - 1), range(nz - 1)):
        for perm, parity in _PERMS:
            c = [0, 0, 0]
            walk = [_node(i, j, k, ny, nz)]
            for ax in perm:
                c[ax] += 1
                walk.append(_node(i + c[0], j + c[1], k + c[2], ny, nz))
            if parity < 0:
                walk[1], walk[2] = walk[2], walk[1]
            tets.append(walk)
    return BarMesh(X0=X0, tets=np.asarray(tets, dtype=np.int32),
                   dims=(nx, ny, nz), h=float(h))


def face_nodes(mesh, side):
    """Indices of the nodes on the x = 0 face (side=0) or x = L face (side=1)."""
    nx, ny, nz = mesh.dims
    i = 0 if side == 0 else nx - 1
    jj, kk = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
    return ((i * ny + jj) * nz + kk).ravel().astype(np.int32)
