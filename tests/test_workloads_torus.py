"""CPU checks of the voxel torus mesher (inputs of the free-body workload):
orientation, conformity, a closed single-body boundary, and the volume
against the analytic solid-torus volume 2 pi^2 R a^2."""
import numpy as np
import pytest

from workloads import build_problem
from workloads.torus import make_torus


@pytest.mark.parametrize("h,vol_tol", [(0.075, 0.1), (0.04, 0.05)])
def test_voxel_torus_mesh(h, vol_tol):
    R, a = 0.5, 0.15
    m = make_torus(R, a, h, (0.0, 0.0, 0.4))
    X, T = m.X0, m.tets
    D = np.stack([X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]], X[T[:, 3]] - X[T[:, 0]]],
                 axis=2)
    det = np.linalg.det(D)
    assert np.all(det > 0)                                   # positive orientation
    assert np.allclose(det, h ** 3, rtol=1e-9)               # six equal tets per cell
    # conforming: every face is shared by at most two tets; boundary faces
    # (used once) form a closed surface: each of their edges is used twice
    faces = np.sort(np.concatenate([T[:, [0, 1, 2]], T[:, [0, 1, 3]], T[:, [0, 2, 3]],
                                    T[:, [1, 2, 3]]]), axis=1)
    uf, cnt = np.unique(faces, axis=0, return_counts=True)
    assert cnt.max() <= 2
    bnd = uf[cnt == 1]
    edges = np.sort(np.concatenate([bnd[:, [0, 1]], bnd[:, [0, 2]], bnd[:, [1, 2]]]), axis=1)
    _, ecnt = np.unique(edges, axis=0, return_counts=True)
    assert np.all(ecnt % 2 == 0)
    # every vertex is used, and the volume is the solid torus's up to the voxels
    assert np.unique(T).size == X.shape[0]
    vol = det.sum() / 6.0
    assert vol == pytest.approx(2 * np.pi ** 2 * R * a * a, rel=vol_tol)
    # one connected body (union-find over the tets' vertices)
    parent = np.arange(X.shape[0])

    def find(i):
        while parent[i] != i:
            parent[i] = parent[parent[i]]
            i = parent[i]
        return i
    for t in T:
        r0 = find(t[0])
        for v in t[1:]:
            rv = find(v)
            if rv != r0:
                parent[rv] = r0
    assert len({find(i) for i in range(X.shape[0])}) == 1


def test_torus_workload_inputs():
    """The free-body workload: no constraints, the affine centre at the rest
    centroid, the initial velocity a rigid rotation plus the drop speed."""
    p = build_problem("tiny_torus_drop")
    assert p.cnodes.size == 0 and p.targets(5).shape == (0, 3)
    assert np.allclose(p.affine_center, p.X0.mean(0))
    v = p.v0.reshape(-1, 3) - np.array([0.0, 0.0, -p.config.drop_speed])
    # v = omega x (X - c): zero divergence, equal to a skew matrix times X - c
    Xc = p.X0 - p.affine_center
    Wm, *_ = np.linalg.lstsq(Xc, v, rcond=None)
    assert np.allclose(Wm, -Wm.T, atol=1e-10)
    assert np.allclose(Xc @ Wm, v, atol=1e-10)
