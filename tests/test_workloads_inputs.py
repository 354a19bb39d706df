"""CPU checks of the seeded synthetic inputs: the mesh and decoder sizes of
each named workload, reproducibility (every array is a function of the config and
its seeds), and the boundary motions (rigid face rotations and the
twist-and-compress end face)."""
import numpy as np
import pytest

from workloads import build_problem, CONFIGS

SIZES = {  # name: (n, tets, decoder widths without n, cubature size or 0 = all)
    "bar_quasistatic_1824": (1500, 1824, [8, 128, 128], 0),
    "bar_twist_dyn_14976": (9720, 14976, [16, 256, 256, 256], 256),
    "bar_train_44544": (26010, 44544, [16, 256, 256, 256], 512),
    "block_twist_207k": (114375, 207360, [64, 1024, 1024, 1024], 0),
    "block_twist_960k": (509343, 960000, [64, 1024, 1024, 1024], 0),
    "torus_drop_200k": (119268, 200928, [32, 512, 512, 512], 1024),
    "tiny_torus_drop": (3012, 3408, [6, 24, 24], 256),
}


@pytest.mark.parametrize("name", sorted(SIZES))
def test_workload_sizes(name):
    n, ne, widths, S = SIZES[name]
    p = build_problem(name, with_weights=False)
    assert (p.n, p.ne) == (n, ne)
    assert p.widths == [*widths, n]
    if S:
        assert len(p.cub_idx) == S and np.unique(p.cub_idx).size == S
        assert np.all((p.cub_idx >= 0) & (p.cub_idx < ne))
        assert np.allclose(p.cub_w, ne / S)          # uniform draw, weights E / S
    else:
        assert len(p.cub_idx) == 0 or len(p.cub_idx) == ne


@pytest.mark.parametrize("name", ["tiny_dyn", "tiny_torus_drop", "small_dyn_full",
                                  "bar_twist_dyn_14976"])
def test_inputs_are_reproducible(name):
    a, b = build_problem(name), build_problem(name)
    for f in ("X0", "tets", "cub_idx", "cub_w", "cnodes"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    for wa, wb in zip(a.Ws + a.bs, b.Ws + b.bs):
        assert np.array_equal(wa, wb)
    assert (a.v0 is None and b.v0 is None) or np.array_equal(a.v0, b.v0)
    for k in (0, 1, 7, 1000):
        assert np.array_equal(a.targets(k), b.targets(k))


def test_rotating_face_is_rigid_and_holds_after_the_motion():
    p = build_problem("bar_twist_dyn_14976", with_weights=False)
    c = p.config
    X = p.X0[p.cnodes]
    D0 = np.linalg.norm(X[:, None] - X[None], axis=2)
    for k in (1, 30, c.motion_frames, c.motion_frames + 40):
        T = p.targets(k)
        assert np.allclose(np.linalg.norm(T[:, None] - T[None], axis=2), D0, atol=1e-12)
        assert np.allclose(T[:, 0], X[:, 0])         # rotation about the long (x) axis
    # the angle grows to motion_angle and then holds
    assert np.array_equal(p.targets(c.motion_frames), p.targets(c.motion_frames + 40))
    assert np.allclose(p.targets(0), X, rtol=0, atol=1e-15)
    ctr = X.mean(0)
    T = p.targets(c.motion_frames)
    u, v = X[:, 1:] - ctr[1:], T[:, 1:] - ctr[1:]
    ang = np.arctan2(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0], (u * v).sum(1))
    big = np.linalg.norm(u, axis=1) > 1e-9
    assert np.allclose(ang[big], c.motion_angle)


def test_twist_and_compress_end_face():
    c = CONFIGS["small_dyn_full"]
    p = build_problem(c)
    nf = len(p.cnodes) // 2
    L = (c.dims[0] - 1) * c.h
    T = p.targets(c.motion_frames)
    assert np.array_equal(T[:nf], p.X0[p.cnodes[:nf]])          # x = 0 face fixed
    X1 = p.X0[p.cnodes[nf:]]
    assert np.allclose(T[nf:, 0], X1[:, 0] + c.motion_shift * L)  # pushed along x
    D0 = np.linalg.norm(X1[:, None, 1:] - X1[None, :, 1:], axis=2)
    D1 = np.linalg.norm(T[nf:, None, 1:] - T[None, nf:, 1:], axis=2)
    assert np.allclose(D0, D1, atol=1e-12)                       # twisted rigidly in y-z


def test_twist_bend_snapshot_loads():
    """The snapshot loads of the training bar: reproducible by seed, inside
    [0, 3] x [0, 0.5] rad, serpentine order (twist slices increasing, bends
    alternating), and targets that hold the x = 0 face at rest and move the
    x = L face rigidly by the two rotations about its centre."""
    from workloads import twist_bend_loads, twist_bend_targets, make_bar, face_nodes
    L = twist_bend_loads(1024, 2)
    assert L.shape == (1024, 2)
    assert np.array_equal(L, twist_bend_loads(1024, 2))
    assert not np.array_equal(L, twist_bend_loads(1024, 3))
    assert L[:, 0].min() >= 0 and L[:, 0].max() <= 3.0
    assert L[:, 1].min() >= 0 and L[:, 1].max() <= 0.5
    slot = np.minimum((L[:, 0] / 3.0 * 32).astype(int), 31)
    assert np.all(np.diff(slot) >= 0)
    for s in range(32):
        b = L[slot == s, 1]
        assert np.all(np.diff(b) >= 0) if s % 2 == 0 else np.all(np.diff(b) <= 0)
    mesh = make_bar(6, 4, 4, 0.05)
    f0, f1 = face_nodes(mesh, 0), face_nodes(mesh, 1)
    T = twist_bend_targets(mesh.X0, f0, f1, 1.1, 0.3)
    assert np.array_equal(T[:len(f0)], mesh.X0[f0])
    P, Q = mesh.X0[f1], T[len(f0):]
    assert np.allclose(Q.mean(0), P.mean(0))
    dP = np.linalg.norm(P[:, None] - P[None], axis=-1)
    dQ = np.linalg.norm(Q[:, None] - Q[None], axis=-1)
    assert np.allclose(dP, dQ)
    # the face normal (x) turns by the bend angle alone (a twist about x keeps it)
    n = np.linalg.svd(Q - Q.mean(0))[2][-1]
    assert np.isclose(abs(n[0]), np.cos(0.3))
    assert np.allclose(twist_bend_targets(mesh.X0, f0, f1, 0.0, 0.0)[len(f0):], P)
