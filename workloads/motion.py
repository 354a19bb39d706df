"""Prescribed boundary motion (inputs only): constraint targets per frame."""
import numpy as np


def _rot_x(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rotate_face_targets(X0, nodes, theta):
    """Rest positions of `nodes` rotated by theta about the x axis through the
    nodes' centroid (the face centre)."""
    P = X0[nodes]
    c = P.mean(axis=0)
    return (P - c) @ _rot_x(theta).T + c


def twist_compress_targets(X0, nodes, theta, shift):
    """Face nodes twisted by theta about x through the face centre, then moved
    by `shift` along x."""
    T = rotate_face_targets(X0, nodes, theta)
    T[:, 0] += shift
    return T


def _rot_y(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def twist_bend_targets(X0, fixed, moving, twist, bend):
    """Targets of the snapshot loads of the training bar: the `fixed` face at
    rest, the `moving` face rotated about its centre by `twist` about the long
    (x) axis and then by `bend` about the y axis (both faces, fixed first)."""
    P = X0[moving]
    c = P.mean(axis=0)
    R = _rot_x(twist) @ _rot_y(bend)
    return np.concatenate([X0[fixed], (P - c) @ R.T + c], axis=0)


def twist_bend_loads(count, seed, twist_max=3.0, bend_max=0.5, bins=32):
    """`count` loads (twist, bend) drawn uniformly from [0, twist_max] x
    [0, bend_max] by `seed`, in a serpentine order for load continuation: the
    twist range cut into `bins` slices taken in increasing twist, the bends
    within a slice alternately increasing and decreasing."""
    rng = np.random.default_rng(seed)
    L = np.stack([rng.uniform(0.0, twist_max, count), rng.uniform(0.0, bend_max, count)], 1)
    slot = np.minimum((L[:, 0] / twist_max * bins).astype(int), bins - 1)
    key = np.where(slot % 2 == 0, L[:, 1], -L[:, 1])
    return L[np.lexsort((key, slot))]
