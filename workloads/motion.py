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
