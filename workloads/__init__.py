"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This package generates *inputs only*: node grids and tet connectivity of the
bar meshes, decoder weights drawn by seed, cubature index draws, and the
prescribed boundary motion.  It holds none of the method's arithmetic (no
deformation gradient, no energy, no mass, no decoder evaluation); both the
CPU oracle and the CUDA path compute those on their own from these inputs.

The paper's meshes and datasets are not available, so procedurally generated
bars sized like the paper's examples (Table 1: n 1.6K-44K, E 1K-62K,
r 8-65) stand in for them.
"""
from .bar import BarMesh, make_bar, face_nodes
from .decoder_init import xavier_decoder
from .cubature import draw_cubature
from .motion import (rotate_face_targets, twist_compress_targets, twist_bend_targets,
                     twist_bend_loads)
from .configs import CONFIGS, Config, build_problem, Problem

__all__ = [
    "BarMesh", "make_bar", "face_nodes", "xavier_decoder", "draw_cubature",
    "rotate_face_targets", "twist_compress_targets", "twist_bend_targets",
    "twist_bend_loads", "CONFIGS", "Config",
    "build_problem", "Problem",
]
