"""The synthetic workloads, by name, with their sizes and seeds.

Seeds: 0 decoder weights, 1 cubature draw, 2 snapshot load parameters,
3 training batch order, 100+ finite-difference parameter choice.

* bar_quasistatic_1824 - cantilever bar 20x5x5 nodes (h = 0.05 m, 1,824 tets,
  n = 1,500), x = 0 face pinned, gravity -9.8 z, quasi-static solve from
  z = 0 to ||g||_inf < 1e-6; r = 8, decoder 8-128-128-1500, all tets w = 1.
* bar_twist_dyn_14976 - bar 40x9x9 nodes (14,976 tets, n = 9,720), x = 0 face
  rotated 2 rad about the long axis over 60 frames, implicit Euler
  dt = 1/60, 200 steps; r = 16, decoder 16-256-256-256-9720; 256 cubature
  tets drawn uniformly (weights 14976/256).
* bar_train_44544 - bar 30x17x17 nodes (44,544 tets, n = 26,010), decoder
  training workload: r = 16, 16-256x3-26010, 512 cubature tets, batch 64.
* block_twist_960k - block 101x41x41 nodes (960,000 tets, n = 509,343),
  x = 0 face fixed, x = L face twisted 2 rad and pushed in by 0.2 L over 150
  frames, implicit Euler dt = 1/60; r = 64, decoder 64-1024x3-509343, all tets.
* block_twist_207k - the same block motion on 61x25x25 nodes (207,360 tets,
  n = 114,375) with the same decoder widths: a mid-size case for profiling.
* torus_drop_200k - free voxel torus (R = 0.5 m, a = 0.15 m, h = 0.0188 m:
  200,928 tets, n = 119,268), centre 0.4 m above a ground plane z = 0
  (penalty k = 1e6), spinning at omega with axis uniform on the sphere and
  |omega| ~ U[0, 5] rad/s (seed 2), v0 = omega x (X - c); E = 5e5 Pa,
  nu = 0.4; implicit Euler dt = 0.01, 500 steps; r = 32 network coordinates
  + 12 affine modes, decoder 32-512x3-119268, 1,024 cubature tets.
* tiny_* - small cases that the oracle finishes in well under a second
  (tiny_torus_drop: the torus at h = 0.075 m, 3,408 tets, dropped at 1 m/s
  from 1 cm above the ground).

Material for the bars: Young's modulus 1e5 Pa, Poisson ratio 0.45, density
1000 kg/m^3, gravity (0, 0, -9.8) m/s^2.
"""
from dataclasses import dataclass, field
import numpy as np

from .bar import make_bar, face_nodes
from .torus import make_torus
from .decoder_init import xavier_decoder
from .cubature import draw_cubature
from .motion import rotate_face_targets, twist_compress_targets


@dataclass
class Config:
    name: str
    dims: tuple                 # (nx, ny, nz) nodes, x long
    h: float
    r: int
    hidden: tuple               # hidden widths of the decoder
    cubature: int               # 0: every tet with weight 1
    dt: float                   # 0: quasi-static
    steps: int
    eps: float                  # ||g||_inf tolerance
    motion: str                 # 'pin' | 'rotate' | 'twist_compress'
    youngs: float = 1e5
    poisson: float = 0.45
    density: float = 1000.0
    gravity: tuple = (0.0, 0.0, -9.8)
    out_scale: float = 1e-2
    motion_frames: int = 60
    motion_angle: float = 2.0
    motion_shift: float = 0.0   # fraction of the bar length
    max_newton: int = 1024
    max_ls: int = 128
    mesh: str = "bar"           # 'bar' | 'torus' (then `motion` is 'free')
    torus: tuple = (0.5, 0.15)  # major, minor radius
    center_height: float = 0.4  # torus centre above the ground plane
    ground_h: float = 0.0       # ground plane z = ground_h ...
    ground_k: float = 0.0       # ... with penalty stiffness (0: no ground)
    affine: bool = False        # 12 affine modes in parallel with the network
    spin_max: float = 0.0       # |omega| ~ U[0, spin_max] (seed 2)
    drop_speed: float = 0.0     # initial downward speed
    armijo_c: float = 1e-4
    weight_seed: int = 0
    cubature_seed: int = 1


CONFIGS = {
    "bar_quasistatic_1824": Config(
        "bar_quasistatic_1824", (20, 5, 5), 0.05, 8, (128, 128), 0, 0.0, 1,
        1e-6, "pin"),
    "bar_twist_dyn_14976": Config(
        "bar_twist_dyn_14976", (40, 9, 9), 0.05, 16, (256, 256, 256), 256,
        1.0 / 60.0, 200, 1e-5, "rotate", motion_frames=60, motion_angle=2.0),
    "bar_train_44544": Config(
        "bar_train_44544", (30, 17, 17), 0.05, 16, (256, 256, 256), 512, 0.0,
        1, 1e-5, "pin"),
    "block_twist_960k": Config(
        "block_twist_960k", (101, 41, 41), 0.05, 64, (1024, 1024, 1024), 0,
        1.0 / 60.0, 300, 1e-5, "twist_compress", motion_frames=150,
        motion_angle=2.0, motion_shift=-0.2),
    # the same block at a fifth of the size (profiling and mid-size parity)
    "block_twist_207k": Config(
        "block_twist_207k", (61, 25, 25), 0.05, 64, (1024, 1024, 1024), 0,
        1.0 / 60.0, 300, 1e-5, "twist_compress", motion_frames=150,
        motion_angle=2.0, motion_shift=-0.2),
    "torus_drop_200k": Config(
        "torus_drop_200k", (0, 0, 0), 0.0188, 32, (512, 512, 512), 1024, 0.01, 500,
        1e-5, "free", youngs=5e5, poisson=0.4, mesh="torus", ground_k=1e6, affine=True,
        spin_max=5.0, motion_frames=0),
    # small cases for parity tests
    "tiny_torus_drop": Config(
        "tiny_torus_drop", (0, 0, 0), 0.075, 6, (24, 24), 256, 0.01, 8, 1e-5, "free",
        youngs=5e5, poisson=0.4, mesh="torus", center_height=0.16, ground_k=1e4,
        affine=True, spin_max=3.0, drop_speed=1.0, motion_frames=0),
    "tiny_quasistatic": Config(
        "tiny_quasistatic", (8, 3, 3), 0.05, 4, (16, 16), 0, 0.0, 1, 1e-8,
        "pin"),
    "tiny_dyn": Config(
        "tiny_dyn", (10, 4, 4), 0.05, 6, (24, 24, 24), 60, 1.0 / 60.0, 8,
        1e-7, "rotate", motion_frames=6, motion_angle=1.0),
    "small_dyn_full": Config(
        "small_dyn_full", (16, 5, 5), 0.05, 12, (64, 64, 64), 0, 1.0 / 60.0,
        6, 1e-6, "twist_compress", motion_frames=6, motion_angle=1.0,
        motion_shift=-0.1),
}


@dataclass
class Problem:
    config: Config
    X0: np.ndarray          # (nv, 3) float64
    tets: np.ndarray        # (ne, 4) int32
    Ws: list                # float32 (out, in)
    bs: list                # float32 (out,)
    cub_idx: np.ndarray     # (S,) int32
    cub_w: np.ndarray       # (S,) float64
    cnodes: np.ndarray      # (nc,) int32 constrained nodes
    widths: list = field(default_factory=list)
    affine_center: np.ndarray = None   # (3,) centre of the affine modes, or None
    v0: np.ndarray = None              # (n,) initial velocity, or None (rest)

    @property
    def nv(self):
        return self.X0.shape[0]

    @property
    def n(self):
        return 3 * self.X0.shape[0]

    @property
    def ne(self):
        return self.tets.shape[0]

    def targets(self, frame):
        """Constraint targets (nc, 3) for `frame` (frame 0 = rest)."""
        c = self.config
        t = min(frame / c.motion_frames, 1.0) if c.motion_frames else 0.0
        if c.motion == "free":
            return np.zeros((0, 3))
        if c.motion == "pin":
            return self.X0[self.cnodes].copy()
        if c.motion == "rotate":
            return rotate_face_targets(self.X0, self.cnodes, c.motion_angle * t)
        # twist_compress: first half of cnodes is the fixed x = 0 face
        nf = self.cnodes.shape[0] // 2
        fixed = self.X0[self.cnodes[:nf]].copy()
        L = (c.dims[0] - 1) * c.h
        moving = twist_compress_targets(self.X0, self.cnodes[nf:],
                                        c.motion_angle * t,
                                        c.motion_shift * L * t)
        return np.concatenate([fixed, moving], axis=0)


def build_problem(name_or_config, with_weights=True):
    c = CONFIGS[name_or_config] if isinstance(name_or_config, str) else name_or_config
    if c.mesh == "torus":
        return _build_torus(c, with_weights)
    mesh = make_bar(*c.dims, c.h)
    n = 3 * mesh.nv
    widths = [c.r, *c.hidden, n]
    Ws, bs = xavier_decoder(widths, c.weight_seed) if with_weights else ([], [])
    cub_idx, cub_w = draw_cubature(mesh.ne, c.cubature, c.cubature_seed)
    if c.motion == "twist_compress":
        cnodes = np.concatenate([face_nodes(mesh, 0), face_nodes(mesh, 1)])
    else:
        cnodes = face_nodes(mesh, 0)
    return Problem(c, mesh.X0, mesh.tets, Ws, bs, cub_idx, cub_w, cnodes, widths)


def _build_torus(c, with_weights):
    """Free torus above the ground: no constraints, affine centre at the rest
    centroid, initial spin omega x (X - c) (axis uniform on the sphere and
    |omega| ~ U[0, spin_max], seed 2) plus a downward speed."""
    R, a = c.torus
    mesh = make_torus(R, a, c.h, (0.0, 0.0, c.ground_h + c.center_height))
    n = 3 * mesh.nv
    widths = [c.r, *c.hidden, n]
    Ws, bs = xavier_decoder(widths, c.weight_seed) if with_weights else ([], [])
    cub_idx, cub_w = draw_cubature(mesh.ne, c.cubature, c.cubature_seed)
    center = mesh.X0.mean(0)
    rng = np.random.default_rng(2)
    axis = rng.standard_normal(3)
    omega = axis / np.linalg.norm(axis) * rng.uniform(0.0, c.spin_max)
    v0 = np.cross(omega, mesh.X0 - center) + np.array([0.0, 0.0, -c.drop_speed])
    return Problem(c, mesh.X0, mesh.tets, Ws, bs, cub_idx, cub_w,
                   np.zeros(0, dtype=np.int32), widths,
                   affine_center=center if c.affine else None, v0=v0.ravel())
