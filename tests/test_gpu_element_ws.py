"""GPU parity of the warp-specialised tensor-core element kernel (the path the
BF16 form takes for large tet sets: at least 160 tets per SM, r a multiple of
4) against the FP64 oracle; the TF32 form on the same cases runs the tiled
tensor-core kernel and is checked alongside.

Cases on the 30x17x17 bar (44,544 tets): every tet at r = 64 (ragged: 278.4
units of 160 tets), a ragged cubature set of 40,003 tets with non-uniform weights at
r = 32, and r = 44 (eleven column quads, so the column-build slots do not
divide a chunk evenly), plus the cubature set in random order at r = 64 and
r = 32 (neighbouring tets of a chunk then share no vertices, so the staged J
rows are scattered gathers).  E, g, K at random z are compared norm-wise and
element-wise (tolerances of the tensor-core forms: the BF16 form against the
oracle of its BF16-rounded output weights, the TF32 form against the FP32
weights), and two implicit-Euler frames of the r = 64 case are solved in the
BF16 form against the oracle's trajectory (this also exercises the
line-search trial energies the kernel computes)."""
import dataclasses

import numpy as np
import pytest

from oracle.reduced import model_from_problem, ReducedSimulator
from workloads import build_problem, CONFIGS
from tests.gpu_util import random_qbar, round_bf16, assert_close

pytestmark = pytest.mark.gpu

TOL = {"bf16": dict(E=2e-4, g=2e-4, K=5e-3), "tf32": dict(E=5e-3, g=1e-2, K=1e-2)}
# element-wise floors (fraction of the largest entry): TF32 rounds J and the
# activations to 11 significant bits, and g = J^T g_full sums rows that cancel,
# so a small entry carries an error of the size of the large ones' rounding
FLOOR = {"bf16": 1e-2, "tf32": 5e-2}


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    pkg.load()
    return pkg


def bar(r, cubature, shuffle=False):
    c = dataclasses.replace(CONFIGS["block_twist_207k"], name=f"ws_bar_r{r}", dims=(30, 17, 17),
                            r=r, hidden=(128, 128), cubature=0, motion_frames=20)
    p = build_problem(c)
    if cubature:
        rng = np.random.default_rng(77)
        idx = np.sort(rng.choice(p.ne, cubature, replace=False)).astype(np.int32)
        w = rng.uniform(0.5, 4.0, cubature)
        if shuffle:  # the same tets and weights in random order
            perm = np.random.default_rng(78).permutation(cubature)
            idx, w = idx[perm], w[perm]
        p = dataclasses.replace(p, cub_idx=idx, cub_w=w)
    return p


def oracle_for(p, prec):
    if prec == "bf16":
        p = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    return model_from_problem(p)


def make_ctx(pkg, p, prec):
    ctx = pkg.context_from_problem(p, precision=prec)
    if len(p.cub_idx) and len(p.cub_idx) < p.ne:
        ctx.set_cubature(p.cub_idx, p.cub_w)
    return ctx


CASES = [(r, cub, False, prec) for r, cub in [(64, 0), (32, 40003), (44, 0)]
         for prec in ("bf16", "tf32")]
# the cubature set in random order: the tets of a chunk are scattered over the
# mesh, so their J rows share nothing
CASES += [(64, 40003, True, "bf16"), (32, 40003, True, "bf16")]


@pytest.mark.parametrize("r,cubature,shuffle,prec", CASES)
def test_ws_element_system_matches_oracle(pkg, r, cubature, shuffle, prec):
    import torch
    p = bar(r, cubature, shuffle)
    S = len(p.cub_idx) if len(p.cub_idx) else p.ne
    assert S >= 160 * torch.cuda.get_device_properties(0).multi_processor_count
    m = oracle_for(p, prec)
    ctx = make_ctx(pkg, p, prec)
    t = TOL[prec]
    rng = np.random.default_rng(5 + r)
    tg = p.targets(7)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    qbar = random_qbar(p, 3)
    ctx.set_dynamics(p.config.dt, qbar)
    m.set_dynamics(p.config.dt, qbar)
    try:
        for trial in range(2):
            z = rng.standard_normal(r) * 0.5
            E, g, K = ctx.eval(z)
            E0, g0, K0 = m.eval(z)
            assert abs(E - E0) <= t["E"] * max(1.0, abs(E0)), (E, E0)
            assert_close(g, g0, t["g"], floor=FLOOR[prec])
            assert_close(K, K0, t["K"], floor=FLOOR[prec])
    finally:
        ctx.close()


def test_ws_bf16_frames_follow_the_oracle(pkg):
    p = bar(64, 0)
    c = p.config
    pb = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    sim = ReducedSimulator(model_from_problem(pb), c.dt, eps=c.eps)
    ctx = make_ctx(pkg, p, "bf16")
    X0 = p.X0.ravel()
    try:
        for k in range(1, 3):
            sim.step(p.targets(k))
            ctx.set_constraints(None, p.targets(k))
            rc, st, _ = ctx.step(dt=c.dt)
            assert rc in (0, 4), (rc, st)
            u, uo = ctx.get_positions() - X0, sim.q - X0
            assert np.linalg.norm(u - uo) / np.linalg.norm(uo) < 1e-4
    finally:
        ctx.close()
