"""Solve trajectory at the largest workload's full size against the FP64
oracle: block_twist_960k (101x41x41 nodes, 960,000 tets, n = 509,343,
r = 64, decoder 64-1024x3-509343, every tet evaluated), implicit Euler
dt = 1/60 (Eq. 2) from rest over its first frames, in every precision form
(FP64, FP32, TF32, BF16), in the launch configuration bench.py times.

The oracle is the FP64 reduced solve of the same decoder weights (the
seeded FP32 values), its element sums evaluated by worker processes.  Each
form's positions after every frame are compared with the oracle's by the
relative displacement error ||u_gpu - u_oracle|| / ||u_oracle||
(u = x - X0) and, element-wise, per vertex coordinate.  Tolerances: the
spec bands (1e-4 FP32, 1e-3 in the tensor-core forms) and 1e-7 in
FP64 (the same iterates in the same arithmetic up to summation order)."""
import os

import numpy as np
import pytest

from workloads import build_problem
from tests.gpu_util import elementwise_ratio

pytestmark = pytest.mark.gpu

FRAMES = 3
TOL = {"fp64": 1e-7, "fp32": 1e-4, "tf32": 1e-3, "bf16": 1e-3}


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


@pytest.fixture(scope="module")
def block():
    return build_problem("block_twist_960k")


@pytest.fixture(scope="module")
def oracle_frames(block):
    """The FP64 oracle's positions after frames 1..FRAMES from rest."""
    from oracle.pool import ElementPool
    from oracle.reduced import model_from_problem, ReducedSimulator
    p = block
    c = p.config
    m = model_from_problem(p, chunk=16384)
    pool = ElementPool(m, os.cpu_count())
    m.pool = pool
    try:
        sim = ReducedSimulator(m, c.dt, eps=c.eps, max_newton=c.max_newton, max_ls=c.max_ls,
                               c=c.armijo_c)
        qs, stats = [], []
        for k in range(1, FRAMES + 1):
            st = sim.step(p.targets(k))
            assert st.status == 0, st
            qs.append(sim.q.copy())
            stats.append(st)
    finally:
        pool.close()
    return qs, stats


@pytest.mark.parametrize("precision", ["bf16", "tf32", "fp32", "fp64"])
def test_block_960k_first_frames_match_the_oracle(pkg, block, oracle_frames, precision):
    p = block
    c = p.config
    qs, stats = oracle_frames
    X0 = p.X0.ravel()
    ctx = pkg.context_from_problem(p, precision=precision)
    try:
        for k in range(1, FRAMES + 1):
            ctx.set_constraints(None, p.targets(k))
            rc, st, _ = ctx.step(dt=c.dt)
            assert rc in (0, 4), (k, rc, st)       # converged (or the form's rounding floor)
            u = ctx.get_positions() - X0
            uo = qs[k - 1] - X0
            err = np.linalg.norm(u - uo) / np.linalg.norm(uo)
            ratio = elementwise_ratio(u, uo, TOL[precision], floor=1e-2)
            print(f"{precision} frame {k}: rel. displacement error {err:.3e}, "
                  f"element-wise ratio {ratio:.3f}, Newton {st['newton_iters']} "
                  f"(oracle {stats[k - 1].newton_iters}), exit {rc}")
            assert err < TOL[precision], (k, err)
            assert ratio <= 1.0, (k, ratio)
            if precision == "fp64":
                assert st["newton_iters"] == stats[k - 1].newton_iters
    finally:
        ctx.close()
