"""GPU parity of the exact-form reduced Hessian (lsn_set_exact_hessian)
against the oracle's ReducedModel.eval_exact: the Gauss-Newton K plus the
decoder-curvature term sum_{k free} dE/dx_k d2x_k/dz2 (Eq. 2 differentiated
twice), projected as an r x r matrix.

Tolerances: FP64 form 1e-9 on K (rounding of the second-order tangents and
the Jacobi eigen-decomposition); FP32 form 1e-4 (as the Gauss-Newton K); the
tensor-core forms 2e-2 (TF32 products of the second-order tangents, BF16
Gram operands).  Trajectories: FP64 positions to 1e-8 and the same Newton
iteration counts as the oracle's exact-form solve."""
import dataclasses

import numpy as np
import pytest

from oracle.decoder import Decoder
from oracle.reduced import ReducedModel, ReducedSimulator, model_from_problem
from workloads import build_problem, make_bar, face_nodes, xavier_decoder, draw_cubature
from tests.gpu_util import assert_close, random_qbar, rel, round_bf16, UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

TOLK = {"fp64": 1e-9, "fp32": 1e-4, "tf32": 2e-2, "bf16": 2e-2}


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


def _k_unit(prec):
    return UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec]


@pytest.mark.parametrize("name", ["tiny_dyn", "tiny_quasistatic", "tiny_torus_drop"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
def test_exact_hessian_matches_oracle(pkg, name, prec):
    p = build_problem(name)
    ctx = pkg.context_from_problem(p, precision=prec)
    ctx.set_exact_hessian(True, 1e-10)
    if prec == "bf16":  # the BF16 form stores W_L rounded to BF16
        p = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    m = model_from_problem(p)
    rng = np.random.default_rng(21)
    tg = p.targets(2)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    if p.config.dt > 0:
        qbar = random_qbar(p, 9)
        ctx.set_dynamics(p.config.dt, qbar)
        m.set_dynamics(p.config.dt, qbar)
    r = m.r
    for trial in range(3):
        z = rng.standard_normal(r) * (0.8 if trial else 0.1)
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval_exact(z)
        _, _, K_gn = m.eval(z)
        assert_close(K, K_ref, TOLK[prec], u=_k_unit(prec))
        # the test is not vacuous: the curvature term moves K
        assert rel(K_gn, K_ref) > 10 * TOLK[prec] or rel(K_gn, K_ref) > 1e-3
    ctx.close()


def test_projection_with_odd_r_and_negative_eigenvalues(pkg):
    """r = 5 (the Jacobi ordering pads a dummy index) at a point where the
    curvature term makes the unprojected sum indefinite; quasi-static under
    gravity, FP64."""
    mesh = make_bar(8, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([5, 24, 24, n], 3)
    Ws[-1] = Ws[-1] * 40.0
    cn = face_nodes(mesh, 0)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0,
                     (0.0, 0.0, -9.8), cnodes=cn)
    ctx = pkg.Context()
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0.0, 0.0, -9.8))
    ctx.set_constraints(cn, mesh.X0[cn])
    ctx.set_decoder(Ws, bs, 1e-2, "fp64")
    ctx.set_exact_hessian(True, 1e-6)
    ctx.set_dynamics(0.0, None)
    rng = np.random.default_rng(4)
    seen_negative = False
    for _ in range(6):
        z = rng.standard_normal(5) * 1.5
        _, _, Kraw = m.eval_exact(z, project=False)
        Kp = m.eval(z)[2] + m.curvature_term(z)
        lam = np.linalg.eigvalsh(0.5 * (Kp + Kp.T))
        seen_negative |= lam.min() < -1e-6 * np.abs(lam).max()
        _, _, K = ctx.eval(z)
        _, _, K_ref = m.eval_exact(z, clamp=1e-6)
        assert_close(K, K_ref, 1e-9, u=UNIT_ROUNDOFF["fp64"])
        assert np.linalg.eigvalsh(K).min() > 0
    assert seen_negative
    ctx.close()


@pytest.mark.parametrize("name,frames", [("tiny_dyn", 6), ("tiny_quasistatic", 1)])
def test_exact_newton_trajectory_matches_oracle(pkg, name, frames):
    p = build_problem(name)
    m = model_from_problem(p)
    c = p.config
    sim = ReducedSimulator(m, c.dt, eps=c.eps, exact_hessian=True)
    ctx = pkg.context_from_problem(p, precision="fp64")
    ctx.set_exact_hessian(True, 1e-10)
    X0 = p.X0.ravel()
    for k in range(1, frames + 1):
        st_ref = sim.step(p.targets(k))
        ctx.set_constraints(None, p.targets(k))
        rc, st, _ = ctx.step(dt=c.dt)
        assert rc == pkg.LSN_OK and st_ref.status == 0, (k, rc, st_ref)
        assert st["newton_iters"] == st_ref.newton_iters, (k, st, st_ref)
        u, u_ref = ctx.get_positions() - X0, sim.q - X0
        assert rel(u, u_ref) < 1e-8, (k, rel(u, u_ref))
    ctx.close()
