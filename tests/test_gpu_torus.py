"""GPU parity of the free-body path (the torus workloads): 12 affine modes in
parallel with the network (lsn_set_affine_modes), ground contact, no
constraints, an initial spin, against the FP64 oracle; and a closed form
for the affine modes that does not use the oracle (free fall)."""
import dataclasses

import numpy as np
import pytest

from oracle.reduced import model_from_problem, ReducedSimulator
from workloads import build_problem, CONFIGS
from tests.gpu_util import rel, random_qbar, round_bf16, assert_close, UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(x=1e-12, J=1e-12, E=1e-10, g=1e-9, K=1e-9, u=1e-8),
       "fp32": dict(x=1e-6, J=2e-6, E=1e-4, g=2e-4, K=1e-4, u=1e-4),
       "bf16": dict(x=1e-6, J=2e-6, E=1e-4, g=2e-4, K=2e-3, u=1e-4)}


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


def _oracle(p, prec):
    if prec == "bf16":
        p = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    return model_from_problem(p)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_positions_jacobian_with_affine_modes(pkg, prec):
    p = build_problem("tiny_torus_drop")
    m = _oracle(p, prec)
    ctx = pkg.context_from_problem(p, precision=prec)
    r = p.config.r + 12
    assert ctx.r == r and m.r == r
    rng = np.random.default_rng(4)
    z = rng.standard_normal(r) * 0.3
    x, J = ctx.decode(z)
    x_ref, J_ref = m.positions_jac(z)
    t = TOL[prec]
    assert_close(x - p.X0.ravel(), x_ref - p.X0.ravel(), 10 * t["x"], u=UNIT_ROUNDOFF[prec])
    assert_close(J, J_ref, 10 * t["J"], u=UNIT_ROUNDOFF[prec])
    # the affine columns are the constant map itself (times the output scale)
    s = p.config.out_scale
    dX = p.X0 - p.affine_center
    assert np.allclose(J[2::3, r - 12 + 6:r - 12 + 9], s * dX, rtol=0, atol=1e-8)
    assert np.allclose(J[0::3, r - 1], 0.0) and np.allclose(J[2::3, r - 1], s)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_energy_gradient_hessian_with_affine_modes_and_contact(pkg, prec):
    p = build_problem("tiny_torus_drop")
    c = p.config
    m = _oracle(p, prec)
    ctx = pkg.context_from_problem(p, precision=prec)
    qbar = random_qbar(p, 7)
    ctx.set_dynamics(c.dt, qbar)
    m.set_dynamics(c.dt, qbar)
    rng = np.random.default_rng(8)
    r = c.r + 12
    for _ in range(2):
        z = rng.standard_normal(r) * 0.2
        z[r - 1] = -2.0          # translate down (2 cm) into the ground
        assert m._ground(m.positions(z))[0] > 0.0
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval(z)
        t = TOL[prec]
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref)), (E, E_ref)
        assert_close(g, g_ref, t["g"], u=UNIT_ROUNDOFF[prec])
        assert_close(K, K_ref, t["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_drop_trajectory_matches_oracle(pkg, prec):
    """Spinning torus dropped onto the ground: 8 implicit-Euler steps with
    contact from the first step on.  Each step starts both sides from the
    oracle's state.  The quadratic penalty's curvature jumps where a vertex
    crosses the plane, so Newton iterates near such a kink can differ with
    rounding (the FP64 oracle itself takes different paths on different
    machines): the GPU's end point must pass the oracle's own gradient test
    (||g||_inf below 2 eps in FP64, 100 eps in the FP32 forms) and lie within
    1e-4 of the oracle's end point wherever the oracle converged."""
    from oracle.reduced import newton_solve
    p = build_problem("tiny_torus_drop")
    c = p.config
    m = _oracle(p, prec)
    ctx = pkg.context_from_problem(p, precision=prec)
    ctx.set_solver(c.eps, 100, c.max_ls, c.armijo_c)
    z = np.zeros(c.r + 12)
    q = m.positions(z)
    v = p.v0.copy()
    grav = np.tile(c.gravity, p.nv)
    contact = 0
    for k in range(1, c.steps + 1):
        ctx.set_state(z, q, v)
        qbar = q + c.dt * v + c.dt ** 2 * grav
        m.set_dynamics(c.dt, qbar)
        z_ref, st_ref = newton_solve(m, z, c.eps, max_newton=100)
        rc, st, z_gpu = ctx.step(dt=c.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        gi = np.max(np.abs(m.eval(z_gpu)[1]))
        assert gi < (2.0 if prec == "fp64" else 100.0) * c.eps, (k, gi)
        x_ref = m.positions(z_ref)
        if st_ref.status == 0:
            err = rel(ctx.get_positions() - p.X0.ravel(), x_ref - p.X0.ravel())
            assert err < 1e-4, (k, err)
        contact += m._ground(x_ref)[0] > 0.0
        z, v, q = z_ref, (x_ref - q) / c.dt, x_ref
    assert contact >= c.steps - 1
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_fall_closed_form(pkg, prec):
    """Network output zero (W_L = 0), affine modes, no ground: one implicit
    Euler step from rest with uniform velocity v0 lands on
    X0 + dt v0 + dt^2 g exactly (projectile motion)."""
    c = dataclasses.replace(CONFIGS["tiny_torus_drop"], ground_k=0.0)
    p = build_problem(c)
    p = dataclasses.replace(p, Ws=[*p.Ws[:-1], np.zeros_like(p.Ws[-1])],
                            v0=np.tile([0.3, -0.2, 0.5], p.nv))
    ctx = pkg.context_from_problem(p, precision=prec, tol=1e-9)
    rc, st, z = ctx.step(dt=c.dt)
    assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
    g = np.tile(c.gravity, p.nv)
    x = ctx.get_positions()
    expect = p.X0.ravel() + c.dt * p.v0 + c.dt ** 2 * g
    assert np.max(np.abs(x - expect)) < (1e-11 if prec == "fp64" else 2e-6)
    ctx.close()
