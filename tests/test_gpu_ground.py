"""GPU parity of the ground-contact penalty E_c = k/2 sum_v min(0, x_vz - h)^2
(lsn_set_ground; Sec. 5's collision examples) against the FP64 oracle: E, g,
K with part of the mesh below the plane, in every precision form, and
quasi-static solves (Newton and L-BFGS) that end in contact."""
import dataclasses

import numpy as np
import pytest

from oracle.lbfgs import lbfgs_solve
from oracle.reduced import model_from_problem, newton_solve
from workloads import build_problem
from tests.gpu_util import rel, random_qbar, round_bf16, assert_close, UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-10, g=1e-9, K=1e-9, u=1e-8), "fp32": dict(E=1e-4, g=2e-4, K=1e-4, u=1e-4),
       "bf16": dict(E=1e-4, g=2e-4, K=2e-3, u=1e-4)}
H, KG = 0.06, 2e4   # the plane cuts the bars' second node layer


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


def _model(p, prec):
    if prec == "bf16":
        p = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    m = model_from_problem(p)
    m.set_ground(H, KG)
    return m


@pytest.mark.parametrize("name", ["tiny_dyn", "bar_quasistatic_1824"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_energy_gradient_hessian_with_contact(pkg, name, prec):
    p = build_problem(name)
    m = _model(p, prec)
    ctx = pkg.context_from_problem(p, precision=prec)
    ctx.set_ground(H, KG)
    tg = p.targets(2)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    if p.config.dt > 0:
        qbar = random_qbar(p, 7)
        ctx.set_dynamics(p.config.dt, qbar)
        m.set_dynamics(p.config.dt, qbar)
    rng = np.random.default_rng(9)
    for _ in range(2):
        z = rng.standard_normal(p.config.r) * 0.5
        assert m._ground(m.positions(z))[0] > 0.0  # contact is active
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval(z)
        t = TOL[prec]
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref)), (E, E_ref)
        assert_close(g, g_ref, t["g"], u=UNIT_ROUNDOFF[prec])
        assert_close(K, K_ref, t["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
    ctx.close()


@pytest.mark.parametrize("optimizer", ["newton", "lbfgs"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_quasistatic_solve_into_contact(pkg, optimizer, prec):
    """The pinned bar under gravity with the plane 2 cm above its bottom face:
    the subspace cannot lift the bar clear, so the solution balances the
    penalty against the elastic and gravity forces (contact stays active)."""
    p = build_problem("bar_quasistatic_1824")
    c = p.config
    grav = c.gravity
    h = 0.02
    m = model_from_problem(p)
    m.gravity = np.asarray(grav)
    m.set_ground(h, KG)
    m.set_targets(p.targets(1))
    z0 = np.zeros(c.r)
    if optimizer == "newton":
        z_ref, st_ref = newton_solve(m, z0, 1e-6)
        iters = st_ref.newton_iters
    else:
        z_ref, st_ref = lbfgs_solve(m, z0, 1e-6)
        iters = st_ref.iters
    assert st_ref.status == 0
    x_ref = m.positions(z_ref)
    assert m._ground(x_ref)[0] > 0.0  # the solution is in contact
    ctx = pkg.context_from_problem(p, precision=prec, tol=1e-6, optimizer=optimizer)
    ctx.set_material(c.youngs, c.poisson, c.density, grav)
    ctx.set_ground(h, KG)
    ctx.set_constraints(None, p.targets(1))
    rc, st, z = ctx.step(z_in=z0, dt=0.0)
    assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
    if prec == "fp64":
        assert rc == 0 and st["newton_iters"] == iters
    assert_close(ctx.get_positions() - p.X0.ravel(), x_ref - p.X0.ravel(), TOL[prec]["u"])
    ctx.close()
