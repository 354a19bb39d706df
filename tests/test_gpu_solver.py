"""GPU parity of the reduced Newton path (CUDA through the C ABI) against the
FP64 CPU oracle, element by element on seeded inputs.

Tolerances: FP64 mode agrees to rounding (relative 1e-10 for x, J, E, g, K);
FP32 mode to the relative error that FP32 element arithmetic and FP32
accumulation over a tile leave (x, J: 1e-6; g, K, E: 1e-4); solves: relative
displacement error 1e-8 (FP64) and 1e-4 (FP32).
"""
import numpy as np
import pytest

from oracle.reduced import model_from_problem, ReducedSimulator
from workloads import build_problem
from tests.gpu_util import rel, random_qbar, assert_close

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(x=1e-12, J=1e-12, E=1e-10, g=1e-9, K=1e-9, u=1e-8),
       "fp32": dict(x=1e-6, J=2e-6, E=1e-4, g=2e-4, K=1e-4, u=1e-4)}


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


@pytest.mark.parametrize("name", ["tiny_dyn", "bar_quasistatic_1824", "bar_twist_dyn_14976"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_decoder_positions_and_jacobian(pkg, name, prec):
    p = build_problem(name)
    m = model_from_problem(p)
    ctx = pkg.context_from_problem(p, precision=prec)
    rng = np.random.default_rng(11)
    for frame in (0, 3):
        tg = p.targets(frame)
        ctx.set_constraints(None, tg)
        m.set_targets(tg)
        z = rng.standard_normal(p.config.r) * 0.7
        x, J = ctx.decode(z)
        x_ref, J_ref = m.positions_jac(z)
        u_ref = x_ref - p.X0.ravel()
        assert_close(x - p.X0.ravel(), u_ref, TOL[prec]["x"] * 10)
        assert_close(J, J_ref, TOL[prec]["J"] * 10)
        # constrained rows are exact targets with zero Jacobian rows
        cd = (3 * p.cnodes[:, None] + np.arange(3)).ravel()
        assert np.allclose(x[cd], tg.ravel(), atol=1e-6 if prec == "fp32" else 1e-14)
        assert np.all(J[cd] == 0.0)
    ctx.close()


@pytest.mark.parametrize("name", ["tiny_dyn", "tiny_quasistatic", "bar_quasistatic_1824",
                                  "bar_twist_dyn_14976"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_reduced_energy_gradient_hessian(pkg, name, prec):
    p = build_problem(name)
    m = model_from_problem(p)
    ctx = pkg.context_from_problem(p, precision=prec)
    rng = np.random.default_rng(5)
    tg = p.targets(2)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    dyn = p.config.dt > 0
    if dyn:
        qbar = random_qbar(p, 7)
        ctx.set_dynamics(p.config.dt, qbar)
        m.set_dynamics(p.config.dt, qbar)
    for trial in range(2):
        z = rng.standard_normal(p.config.r) * 0.5
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval(z)
        t = TOL[prec]
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref))
        assert_close(g, g_ref, t["g"])
        assert_close(K, K_ref, t["K"])
        assert np.allclose(K, K.T)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_quasistatic_solve_matches_oracle(pkg, prec):
    p = build_problem("bar_quasistatic_1824")
    m = model_from_problem(p)
    sim = ReducedSimulator(m, 0.0, eps=p.config.eps)
    st_ref = sim.step(p.targets(1))
    assert st_ref.status == 0
    ctx = pkg.context_from_problem(p, precision=prec)
    ctx.set_constraints(None, p.targets(1))
    rc, st, z = ctx.step(dt=0.0)
    x = ctx.get_positions()
    assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
    u_ref = sim.q - p.X0.ravel()
    assert_close(x - p.X0.ravel(), u_ref, TOL[prec]["u"])
    # the oracle's own gradient at the GPU's solution is small
    _, g_at, _ = m.eval(z)
    assert np.max(np.abs(g_at)) < (1.0 if prec == "fp64" else 100.0) * p.config.eps * 10
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dynamics_trajectory_matches_oracle(pkg, prec):
    p = build_problem("tiny_dyn")
    m = model_from_problem(p)
    sim = ReducedSimulator(m, p.config.dt, eps=p.config.eps)
    ctx = pkg.context_from_problem(p, precision=prec, tol=p.config.eps if prec == "fp64" else 1e-5)
    for k in range(1, p.config.steps + 1):
        st_ref = sim.step(p.targets(k))
        ctx.set_constraints(None, p.targets(k))
        rc, st, z = ctx.step(dt=p.config.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        x = ctx.get_positions()
        err = rel(x - p.X0.ravel(), sim.q - p.X0.ravel())
        assert err < TOL[prec]["u"] * (10 if prec == "fp32" else 1), (k, err)
    ctx.close()


def test_bar_twist_first_steps_match_oracle(pkg):
    p = build_problem("bar_twist_dyn_14976")
    m = model_from_problem(p)
    sim = ReducedSimulator(m, p.config.dt, eps=p.config.eps)
    ctx = pkg.context_from_problem(p, precision="fp32")
    for k in range(1, 6):
        sim.step(p.targets(k))
        ctx.set_constraints(None, p.targets(k))
        rc, st, z = ctx.step(dt=p.config.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        err = rel(ctx.get_positions() - p.X0.ravel(), sim.q - p.X0.ravel())
        assert err < 1e-4, (k, err)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_large_deformation_projection(pkg, prec):
    """Large z: strongly stretched / compressed / inverted tets, so the
    projection clamps many eigenvalues (analytic eigensystem on the GPU vs
    numeric eigh in the oracle)."""
    p = build_problem("tiny_dyn")
    m = model_from_problem(p)
    ctx = pkg.context_from_problem(p, precision=prec)
    rng = np.random.default_rng(21)
    tg = p.targets(p.config.motion_frames)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    m.set_dynamics(0.0, None)
    ctx.set_dynamics(0.0)
    nclamped = 0
    for trial in range(3):
        z = rng.standard_normal(p.config.r) * 40.0
        x, _ = m.positions_jac(z)
        from oracle import fem, snh
        F = fem.deformation_gradient(x.reshape(-1, 3), m.tets, m.DmInv)
        nclamped += int(np.sum(np.linalg.eigvalsh(snh.d2psi_dF2(F, m.mu, m.lam)) < 0))
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval(z)
        t = TOL[prec]
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref))
        assert_close(g, g_ref, t["g"])
        assert_close(K, K_ref, (t["K"] if prec == "fp64" else 5e-4))
    assert nclamped > 0
    ctx.close()


def test_graph_and_host_loop_execution_agree(pkg):
    """The CUDA-graph solve loop and the host-driven loop run the same kernels
    in the same order: identical iterates."""
    p = build_problem("tiny_dyn")
    out = {}
    for mode in ("graph", "host"):
        ctx = pkg.context_from_problem(p, precision="fp32", tol=1e-5)
        ctx.set_execution(mode)
        zs = []
        for k in range(1, 5):
            ctx.set_constraints(None, p.targets(k))
            rc, st, z = ctx.step(dt=p.config.dt)
            zs.append((rc, st["newton_iters"], st["ls_trials"], z.copy()))
        out[mode] = zs
        ctx.close()
    for a, b in zip(out["graph"], out["host"]):
        assert a[:3] == b[:3]
        assert np.array_equal(a[3], b[3])


def test_backtracking_trajectory_matches_oracle(pkg):
    """A heavy load (gravity x 1000, quasi-static) makes the line search
    backtrack; in FP64 the GPU solve follows the oracle's trajectory: same
    step lengths, same iteration count, same gradient norms."""
    from oracle.reduced import newton_solve
    p = build_problem("tiny_dyn")
    c = p.config
    grav = (0.0, 0.0, -9800.0)
    m = model_from_problem(p)
    m.gravity = np.asarray(grav)
    m.set_targets(p.targets(6))
    m.set_dynamics(0.0, None)
    trace = []
    z_ref, st_ref = newton_solve(m, np.zeros(c.r), 1e-7, trace=trace)
    alphas = [t[2] for t in trace[:-1]]
    assert min(alphas) < 1.0, "the case must exercise backtracking"
    ctx = pkg.context_from_problem(p, precision="fp64", tol=1e-7)
    ctx.set_material(c.youngs, c.poisson, c.density, grav)
    ctx.set_constraints(p.cnodes, p.targets(6))
    rc, st, z = ctx.step(z_in=np.zeros(c.r), dt=0.0)
    tr = ctx.get_trace()
    assert rc == st_ref.status
    # the first iterations follow the oracle step for step; the tail of a
    # backtracking solve depends on rounding in energy differences
    n = min(len(alphas), len(tr["alpha"]) - 1, 20)
    assert np.array_equal(tr["alpha"][:n], np.asarray(alphas[:n]))
    assert np.allclose(tr["grad_inf"][:n], [t[1] for t in trace[:n]], rtol=1e-6, atol=1e-12)
    # both ends are stationary to 1e-7: same point to the conditioning of K
    assert_close(z, z_ref, 1e-6)
    assert np.max(np.abs(m.eval(z)[1])) < 1e-6
    ctx.close()
