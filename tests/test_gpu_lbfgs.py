"""GPU parity of the L-BFGS solve (Sec. 5: the optimiser of the main results,
exits I-IV) through the C ABI against the FP64 CPU oracle.

The L-BFGS passes evaluate E and g with the gradient-only element kernel
(no per-element Hessian).  FP64: the GPU solve follows the oracle's
iterations (same exit, iteration and trial counts, same step lengths) and
lands on its point to 1e-8; FP32 and the tensor-core forms: relative
displacement error 1e-4 against the oracle's L-BFGS solution of the same
weights (BF16: the weights the form stores)."""
import dataclasses

import numpy as np
import pytest

from oracle.lbfgs import lbfgs_solve, SADDLE
from oracle.reduced import model_from_problem, ReducedSimulator
from workloads import build_problem
from tests.gpu_util import rel, random_qbar, round_bf16, assert_close
from tests.test_gpu_tensor_core import wide_problem

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-11, g=1e-9, u=1e-8), "fp32": dict(E=1e-5, g=2e-4, u=1e-4),
       "tf32": dict(E=5e-3, g=5e-2, u=2e-3), "bf16": dict(E=1e-5, g=2e-4, u=1e-4)}


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


def _oracle_problem(p, prec):
    """The weights the precision form computes with (BF16: W_L rounded)."""
    if prec == "bf16":
        return dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    return p


@pytest.mark.parametrize("name", ["tiny_dyn", "tiny_quasistatic", "bar_quasistatic_1824",
                                  "bar_twist_dyn_14976", "wide_r64"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_gradient_pass_matches_oracle(pkg, name, prec):
    """E and g of the gradient-only pass (ragged last tiles, r = 4 ... 64)."""
    p = wide_problem() if name == "wide_r64" else build_problem(name)
    m = model_from_problem(_oracle_problem(p, prec))
    ctx = pkg.context_from_problem(p, precision=prec, optimizer="lbfgs")
    tg = p.targets(2)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    if p.config.dt > 0:
        qbar = random_qbar(p, 7)
        ctx.set_dynamics(p.config.dt, qbar)
        m.set_dynamics(p.config.dt, qbar)
    rng = np.random.default_rng(5)
    for _ in range(2):
        z = rng.standard_normal(p.config.r) * 0.5
        E, g, K = ctx.eval(z, want_K=False)
        assert K is None
        E_ref, g_ref = m.energy_grad(z)
        t = TOL[prec]
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref)), (E, E_ref)
        assert_close(g, g_ref, t["g"])
        # the full pass of the same context still gives K (and the same g)
        E2, g2, K2 = ctx.eval(z)
        assert_close(g2, g, t["g"])
        assert np.allclose(K2, K2.T)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_quasistatic_solve_matches_oracle(pkg, prec):
    p = build_problem("bar_quasistatic_1824")
    m = model_from_problem(_oracle_problem(p, prec))
    m.set_targets(p.targets(1))
    trace = []
    z_ref, st_ref = lbfgs_solve(m, np.zeros(p.config.r), p.config.eps, trace=trace)
    assert st_ref.status == 0
    ctx = pkg.context_from_problem(p, precision=prec, optimizer="lbfgs")
    ctx.set_constraints(None, p.targets(1))
    rc, st, z = ctx.step(dt=0.0)
    assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
    x = ctx.get_positions()
    u_ref = m.positions(z_ref) - p.X0.ravel()
    assert_close(x - p.X0.ravel(), u_ref, TOL[prec]["u"])
    if prec == "fp64":
        assert (rc, st["newton_iters"], st["ls_trials"]) == (st_ref.status, st_ref.iters,
                                                             st_ref.ls_trials)
        tr = ctx.get_trace()
        n = st_ref.iters
        assert np.array_equal(tr["alpha"][:n], [t[2] for t in trace[:n]])
        assert np.allclose(tr["grad_inf"][:n + 1], [t[1] for t in trace[:n + 1]], rtol=1e-7)
        assert_close(z, z_ref, 1e-8)
    ctx.close()


@pytest.mark.parametrize("prec,history", [("fp64", 10), ("fp64", 2), ("fp64", 1),
                                          ("fp32", 10), ("bf16", 10)])
def test_dynamics_trajectory_matches_oracle(pkg, prec, history):
    """Implicit Euler steps; history 1 and 2 wrap the pair ring every
    iteration.  FP64: per step the same exit and the same ||g||_inf at every
    iteration until the energy decrease of a step reaches the rounding of E
    (there the Armijo test compares rounding noise and the two evaluation
    orders may take different trial steps: only the first 12 iterations and
    the iteration count within 15 % are compared)."""
    from oracle.lbfgs import lbfgs_solve
    p = build_problem("tiny_dyn")
    c = p.config
    m = model_from_problem(_oracle_problem(p, prec))
    ctx = pkg.context_from_problem(p, precision=prec, optimizer="lbfgs", history=history,
                                   tol=c.eps if prec == "fp64" else 1e-5)
    z = np.zeros(c.r)
    q = m.positions(z)
    v = np.zeros_like(q)
    grav = np.tile(m.gravity, m.nv)
    for k in range(1, c.steps + 1):
        # both sides start the step from the oracle's state (z, q, v)
        ctx.set_state(z, q, v)
        m.set_targets(p.targets(k))
        m.set_dynamics(c.dt, q + c.dt * v + c.dt ** 2 * grav)
        trace = []
        z, st_ref = lbfgs_solve(m, z, c.eps, history, trace=trace)
        qn = m.positions(z)
        v, q = (qn - q) / c.dt, qn
        ctx.set_constraints(None, p.targets(k))
        rc, st, _ = ctx.step(dt=c.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        if prec == "fp64":
            assert rc == st_ref.status, (k, st, st_ref)
            nn = min(12, st_ref.iters)
            tr = ctx.get_trace()
            assert np.allclose(tr["grad_inf"][:nn], [t[1] for t in trace[:nn]], rtol=1e-8,
                               atol=1e-12), k
            assert abs(st["newton_iters"] - st_ref.iters) <= max(1, 0.15 * st_ref.iters), \
                (k, st, st_ref)
        err = rel(ctx.get_positions() - p.X0.ravel(), q - p.X0.ravel())
        assert err < TOL[prec]["u"] * 10, (k, err)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
def test_bar_twist_first_steps_match_oracle(pkg, prec):
    """The C2 bar-twist workload (14,976 tets, 256 cubature tets, r = 16)."""
    p = build_problem("bar_twist_dyn_14976")
    m = model_from_problem(_oracle_problem(p, prec))
    sim = ReducedSimulator(m, p.config.dt, eps=p.config.eps, optimizer="lbfgs")
    ctx = pkg.context_from_problem(p, precision=prec, optimizer="lbfgs")
    for k in range(1, 6):
        sim.step(p.targets(k))
        ctx.set_constraints(None, p.targets(k))
        rc, st, z = ctx.step(dt=p.config.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        err = rel(ctx.get_positions() - p.X0.ravel(), sim.q - p.X0.ravel())
        assert err < TOL[prec]["u"], (k, err)
    ctx.close()


def _qs_model(p):
    m = model_from_problem(p)
    m.set_targets(p.targets(0))
    m.set_dynamics(0.0, None)
    return m


def test_saddle_exit_matches_oracle(pkg):
    """A quasi-static solve started far from rest (z0 = 3 N(0, 1)) meets a
    step with s^T y < 0 at its second iteration (exit II, ||g|| ~ 1)."""
    p = build_problem("tiny_quasistatic")
    z0 = np.random.default_rng(0).standard_normal(p.config.r) * 3.0
    z_ref, st_ref = lbfgs_solve(_qs_model(p), z0, 1e-7)
    assert st_ref.status == SADDLE and st_ref.grad_inf > 1e-2
    ctx = pkg.context_from_problem(p, precision="fp64", optimizer="lbfgs", tol=1e-7)
    ctx.set_constraints(None, p.targets(0))
    rc, st, z = ctx.step(z_in=z0, dt=0.0)
    assert rc == pkg.LSN_SADDLE
    assert (st["newton_iters"], st["ls_trials"]) == (st_ref.iters, st_ref.ls_trials)
    assert_close(z, z_ref, 1e-10)
    ctx.close()


@pytest.mark.parametrize("max_iters,max_ls", [(2, 128), (1024, 1)])
def test_iteration_and_line_search_caps_match_oracle(pkg, max_iters, max_ls):
    """Exit IV after two iterations; exit III when the single allowed trial
    (the unit step along -g) is rejected."""
    p = build_problem("tiny_quasistatic")
    r = p.config.r
    z_ref, st_ref = lbfgs_solve(_qs_model(p), np.zeros(r), 1e-9, max_iters=max_iters,
                                max_ls=max_ls)
    assert st_ref.status == (1 if max_iters == 2 else 2)
    ctx = pkg.context_from_problem(p, precision="fp64", optimizer="lbfgs", tol=1e-9)
    ctx.set_solver(1e-9, max_iters, max_ls, 1e-4)
    ctx.set_constraints(None, p.targets(0))
    rc, st, z = ctx.step(z_in=np.zeros(r), dt=0.0)
    assert (rc, st["newton_iters"], st["ls_trials"]) == (st_ref.status, st_ref.iters,
                                                         st_ref.ls_trials)
    if np.any(z_ref):
        assert_close(z, z_ref, 1e-10)
    else:
        assert np.array_equal(z, z_ref)
    ctx.close()
