"""Pins of the oracle's full-space projective Newton solve (Eq. 1)."""
import numpy as np

from oracle.fullspace import FullModel, newton_solve
from oracle.reduced import CONVERGED, model_from_problem, ReducedSimulator
from workloads import make_bar, face_nodes, build_problem


def test_rest_without_load_is_solution():
    mesh = make_bar(5, 3, 3, 0.05)
    cn = face_nodes(mesh, 0)
    fm = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, (0, 0, 0), cn)
    q, st = newton_solve(fm, mesh.X0.ravel(), mesh.X0[cn], 1e-10)
    assert st.status == CONVERGED and st.newton_iters == 0
    assert np.array_equal(q, mesh.X0.ravel())


def test_gravity_sag_converges_and_plain_newton_is_quadratic():
    mesh = make_bar(8, 3, 3, 0.05)
    cn = face_nodes(mesh, 0)
    fm = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, (0, 0, -9.8), cn)
    # projective Newton converges linearly here; 1e-7 is above the level at
    # which float64 energy differences stop resolving the Armijo decrease
    q, st = newton_solve(fm, mesh.X0.ravel(), mesh.X0[cn], 1e-7)
    assert st.status == CONVERGED
    assert np.max(np.abs(fm.gradient(q)[fm.free])) < 1e-7
    # plain Newton (exact Hessian) from a nearby start: |g_{k+1}| <= C |g_k|^2
    fx = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, (0, 0, -9.8), cn,
                   project=False)
    q0 = q + 2e-5 * np.random.default_rng(0).standard_normal(q.shape)
    _, st2 = newton_solve(fx, q0, mesh.X0[cn], 1e-11)
    g = [t[1] for t in st2.trace]
    assert st2.status == CONVERGED and len(g) <= 5
    for a, b in zip(g[:-1], g[1:]):
        if a < 1.0:
            assert b <= 10.0 * a ** 2 + 1e-11


def test_full_space_energy_bounds_subspace_energy():
    """Every subspace configuration is a full-space configuration with the
    same constraints, so the full-space minimum is no higher."""
    p = build_problem("tiny_quasistatic")
    m = model_from_problem(p)
    sim = ReducedSimulator(m, 0.0, eps=1e-9)
    sim.step(p.targets(1))
    fm = FullModel(p.X0, p.tets, 1e5, 0.45, 1000.0, (0, 0, -9.8), p.cnodes)
    q, st = newton_solve(fm, p.X0.ravel(), p.targets(1), 1e-7)
    assert st.status == CONVERGED
    assert fm.energy(q) <= fm.energy(sim.q) + 1e-12
    assert abs(fm.energy(sim.q) - m.energy(sim.z)) < 1e-10
