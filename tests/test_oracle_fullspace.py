"""Pins of the oracle's full-space projective Newton solve (Eq. 1)."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dt", [0.0, 1.0 / 60.0])
def test_first_step_from_rest_is_the_linear_elastic_solution(dt):
    """From rest under a small gravity load, the first full Newton step
    (alpha = 1) solves (K0 + M / dt^2) u = M g on the free DOFs.  Here K0 is
    the stiffness assembled from the closed-form rest Hessian of the density,
    (3 mu / 4)(Id + T) + (lam - 5 mu / 8) v v^T.  Its vec(F) maps
    (F_ij = sum_a (x_a - x_0)_i (Dm^-1)_{a j}) and the lumped mass are built
    in this test, so the oracle's element Hessian, projection, assembly,
    constraint elimination and load terms are all checked against them."""
    mesh = make_bar(6, 3, 3, 0.05)
    cn = face_nodes(mesh, 0)
    E_, nu, rho = 1e5, 0.45, 1000.0
    mu, lam = E_ / (2 * (1 + nu)), E_ * nu / ((1 + nu) * (1 - 2 * nu))
    grav = np.array([0.0, 0.0, -1e-3])
    X, T4 = mesh.X0, mesh.tets
    nv = X.shape[0]
    n = 3 * nv
    v9 = np.eye(3).ravel()
    Tm = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            Tm[3 * i + j, 3 * j + i] = 1.0
    C0 = 0.75 * mu * (np.eye(9) + Tm) + (lam - 0.625 * mu) * np.outer(v9, v9)
    K = np.zeros((n, n))
    m = np.zeros(nv)
    for t in T4:
        Dm = np.stack([X[t[a]] - X[t[0]] for a in (1, 2, 3)], axis=1)
        Dmi = np.linalg.inv(Dm)
        V = np.linalg.det(Dm) / 6.0
        coef = np.vstack([-Dmi.sum(axis=0), Dmi])     # coef[a, j] = dF_ij / dx_{a,i}
        B = np.zeros((9, 12))
        for i in range(3):
            for j in range(3):
                for a in range(4):
                    B[3 * i + j, 3 * a + i] = coef[a, j]
        dofs = (3 * np.asarray(t)[:, None] + np.arange(3)).ravel()
        K[np.ix_(dofs, dofs)] += V * B.T @ C0 @ B
        m[t] += rho * V / 4.0
    mdof = np.repeat(m, 3)
    if dt > 0:
        K += np.diag(mdof / dt ** 2)
    f = mdof * np.tile(grav, nv)
    free = np.ones(n, bool)
    free[(3 * cn[:, None] + np.arange(3)).ravel()] = False
    u_lin = np.linalg.solve(K[np.ix_(free, free)], f[free])
    fm = FullModel(X, T4, E_, nu, rho, grav, cn)
    if dt > 0:
        fm.set_dynamics(dt, X.ravel() + dt ** 2 * np.tile(grav, nv))
    q1, st = newton_solve(fm, X.ravel(), X[cn], 1e-30, max_newton=1)
    assert st.newton_iters == 1 and st.ls_trials == 1     # full step accepted
    u1 = (q1 - X.ravel())[free]
    assert np.linalg.norm(u1 - u_lin) < 1e-9 * np.linalg.norm(u_lin)
