"""Pins of the oracle's L-BFGS solve (Sec. 5: optimiser of the main results,
exits I-IV) against textbook facts that do not depend on its code: the
explicit BFGS inverse update, the secant condition, closed-form minimisers,
and exit conditions forced by hand-picked functions."""
import numpy as np
import pytest

from oracle.lbfgs import (two_loop, lbfgs_minimize, lbfgs_solve, CONVERGED, MAX_ITERS,
                          LS_FAILED, SADDLE)
from oracle.reduced import newton_solve
from tests.test_oracle_reduced import tiny_model


def _spd(r, seed, cond=100.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((r, r)))
    return Q @ np.diag(np.geomspace(1.0, cond, r)) @ Q.T


def _pairs(A, k, seed):
    rng = np.random.default_rng(seed)
    S = [rng.standard_normal(A.shape[0]) for _ in range(k)]
    return S, [A @ s for s in S]


@pytest.mark.parametrize("k", [1, 3, 7])
def test_two_loop_equals_explicit_inverse_update(k):
    """d = -H g with H built by the matrix form of the BFGS update
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T from H0 = gamma I."""
    r = 7
    A = _spd(r, 1)
    S, Y = _pairs(A, k, 2)
    g = np.random.default_rng(3).standard_normal(r)
    H = (S[-1] @ Y[-1]) / (Y[-1] @ Y[-1]) * np.eye(r)
    I = np.eye(r)
    for s, y in zip(S, Y):
        rho = 1.0 / (s @ y)
        H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    assert np.allclose(two_loop(g, S, Y), -H @ g, rtol=1e-11, atol=1e-12)


def test_empty_history_is_steepest_descent():
    g = np.array([1.0, -2.0, 0.5])
    assert np.array_equal(two_loop(g, [], []), -g)


def test_secant_condition_of_newest_pair():
    A = _spd(6, 4)
    S, Y = _pairs(A, 4, 5)
    assert np.allclose(-two_loop(Y[-1], S, Y), S[-1], rtol=1e-11, atol=1e-12)


def test_quadratic_reaches_closed_form_minimiser():
    r = 6
    A = _spd(r, 6)
    zs = np.random.default_rng(7).standard_normal(r)
    # written around its minimiser so that E -> 0 there: the energy test of
    # the line search keeps resolving decreases down to tiny gradients
    f = lambda z: 0.5 * (z - zs) @ A @ (z - zs)
    fg = lambda z: (f(z), A @ (z - zs))
    z, st = lbfgs_minimize(f, fg, np.zeros(r), 1e-11)
    assert st.status == CONVERGED
    assert np.allclose(z, zs, rtol=1e-9, atol=1e-10)


def _convex(r, seed):
    """sum_i (sqrt(1 + w_i^2) - 1) + 0.05 |z - zs|^2 with w = B (z - zs):
    strictly convex, not quadratic, minimiser zs (value 0)."""
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((2 * r, r)) * 3.0
    zs = rng.standard_normal(r)

    def f(z):
        w = B @ (z - zs)
        return float(np.sum(np.sqrt(1 + w * w) - 1) + 0.05 * (z - zs) @ (z - zs))

    def fg(z):
        w = B @ (z - zs)
        return f(z), B.T @ (w / np.sqrt(1 + w * w)) + 0.1 * (z - zs)
    return f, fg, zs


def test_strictly_convex_function_reaches_its_minimiser():
    f, fg, zs = _convex(5, 8)
    z, st = lbfgs_minimize(f, fg, np.zeros(5), 1e-10)
    assert st.status == CONVERGED and np.allclose(z, zs, atol=1e-9)
    z3, st3 = lbfgs_minimize(f, fg, np.zeros(5), 1e-10, max_iters=3)
    assert st3.status == MAX_ITERS and st3.iters == 3


def test_double_well_from_near_its_maximum_is_a_saddle_exit():
    """f = z^4/4 - z^2/2 from z = 0.1: the unit step is accepted (Armijo) but
    crosses the concave region, so s^T y < 0 (exit II)."""
    f = lambda z: float(z[0] ** 4 / 4 - z[0] ** 2 / 2)
    fg = lambda z: (f(z), np.array([z[0] ** 3 - z[0]]))
    z, st = lbfgs_minimize(f, fg, np.array([0.1]), 1e-10)
    assert st.status == SADDLE and st.iters == 1 and z[0] == pytest.approx(0.199)


def test_line_search_cap():
    f = lambda z: float(50 * z @ z)
    fg = lambda z: (f(z), 100 * z)
    z, st = lbfgs_minimize(f, fg, np.ones(2), 1e-10, max_ls=1)
    assert st.status == LS_FAILED and st.ls_trials == 1 and np.array_equal(z, np.ones(2))


@pytest.mark.parametrize("dyn", [False, True])
def test_reduced_solve_reaches_the_newton_stationary_point(dyn):
    m = tiny_model(dyn)
    z0 = np.zeros(4)
    E, g, _ = m.eval(z0 + 0.1)
    E2, g2 = m.energy_grad(z0 + 0.1)
    assert E2 == pytest.approx(E, rel=1e-13) and np.allclose(g2, g, rtol=1e-10, atol=1e-12)
    zl, st = lbfgs_solve(m, z0, 1e-8)
    zn, stn = newton_solve(m, z0, 1e-10)
    assert st.status == CONVERGED and stn.status == CONVERGED
    assert np.max(np.abs(m.eval(zl)[1])) < 1e-8
    assert np.linalg.norm(zl - zn) <= 1e-5 * max(1.0, np.linalg.norm(zn))
