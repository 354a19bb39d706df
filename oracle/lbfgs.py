"""L-BFGS with backtracking line search for the reduced objective of Eq. 2
(Sec. 5: the optimiser of the main results, with its four exit conditions
I-IV and the caps of 128 line-search trials and 1024 iterations).

TEST INFRASTRUCTURE: this module is part of the FP64 CPU oracle; only the
tests, the smoke check and the CPU baseline of the benchmark use it.

The paper names the method and its exits but not its parts; the readings
taken here (each one also listed with the design notes):

  * direction d = -H g by the two-loop recursion over the m most recent
    curvature pairs (s_i, y_i) (Nocedal & Wright, Numerical Optimization,
    2nd ed., Algorithm 7.4), initial matrix H0 = gamma I with
    gamma = s^T y / y^T y of the newest pair (their Eq. 7.20), gamma = 1
    while the history is empty; m = 10 by default;
  * line search: Armijo backtracking from alpha = 1, halving, test
    E(z + alpha d) <= E(z) + c alpha g.d with c = 1e-4 (the same line search
    as the Newton solve), at most 128 trials (exit III);
  * after an accepted step the pair s = alpha d, y = g(z + s) - g(z) enters
    the history; if its curvature s^T y is not positive the objective has
    no positive curvature along the step: the solve ends with exit II
    ("encounters a saddle point");
  * exit I: ||g||_inf < eps at the current point; exit IV: the iteration cap.

Status codes: 0 converged (I), 1 iteration cap (IV), 2 line search
exhausted (III), 5 saddle point (II); the codes shared with the Newton solve
keep their meaning.

Pins (tests/test_oracle_lbfgs.py): the two-loop direction equals the product
with the explicitly updated BFGS inverse matrix; the secant condition holds
for the newest pair; on a strictly convex quadratic the solve reaches the
closed-form minimiser, and so it does on a strictly convex non-quadratic
function; a double well started near its maximum ends with exit II; the
reduced solve reaches a point where the Newton solve's gradient test passes.
(With a line search that tests only the Armijo condition nothing keeps
s^T y positive on a nonconvex function: on Rosenbrock's function from
(-1.2, 1) the fourth step already meets exit II.)
"""
from dataclasses import dataclass
import numpy as np

CONVERGED, MAX_ITERS, LS_FAILED, SADDLE = 0, 1, 2, 5


@dataclass
class LbfgsStats:
    status: int
    iters: int
    ls_trials: int
    grad_inf: float
    energy: float


def two_loop(g, S, Y):
    """-H g for the pairs S[i], Y[i] (oldest first), H0 = gamma I."""
    q = np.array(g, dtype=np.float64)
    k = len(S)
    a = np.zeros(k)
    rho = [1.0 / float(S[i] @ Y[i]) for i in range(k)]
    for i in range(k - 1, -1, -1):  # newest to oldest
        a[i] = rho[i] * float(S[i] @ q)
        q = q - a[i] * Y[i]
    gamma = float(S[-1] @ Y[-1]) / float(Y[-1] @ Y[-1]) if k else 1.0
    rr = gamma * q
    for i in range(k):  # oldest to newest
        b = rho[i] * float(Y[i] @ rr)
        rr = rr + (a[i] - b) * S[i]
    return -rr


def lbfgs_minimize(fun, grad, z0, eps, history=10, max_iters=1024, max_ls=128, c=1e-4,
                   trace=None):
    """Minimise fun from z0; grad(z) returns (E, g).  Returns (z, LbfgsStats)."""
    z = np.asarray(z0, dtype=np.float64).copy()
    S, Y = [], []
    E, g = grad(z)
    gi = float(np.max(np.abs(g)))
    ls_total, it, saddle = 0, 0, False
    while True:
        if trace is not None:
            trace.append([E, gi, 0.0])
        if gi < eps:
            status = CONVERGED
            break
        if saddle:
            status = SADDLE
            break
        if it == max_iters:
            status = MAX_ITERS
            break
        d = two_loop(g, S, Y)
        gd = float(g @ d)
        alpha, accepted = 1.0, False
        for _ in range(max_ls):
            ls_total += 1
            if fun(z + alpha * d) <= E + c * alpha * gd:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            status = LS_FAILED
            break
        if trace is not None:
            trace[-1][2] = alpha
        s = alpha * d
        z = z + s
        it += 1
        E, g_new = grad(z)
        y = g_new - g
        g = g_new
        gi = float(np.max(np.abs(g)))
        if float(s @ y) > 0.0:
            S.append(s)
            Y.append(y)
            if len(S) > history:
                S.pop(0)
                Y.pop(0)
        else:
            saddle = True  # reported unless the new point has converged
    return z, LbfgsStats(status, it, ls_total, gi, E)


def lbfgs_solve(model, z0, eps, history=10, max_iters=1024, max_ls=128, c=1e-4, trace=None):
    """L-BFGS on a ``ReducedModel`` (energy and gradient of Eq. 2)."""
    return lbfgs_minimize(model.energy, model.energy_grad, z0, eps, history, max_iters,
                          max_ls, c, trace)
