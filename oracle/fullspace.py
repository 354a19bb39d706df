"""Full-space implicit Euler / quasi-static solve of Eq. 1 (Sec. 3.1) by
projective Newton with Armijo backtracking: the fallback, the reference for
the subspace error, and the snapshot generator for decoder training (Sec. 3.2,
supervised setting).

Every tet is used with weight 1.  Constrained DOFs are held at their targets
and eliminated from the linear system; the assembled projected Hessian
(plus M / dt^2 in dynamics) restricted to the free DOFs is solved with a
sparse direct factorisation (library primitive).  Same exit codes and
Armijo rule as the reduced solve.

With project=False the exact Hessian is used instead (plain Newton), which
the pins use to check quadratic convergence; projective Newton itself
converges only linearly where elements are compressed (the projection is
active at the solution).

Pins (tests/test_oracle_fullspace.py): at rest with no load the solution is
X0 after zero iterations; plain Newton started near the solution converges
quadratically; the free-DOF gradient at the returned state is below eps;
the full-space minimum energy bounds the subspace minimum from below.
"""
from dataclasses import dataclass
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, snh
from .reduced import CONVERGED, MAX_ITERS, LS_FAILED, NOT_SPD


@dataclass
class FullStats:
    status: int
    newton_iters: int
    ls_trials: int
    grad_inf: float
    energy: float
    trace: list


class FullModel:
    def __init__(self, X0, tets, youngs, poisson, rho, gravity, cnodes,
                 project=True):
        self.project = project
        self.X0 = np.asarray(X0, np.float64)
        self.tets = np.asarray(tets, np.int64)
        self.nv = self.X0.shape[0]
        self.n = 3 * self.nv
        self.mu, self.lam = snh.lame(youngs, poisson)
        self.gravity = np.asarray(gravity, np.float64)
        self.DmInv, self.vol = fem.rest_shape(self.X0, self.tets)
        self.mass = fem.lumped_mass(self.nv, self.tets, self.vol, rho)
        self.mdof = np.repeat(self.mass, 3)
        self.cnodes = np.asarray(cnodes, np.int64)
        self.cdofs = (3 * self.cnodes[:, None] + np.arange(3)).ravel()
        free = np.ones(self.n, bool)
        free[self.cdofs] = False
        self.free = np.nonzero(free)[0]
        self.dt, self.qbar = 0.0, None

    def set_dynamics(self, dt, qbar):
        self.dt = float(dt)
        self.qbar = None if qbar is None else np.asarray(qbar, np.float64)

    def energy(self, q):
        Pe = fem.element_energy(q.reshape(-1, 3), self.tets, self.DmInv,
                                self.vol, self.mu, self.lam)
        E = float(np.sum(Pe))
        if self.dt > 0.0:
            d = q - self.qbar
            E += 0.5 / self.dt ** 2 * float(np.sum(self.mdof * d * d))
        else:
            E -= float(np.sum(self.mass[:, None] * self.gravity * q.reshape(-1, 3)))
        return E

    def gradient(self, q):
        ge = fem.element_gradient(q.reshape(-1, 3), self.tets, self.DmInv,
                                  self.vol, self.mu, self.lam)
        g = fem.assemble_gradient(ge, self.tets, self.n)
        if self.dt > 0.0:
            g += self.mdof * (q - self.qbar) / self.dt ** 2
        else:
            g -= (self.mass[:, None] * self.gravity).ravel()
        return g

    def hessian(self, q):
        He = fem.element_hessian(q.reshape(-1, 3), self.tets, self.DmInv,
                                 self.vol, self.mu, self.lam,
                                 project=self.project)
        K = fem.assemble_hessian(He, self.tets, self.n)
        if self.dt > 0.0:
            K = K + sp.diags(self.mdof / self.dt ** 2)
        return K.tocsr()


def newton_solve(model, q0, targets, eps, max_newton=1024, max_ls=128,
                 c=1e-4):
    q = np.asarray(q0, np.float64).copy()
    q[model.cdofs] = np.asarray(targets, np.float64).ravel()
    fr = model.free
    status, ls_total, trace = MAX_ITERS, 0, []
    it, E, gi = 0, None, None
    for it in range(max_newton + 1):
        E = model.energy(q)
        g = model.gradient(q)[fr]
        gi = float(np.max(np.abs(g)))
        trace.append((E, gi))
        if gi < eps:
            status = CONVERGED
            break
        if it == max_newton:
            break
        K = model.hessian(q)[fr][:, fr].tocsc()
        try:
            d = spla.spsolve(K, -g)
        except RuntimeError:
            status = NOT_SPD
            break
        if not np.all(np.isfinite(d)):
            status = NOT_SPD
            break
        gd = float(g @ d)
        alpha, accepted = 1.0, False
        for _ in range(max_ls):
            ls_total += 1
            qt = q.copy()
            qt[fr] += alpha * d
            if model.energy(qt) <= E + c * alpha * gd:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            status = LS_FAILED
            break
        q = qt
    return q, FullStats(status, it, ls_total, gi, E, trace)
