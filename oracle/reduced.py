"""Reduced-order implicit Euler / quasi-static solve of Eq. 2 (Sec. 3.1) by
projective Newton with backtracking line search (Supplement, "Tests with
Projective Newton's method"; line-search cap of 128 and iteration cap of
1024 from Sec. 5; ||g||_inf < eps exit from the Supplement's convergence
discussion).

    E(z) = 1/(2 dt^2) ||x(z) - qbar||_M^2 + sum_{e in S} w_e P_e(x(z))   (dynamics)
    E(z) = sum_{e in S} w_e P_e(x(z)) - sum_v m_v g . x_v(z)             (quasi-static)

The elastic sum runs over a cubature set S with weights w_e (Eq. 11); S = all
tets with w = 1 is the exact potential.  x(z) = X0 + s f(z) with the
constrained DOFs overwritten by their prescribed targets and their rows of
J = dx/dz set to zero (reading: the paper names positional / moving
constraints but gives no mechanism).  Gravity enters dynamics through the
inertial guess qbar = q^k + dt v^k + dt^2 g (reading of Eq. 1's "inertial
guess determined by previous configurations and the external force") and
quasi-static solves as the potential -sum m_v g . x_v.

Affine modes (optional, off by default): a linear map in parallel with the
network (the "neural + linear in parallel" construction of prior subspace
methods that the paper's related work names; reading for free bodies, which
the network alone cannot translate or rotate):
    x(z) = X0 + s (f(z_nn) + Phi z_aff),   z = (z_nn, z_aff), z_aff in R^12,
    s Phi z_aff:  u_v = s (M (X0_v - c) + t),
    z_aff = (M_00, M_01, ..., M_22, t_0, t_1, t_2),
with c a fixed centre (the rest centroid) and s the decoder's output scale
(the affine coordinates share the network coordinates' scale, so that one
gradient tolerance suits both: in metres, the translation coordinate's
curvature is the body's whole m / dt^2 and its gradient stalls at the
rounding of E above the usual tolerance); s Phi is constant, so it is also
their columns of J.

Ground contact (optional, off by default): the penalty
    E_c = k/2 sum_v min(0, x_{v,z} - h)^2
on every vertex (Sec. 5's collision examples use a penalty; reading: plane
z = h, stiffness k, no mass weighting), with gradient k min(0, x_z - h) and
Gauss-Newton Hessian J^T diag(k [x_z < h]) J (the penalty's own Hessian).

Gradient:  g(z) = sum_e w_e J_e^T g_e + J^T M (x - qbar) / dt^2   (Eq. 11 form)
Hessian:   K(z) = sum_e w_e J_e^T Hproj_e J_e + J^T M J / dt^2   (Gauss-Newton:
           the term sum_k dE/dx_k d2x_k/dz2 is dropped; reading).
Exact form (opt-in, `eval_exact`): the dropped term added back over the free
           DOFs (the constrained ones do not move with z),
               K_x(z) = K(z) + sum_{k free} dE/dx_k d2x_k/dz2,
           then the r x r sum projected: eigenvalues below
           clamp * max_i |lambda_i| raised to that value (the Hessian of E(z)
           itself, differentiated twice through Eq. 2, with the per-element
           Hessians kept projected; reading of the projective Newton of the
           Supplement applied to the subspace Hessian).
Newton:    K d = -g by Cholesky; if K is not positive definite, retry with a
           diagonal shift tau = 1e-12 * max(1, max|diag K|), multiplied by 10
           per retry, 20 retries at most.
Armijo:    alpha = 1, halve until E(z + alpha d) <= E(z) + c alpha g.d.

Exit codes (shared meaning with the C ABI's status values):
    0 converged (||g||_inf < eps), 1 iteration cap, 2 line search exhausted,
    3 Hessian not positive definite after all shifts.

Pins (tests/test_oracle_reduced.py): reduced gradient equals J^T times the
assembled full gradient; with unprojected element Hessians the exact form
before its projection equals central differences of the reduced gradient,
and the added term vanishes for a linear decoder; K equals J^T Hproj_full J + J^T M J / dt^2;
finite differences of E give g; a linear decoder reproduces an independently
written linear-subspace Newton solve; a linear decoder with only the
quadratic inertia term converges in one Newton step to the closed-form
least-squares solution; rest state with no load has E = 0 and g = 0.
"""
from dataclasses import dataclass
import numpy as np

from . import fem, snh
from .decoder import Decoder

CONVERGED, MAX_ITERS, LS_FAILED, NOT_SPD = 0, 1, 2, 3


def chunk_terms(xv, J, tets, DmInv, vol, w, mu, lam, project=True):
    """Elastic terms of one chunk of cubature tets (Eq. 11 with the projected
    element Hessians, or the unprojected ones for pins):
    (sum_e w_e J_e^T g_e, sum_e w_e J_e^T Hproj_e J_e)."""
    r = J.shape[1]
    ge = fem.element_gradient(xv, tets, DmInv, vol, mu, lam)
    He = fem.element_hessian(xv, tets, DmInv, vol, mu, lam, project=project)
    Je = J[fem.element_dofs(tets)]                 # (c, 12, r)
    g = np.einsum("e,eki,ek->i", w, Je, ge)
    HJ = He @ Je                                   # H_e J_e
    WJ = w[:, None, None] * Je
    K = WJ.reshape(-1, r).T @ HJ.reshape(-1, r)    # sum_e w_e J_e^T H_e J_e
    return g, K


class ReducedModel:
    def __init__(self, X0, tets, decoder, youngs, poisson, rho, gravity,
                 cub_idx=None, cub_w=None, cnodes=None, chunk=65536, affine_center=None):
        self.X0 = np.asarray(X0, dtype=np.float64)
        self.tets_all = np.asarray(tets, dtype=np.int64)
        self.nv = self.X0.shape[0]
        self.n = 3 * self.nv
        self.dec = decoder
        self.mu, self.lam = snh.lame(youngs, poisson)
        self.gravity = np.asarray(gravity, dtype=np.float64)
        DmInv, vol = fem.rest_shape(self.X0, self.tets_all)
        self.mass = fem.lumped_mass(self.nv, self.tets_all, vol, rho)
        if cub_idx is None:
            cub_idx = np.arange(self.tets_all.shape[0])
            cub_w = np.ones(self.tets_all.shape[0])
        self.cub_idx = np.asarray(cub_idx, dtype=np.int64)
        self.w = np.asarray(cub_w, dtype=np.float64)
        self.tets = self.tets_all[self.cub_idx]
        self.DmInv = DmInv[self.cub_idx]
        self.vol = vol[self.cub_idx]
        self.cnodes = (np.zeros(0, dtype=np.int64) if cnodes is None
                       else np.asarray(cnodes, dtype=np.int64))
        self.cdofs = (3 * self.cnodes[:, None] + np.arange(3)).ravel()
        self.targets = self.X0[self.cnodes].copy()
        self.dt = 0.0
        self.qbar = None
        self.chunk = chunk
        self.pool = None               # optional oracle.pool.ElementPool
        self.ground_h, self.ground_k = 0.0, 0.0
        self.r_nn = decoder.r
        self.Phi = None
        if affine_center is not None:
            dX = self.X0 - np.asarray(affine_center, dtype=np.float64)
            self.Phi = np.zeros((self.n, 12))
            for a in range(3):
                self.Phi[a::3, 3 * a:3 * a + 3] = dX      # d u_{v,a} / d M_{a,b}
                self.Phi[a::3, 9 + a] = 1.0               # d u_{v,a} / d t_a
            self.Phi *= decoder.scale
        self.r = self.r_nn + (12 if self.Phi is not None else 0)

    # -- problem data ----------------------------------------------------
    def set_targets(self, targets):
        self.targets = np.asarray(targets, dtype=np.float64).reshape(-1, 3)

    def set_ground(self, height, stiffness):
        self.ground_h, self.ground_k = float(height), float(stiffness)

    def _ground(self, x):
        """Penalty energy, its x-gradient and its diagonal x-Hessian."""
        n = x.shape[0]
        g = np.zeros(n)
        h = np.zeros(n)
        if self.ground_k > 0.0:
            pen = np.minimum(0.0, x[2::3] - self.ground_h)
            g[2::3] = self.ground_k * pen
            h[2::3] = np.where(pen < 0.0, self.ground_k, 0.0)
            return 0.5 * self.ground_k * float(pen @ pen), g, h
        return 0.0, g, h

    def set_dynamics(self, dt, qbar):
        self.dt = float(dt)
        self.qbar = None if qbar is None else np.asarray(qbar, np.float64).ravel()

    # -- subspace map with constraints ------------------------------------
    def positions(self, z):
        z = np.asarray(z, dtype=np.float64)
        x = self.X0.ravel() + self.dec.out(z[:self.r_nn])
        if self.Phi is not None:
            x = x + self.Phi @ z[self.r_nn:]
        x[self.cdofs] = self.targets.ravel()
        return x

    def positions_jac(self, z):
        z = np.asarray(z, dtype=np.float64)
        o, J = self.dec.out_jac(z[:self.r_nn])
        x = self.X0.ravel() + o
        if self.Phi is not None:
            x = x + self.Phi @ z[self.r_nn:]
            J = np.hstack([J, self.Phi])
        x[self.cdofs] = self.targets.ravel()
        J[self.cdofs, :] = 0.0
        return x, J

    # -- objective -------------------------------------------------------
    def _mass_dof(self):
        return np.repeat(self.mass, 3)

    def energy_x(self, x):
        Pe = fem.element_energy(x.reshape(-1, 3), self.tets, self.DmInv,
                                self.vol, self.mu, self.lam)
        E = float(np.sum(self.w * Pe))
        m = self._mass_dof()
        if self.dt > 0.0:
            d = x - self.qbar
            E += 0.5 / self.dt ** 2 * float(np.sum(m * d * d))
        else:
            E -= float(np.sum(self.mass[:, None] * self.gravity[None, :]
                              * x.reshape(-1, 3)))
        return E + self._ground(x)[0]

    def energy(self, z):
        return self.energy_x(self.positions(z))

    def energy_grad(self, z):
        """E and the reduced gradient g = J^T dE/dx (no Hessian; L-BFGS)."""
        x, J = self.positions_jac(z)
        return self.energy_x(x), J.T @ self.full_gradient_x(x)

    def full_gradient_x(self, x):
        """dE/dx as an assembled n-vector (used by pins and the full space)."""
        ge = fem.element_gradient(x.reshape(-1, 3), self.tets, self.DmInv,
                                  self.vol, self.mu, self.lam)
        g = fem.assemble_gradient(ge, self.tets, self.n, self.w)
        m = self._mass_dof()
        if self.dt > 0.0:
            g += m * (x - self.qbar) / self.dt ** 2
        else:
            g -= (self.mass[:, None] * self.gravity[None, :]).ravel()
        return g + self._ground(x)[1]

    def eval(self, z, project=True):
        """E, reduced gradient g (r), Gauss-Newton reduced Hessian K (r, r)
        (project=False: unprojected element Hessians, for pins)."""
        x, J = self.positions_jac(z)
        r = J.shape[1]
        E = self.energy_x(x)
        g = np.zeros(r)
        K = np.zeros((r, r))
        xv = x.reshape(-1, 3)
        starts = range(0, self.tets.shape[0], self.chunk)
        if self.pool is not None and project:  # the same chunks, in worker processes
            parts = self.pool.chunk_terms(x, J, self.chunk)
        else:
            parts = (chunk_terms(xv, J, self.tets[s:s + self.chunk],
                                 self.DmInv[s:s + self.chunk], self.vol[s:s + self.chunk],
                                 self.w[s:s + self.chunk], self.mu, self.lam, project)
                     for s in starts)
        for gp, Kp in parts:           # summed in chunk order either way
            g += gp
            K += Kp
        m = self._mass_dof()
        if self.dt > 0.0:
            g += J.T @ (m * (x - self.qbar)) / self.dt ** 2
            K += (J.T * m) @ J / self.dt ** 2
        else:
            g -= J.T @ (self.mass[:, None] * self.gravity[None, :]).ravel()
        _, gc, hc = self._ground(x)
        if self.ground_k > 0.0:
            g += J.T @ gc
            K += (J.T * hc) @ J
        return E, g, 0.5 * (K + K.T)

    def curvature_term(self, z):
        """sum_{k free} dE/dx_k d2x_k/dz2 (r x r): the second derivative of
        the decoder (forward second-order tangents) contracted with the full
        gradient; zero in the affine coordinates (x is linear in them) and on
        the constrained DOFs."""
        z = np.asarray(z, dtype=np.float64)
        x = self.positions(z)
        G = self.full_gradient_x(x)
        G[self.cdofs] = 0.0
        _, _, Hx = self.dec.out_jac_hess(z[:self.r_nn])      # (n, r_nn, r_nn)
        C = np.zeros((self.r, self.r))
        C[:self.r_nn, :self.r_nn] = np.einsum("k,kab->ab", G, Hx)
        return C

    def eval_exact(self, z, clamp=1e-10, project=True):
        """E, g and the exact-form reduced Hessian: K + curvature_term,
        projected (eigenvalues below clamp * max |eigenvalue| raised to it);
        project=False returns the sum unprojected, with unprojected element
        Hessians (pins)."""
        E, g, K = self.eval(z, project=project)
        K = K + self.curvature_term(z)
        K = 0.5 * (K + K.T)
        if not project:
            return E, g, K
        lam_, Q = np.linalg.eigh(K)
        floor = clamp * max(float(np.max(np.abs(lam_))), np.finfo(float).tiny)
        return E, g, (Q * np.maximum(lam_, floor)) @ Q.T


@dataclass
class SolveStats:
    status: int
    newton_iters: int
    ls_trials: int
    grad_inf: float
    energy: float


def cholesky_direction(K, g):
    """Solve K d = -g by Cholesky with the diagonal-shift retry schedule."""
    shift = 0.0
    base = 1e-12 * max(1.0, float(np.max(np.abs(np.diag(K)))))
    for attempt in range(21):
        try:
            L = np.linalg.cholesky(K + shift * np.eye(K.shape[0]))
            y = np.linalg.solve(L, -g)
            return np.linalg.solve(L.T, y), True
        except np.linalg.LinAlgError:
            shift = base if shift == 0.0 else shift * 10.0
    return None, False


def newton_solve(model, z0, eps, max_newton=1024, max_ls=128, c=1e-4,
                 trace=None, exact=False):
    """exact: the exact-form reduced Hessian (ReducedModel.eval_exact)."""
    z = np.asarray(z0, dtype=np.float64).copy()
    status, ls_total, it = MAX_ITERS, 0, 0
    E = gi = None
    for it in range(max_newton + 1):
        E, g, K = model.eval_exact(z) if exact else model.eval(z)
        gi = float(np.max(np.abs(g)))
        if trace is not None:
            trace.append([E, gi, 0.0])
        if gi < eps:
            status = CONVERGED
            break
        if it == max_newton:
            break
        d, ok = cholesky_direction(K, g)
        if not ok:
            status = NOT_SPD
            break
        gd = float(g @ d)
        alpha, accepted = 1.0, False
        for _ in range(max_ls):
            ls_total += 1
            if model.energy(z + alpha * d) <= E + c * alpha * gd:
                accepted = True
                break
            alpha *= 0.5
        if not accepted:
            status = LS_FAILED
            break
        if trace is not None:
            trace[-1][2] = alpha
        z = z + alpha * d
    return z, SolveStats(status, it, ls_total, gi, E)


class ReducedSimulator:
    """Implicit Euler stepping (Eq. 2) or a quasi-static solve (dt = 0), each
    step solved by projective Newton or (optimizer="lbfgs") by L-BFGS."""

    def __init__(self, model, dt, z0=None, eps=1e-5, max_newton=1024,
                 max_ls=128, c=1e-4, optimizer="newton", history=10, v0=None,
                 exact_hessian=False):
        self.optimizer, self.history = optimizer, history
        self.exact = exact_hessian
        self.m = model
        self.dt = float(dt)
        r = model.r
        self.z = np.zeros(r) if z0 is None else np.asarray(z0, np.float64)
        self.q = model.positions(self.z)
        self.v = np.zeros_like(self.q) if v0 is None else np.asarray(v0, np.float64).copy()
        self.eps, self.max_newton, self.max_ls, self.c = eps, max_newton, max_ls, c

    def step(self, targets):
        m = self.m
        m.set_targets(targets)
        if self.dt > 0.0:
            g = np.tile(m.gravity, m.nv)
            m.set_dynamics(self.dt, self.q + self.dt * self.v + self.dt ** 2 * g)
        else:
            m.set_dynamics(0.0, None)
        if self.optimizer == "lbfgs":
            from .lbfgs import lbfgs_solve
            z, st = lbfgs_solve(m, self.z, self.eps, self.history, self.max_newton,
                                self.max_ls, self.c)
        else:
            z, st = newton_solve(m, self.z, self.eps, self.max_newton, self.max_ls,
                                 self.c, exact=self.exact)
        self.z = z
        qn = m.positions(z)
        if self.dt > 0.0:
            self.v = (qn - self.q) / self.dt
        self.q = qn
        return st


def model_from_problem(p, chunk=65536):
    """Oracle model for a ``workloads.Problem`` (with its affine modes and
    ground plane when the workload has them)."""
    c = p.config
    dec = Decoder(p.Ws, p.bs, c.out_scale)
    m = ReducedModel(p.X0, p.tets, dec, c.youngs, c.poisson, c.density,
                     c.gravity, p.cub_idx, p.cub_w, p.cnodes, chunk=chunk,
                     affine_center=getattr(p, "affine_center", None))
    if getattr(c, "ground_k", 0.0) > 0.0:
        m.set_ground(c.ground_h, c.ground_k)
    return m
