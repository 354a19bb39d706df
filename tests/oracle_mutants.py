"""Plausible mistakes planted in the oracle, on the CPU, to show that its pins
catch them (tests/test_oracle_pins_catch_mutants.py).  Each mutant swaps one
oracle function, or method, for a wrong variant.  The swap reaches every
loaded module that holds a reference to the original, so it also covers
`from oracle.x import f` bindings.  Nothing here is used outside that test."""
import importlib
import sys

import numpy as np

ORACLE = ("oracle.snh", "oracle.fem", "oracle.decoder", "oracle.reduced", "oracle.fullspace",
          "oracle.lbfgs", "oracle.cubature_fit", "oracle.training")


def _swap(module_name, attr, make):
    for m in ORACLE:
        importlib.import_module(m)
    mod = importlib.import_module(module_name)
    old = getattr(mod, attr)
    new = make(old)
    for m in list(sys.modules.values()):
        name = getattr(m, "__name__", "") or ""
        if name.startswith(("oracle", "tests")):
            for k, v in list(vars(m).items()):
                if v is old:
                    setattr(m, k, new)
    setattr(mod, attr, new)


def _swap_method(module_name, cls, attr, make):
    for m in ORACLE:
        importlib.import_module(m)
    klass = getattr(importlib.import_module(module_name), cls)
    setattr(klass, attr, make(getattr(klass, attr)))


def _psi_without_log(old):
    def psi(F, mu, lam):   # the -mu/2 log(Ic + 1) term dropped (rest value kept at 0)
        Ic = np.einsum("...ij,...ij->...", F, F)
        return old(F, mu, lam) + 0.5 * mu * (np.log(Ic + 1.0) - np.log(4.0))
    return psi


def _stress_transposed(old):
    return lambda F, mu, lam: np.swapaxes(old(F, mu, lam), -1, -2)


def _psd_by_abs(old):
    def project_psd(A):    # |lambda| instead of max(lambda, 0)
        A = 0.5 * (A + np.swapaxes(A, -1, -2))
        w, Q = np.linalg.eigh(A)
        return np.einsum("...ik,...k,...jk->...ij", Q, np.abs(w), Q)
    return project_psd


def _mass_thirds(old):
    return lambda nv, tets, vol, rho: old(nv, tets, vol, rho) * (4.0 / 3.0)


def _vertex0_sign(old):
    def dF_dx(DmInv):      # vertex 0's columns with the wrong sign
        B = old(DmInv).copy()
        B[:, :, 0:3] *= -1.0
        return B
    return dF_dx


def _elu_d1_wrong_branch(old):
    return lambda a: np.where(a > 0.0, np.exp(np.minimum(a, 50.0)), 1.0)


def _inertia_over_dt(old):
    def full_gradient_x(self, x):   # M (x - qbar) / dt instead of / dt^2
        g = old(self, x)
        if self.dt > 0.0:
            d = np.repeat(self.mass, 3) * (x - self.qbar)
            g = g - d / self.dt ** 2 + d / self.dt
        return g
    return full_gradient_x


def _ground_energy_doubled(old):
    def _ground(self, x):
        E, g, h = old(self, x)
        return 2.0 * E, g, h
    return _ground


def _two_loop_reversed(old):
    return lambda g, S, Y: old(g, list(S)[::-1], list(Y)[::-1])


def _nnls_weights_off(old):
    def nnls_active_set(A, b, S=None, tol=None, max_inner=None):
        idx, w, rel = old(A, b, S, tol, max_inner)
        return idx, 1.01 * w, rel
    return nnls_active_set


def _lipschitz_unordered(old):
    return lambda H, Z: 2.0 * old(H, Z)   # mean over unordered pairs


def _fullspace_gravity_sign(old):
    def gradient(self, q):
        g = old(self, q)
        if self.dt == 0.0:
            g = g + 2.0 * (self.mass[:, None] * self.gravity).ravel()
        return g
    return gradient


def _elu_d2_zero(old):
    return lambda a: np.zeros_like(np.asarray(a, dtype=np.float64))


def _repulsion_halved(old):
    def unsupervised_losses(tp, theta, Z, lam, sigma):
        Lp, Lr, _ = old(tp, theta, Z, lam, sigma)
        return Lp, 0.5 * Lr, Lp + lam * 0.5 * Lr
    return unsupervised_losses


def _forces_scaled(old):
    return lambda model, Z: 1.0001 * old(model, Z)


def _gradient_unweighted(old):
    return lambda ge, tets, n, w=None: old(ge, tets, n, None)


def _steepest_descent(old):
    def cholesky_direction(K, g):   # -g instead of -K^-1 g
        d, ok = old(K, g)
        return (-np.asarray(g, dtype=np.float64), ok) if ok else (d, ok)
    return cholesky_direction


# name: (apply, the pin files that must catch it)
def _curvature_on_constrained_rows(old):
    def curvature_term(self, z):   # the constrained DOFs' reactions kept in the sum
        z = np.asarray(z, dtype=np.float64)
        G = self.full_gradient_x(self.positions(z))
        _, _, Hx = self.dec.out_jac_hess(z[:self.r_nn])
        C = np.zeros((self.r, self.r))
        C[:self.r_nn, :self.r_nn] = np.einsum("k,kab->ab", G, Hx)
        return C
    return curvature_term


def _curvature_sign(old):
    return lambda self, z: -old(self, z)


MUTANTS = {
    "curvature_on_constrained_rows": (lambda: _swap_method("oracle.reduced", "ReducedModel",
                                                           "curvature_term",
                                                           _curvature_on_constrained_rows),
                                      ["tests/test_oracle_reduced.py"]),
    "curvature_sign": (lambda: _swap_method("oracle.reduced", "ReducedModel", "curvature_term",
                                            _curvature_sign),
                       ["tests/test_oracle_reduced.py"]),
    "snh_psi_without_log_term": (lambda: _swap("oracle.snh", "psi", _psi_without_log),
                                 ["tests/test_oracle_snh.py"]),
    "snh_stress_transposed": (lambda: _swap("oracle.snh", "dpsi_dF", _stress_transposed),
                              ["tests/test_oracle_snh.py"]),
    "psd_projection_by_abs": (lambda: _swap("oracle.snh", "project_psd", _psd_by_abs),
                              ["tests/test_oracle_snh.py"]),
    "lumped_mass_thirds": (lambda: _swap("oracle.fem", "lumped_mass", _mass_thirds),
                           ["tests/test_oracle_fem.py"]),
    "dF_dx_vertex0_sign": (lambda: _swap("oracle.fem", "dF_dx", _vertex0_sign),
                           ["tests/test_oracle_fem.py"]),
    "elu_derivative_wrong_branch": (lambda: _swap("oracle.decoder", "elu_d1",
                                                  _elu_d1_wrong_branch),
                                    ["tests/test_oracle_decoder.py"]),
    "inertia_over_dt": (lambda: _swap_method("oracle.reduced", "ReducedModel",
                                             "full_gradient_x", _inertia_over_dt),
                        ["tests/test_oracle_reduced.py"]),
    "ground_energy_doubled": (lambda: _swap_method("oracle.reduced", "ReducedModel", "_ground",
                                                   _ground_energy_doubled),
                              ["tests/test_oracle_reduced.py"]),
    "two_loop_pairs_reversed": (lambda: _swap("oracle.lbfgs", "two_loop", _two_loop_reversed),
                                ["tests/test_oracle_lbfgs.py"]),
    "nnls_weights_off": (lambda: _swap("oracle.cubature_fit", "nnls_active_set",
                                       _nnls_weights_off),
                         ["tests/test_oracle_cubature.py"]),
    "lipschitz_unordered_pairs": (lambda: _swap("oracle.training", "lipschitz_loss",
                                                _lipschitz_unordered),
                                  ["tests/test_oracle_training.py"]),
    "fullspace_gravity_sign": (lambda: _swap_method("oracle.fullspace", "FullModel", "gradient",
                                                    _fullspace_gravity_sign),
                               ["tests/test_oracle_fullspace.py"]),
    "elu_second_derivative_zero": (lambda: _swap("oracle.decoder", "elu_d2", _elu_d2_zero),
                                   ["tests/test_oracle_decoder.py"]),
    "unsupervised_repulsion_halved": (lambda: _swap("oracle.training", "unsupervised_losses",
                                                    _repulsion_halved),
                                      ["tests/test_oracle_training.py"]),
    "tet_forces_scaled": (lambda: _swap("oracle.cubature_fit", "tet_force_matrix",
                                        _forces_scaled),
                          ["tests/test_oracle_cubature.py"]),
    "cubature_weights_ignored": (lambda: _swap("oracle.fem", "assemble_gradient",
                                               _gradient_unweighted),
                                 ["tests/test_oracle_fem.py"]),
    "newton_direction_is_steepest_descent": (lambda: _swap("oracle.reduced", "cholesky_direction",
                                                           _steepest_descent),
                                             ["tests/test_oracle_reduced.py"]),
}


def apply(name):
    MUTANTS[name][0]()
