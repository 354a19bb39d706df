"""Stable Neo-Hookean energy density (Sec. 5.1 names the stable neo-Hookean
model of Smith et al. 2018 for every supervised example) and the PSD
projection used by projective Newton (Supplement, "Tests with Projective
Newton's method").

Reading of the paper (it gives no formula):
    Psi(F) = mu/2 (I_C - 3) + lam/2 (J - a)^2 - mu/2 log(I_C + 1) - Psi_0
with I_C = ||F||_F^2, J = det F, a = 1 + 3 mu / (4 lam) (the value for which
dPsi/dF vanishes at F = I) and Psi_0 = Psi(I) without the shift, so that the
energy is zero at rest.  mu and lam are the Lame parameters of the given
Young's modulus and Poisson ratio, used as they are (no reparametrisation).

Vectorisation convention: vec(F)[3 i + j] = F[i, j] (row-major).

Pins (tests/test_oracle_snh.py): Psi(I) = 0 and dPsi/dF(I) = 0; rotation and
isotropy invariance; central finite differences of Psi and of dPsi/dF; the
rest Hessian equals the hand-derived closed form
(3 mu / 4)(I + T) + (lam - 5 mu / 8) vec(I) vec(I)^T; torch float64
autodiff of an independent torch transcription; projection characterised by
A - P(A) <= 0, P(A) >= 0 and P(A)(A - P(A)) = 0.
"""
import numpy as np

# Levi-Civita symbol, written out from its definition
LEVI = np.zeros((3, 3, 3))
for (i, j, k), s in {(0, 1, 2): 1, (1, 2, 0): 1, (2, 0, 1): 1,
                     (0, 2, 1): -1, (2, 1, 0): -1, (1, 0, 2): -1}.items():
    LEVI[i, j, k] = s


def lame(youngs, poisson):
    mu = youngs / (2.0 * (1.0 + poisson))
    lam = youngs * poisson / ((1.0 + poisson) * (1.0 - 2.0 * poisson))
    return mu, lam


def snh_alpha(mu, lam):
    return 1.0 + 3.0 * mu / (4.0 * lam)


def snh_psi0(mu, lam):
    a = snh_alpha(mu, lam)
    return 0.5 * lam * (1.0 - a) ** 2 - 0.5 * mu * np.log(4.0)


def det3(F):
    return np.linalg.det(F)


def cofactor(F):
    """cof(F)_ij = dJ/dF_ij = 1/2 eps_ikm eps_jln F_kl F_mn."""
    return 0.5 * np.einsum("ikm,jln,...kl,...mn->...ij", LEVI, LEVI, F, F)


def d2J_dF2(F):
    """d^2 J / dF_ij dF_kl = eps_ikm eps_jln F_mn, as a (..., 9, 9) matrix."""
    T = np.einsum("ikm,jln,...mn->...ijkl", LEVI, LEVI, F)
    return T.reshape(F.shape[:-2] + (9, 9))


def psi(F, mu, lam):
    Ic = np.einsum("...ij,...ij->...", F, F)
    J = det3(F)
    a = snh_alpha(mu, lam)
    return (0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - a) ** 2
            - 0.5 * mu * np.log(Ic + 1.0) - snh_psi0(mu, lam))


def dpsi_dF(F, mu, lam):
    Ic = np.einsum("...ij,...ij->...", F, F)[..., None, None]
    J = det3(F)[..., None, None]
    a = snh_alpha(mu, lam)
    return mu * F + lam * (J - a) * cofactor(F) - mu * F / (Ic + 1.0)


def d2psi_dF2(F, mu, lam):
    """(..., 9, 9) second derivative in row-major vec ordering."""
    Ic = np.einsum("...ij,...ij->...", F, F)[..., None, None]
    J = det3(F)[..., None, None]
    a = snh_alpha(mu, lam)
    f = F.reshape(F.shape[:-2] + (9,))
    c = cofactor(F).reshape(F.shape[:-2] + (9,))
    eye = np.broadcast_to(np.eye(9), F.shape[:-2] + (9, 9))
    return (mu * (1.0 - 1.0 / (Ic + 1.0)) * eye
            + 2.0 * mu / (Ic + 1.0) ** 2 * np.einsum("...a,...b->...ab", f, f)
            + lam * np.einsum("...a,...b->...ab", c, c)
            + lam * (J - a) * d2J_dF2(F))


def project_psd(A):
    """Closest PSD matrix in the Frobenius norm: eigen-decompose the symmetric
    matrix and clamp negative eigenvalues to zero."""
    A = 0.5 * (A + np.swapaxes(A, -1, -2))
    lam_, Q = np.linalg.eigh(A)
    lam_ = np.maximum(lam_, 0.0)
    return np.einsum("...ik,...k,...jk->...ij", Q, lam_, Q)
