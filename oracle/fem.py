"""Tetrahedral FEM quantities for Eq. 1-2 (Sec. 3.1): the DOF vector q holds
the vertex positions (xyz interleaved, q[3 v + c]); M is the lumped mass
matrix; P(q) is the elastic potential obtained by integrating the energy
density over each linear tetrahedron.

Per element e with vertices (v0, v1, v2, v3):
    Dm = [X1-X0, X2-X0, X3-X0] (rest edges as columns), V_e = det(Dm)/6,
    F  = Ds Dm^-1 with Ds the same edge matrix of the deformed positions,
    P_e = V_e Psi(F),  g_e = dP_e/dx_e = V_e B^T vec(dPsi/dF),
    H_e = V_e B^T dPsi2 B, and the projected H_e uses P_psd(dPsi2),
where B = d vec(F) / d x_e is 9 x 12 and x_e = [x_v0, x_v1, x_v2, x_v3].
Lumped mass: m_v = sum over elements containing v of rho V_e / 4.

Pins (tests/test_oracle_fem.py): volumes sum to the bar volume; F equals A
for every tet under x = A X; central finite differences of P_e and g_e;
assembled gradient / Hessian equal the element sums; total mass is rho times
the volume.
"""
import numpy as np
import scipy.sparse as sp

from . import snh


def rest_shape(X0, tets):
    """Returns (DmInv (E,3,3), vol (E,))."""
    X = X0[tets]                                  # (E, 4, 3)
    Dm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]],
                  axis=2)                         # columns are edges
    vol = np.linalg.det(Dm) / 6.0
    return np.linalg.inv(Dm), vol


def lumped_mass(nv, tets, vol, rho):
    m = np.zeros(nv)
    for a in range(4):
        np.add.at(m, tets[:, a], rho * vol / 4.0)
    return m


def deformation_gradient(x, tets, DmInv):
    """x is (nv, 3)."""
    P = x[tets]
    Ds = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]],
                  axis=2)
    return Ds @ DmInv


def dF_dx(DmInv):
    """B[e, 3i+j, 3a+c] = delta_ic * D[e, a, j], D[e,0,:] = -sum_k DmInv[e,k,:],
    D[e,a,:] = DmInv[e,a-1,:] for a = 1..3."""
    E = DmInv.shape[0]
    D = np.concatenate([-DmInv.sum(axis=1, keepdims=True), DmInv], axis=1)
    B = np.zeros((E, 3, 3, 4, 3))
    for i in range(3):
        B[:, i, :, :, i] = np.swapaxes(D, 1, 2)    # [e, j, a]
    return B.reshape(E, 9, 12)


def element_energy(x, tets, DmInv, vol, mu, lam):
    F = deformation_gradient(x, tets, DmInv)
    return vol * snh.psi(F, mu, lam)


def element_gradient(x, tets, DmInv, vol, mu, lam):
    F = deformation_gradient(x, tets, DmInv)
    B = dF_dx(DmInv)
    p = snh.dpsi_dF(F, mu, lam).reshape(-1, 9)
    return vol[:, None] * np.einsum("eak,ea->ek", B, p)


def element_hessian(x, tets, DmInv, vol, mu, lam, project=True):
    F = deformation_gradient(x, tets, DmInv)
    B = dF_dx(DmInv)
    A = snh.d2psi_dF2(F, mu, lam)
    if project:
        A = snh.project_psd(A)
    return vol[:, None, None] * np.einsum("eak,eab,ebl->ekl", B, A, B)


def element_dofs(tets):
    """(E, 12) global DOF index of each element DOF."""
    return (3 * tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)


def assemble_gradient(ge, tets, n, w=None):
    w = np.ones(ge.shape[0]) if w is None else w
    g = np.zeros(n)
    np.add.at(g, element_dofs(tets), w[:, None] * ge)
    return g


def assemble_hessian(He, tets, n, w=None):
    w = np.ones(He.shape[0]) if w is None else w
    dofs = element_dofs(tets)
    rows = np.repeat(dofs, 12, axis=1).ravel()
    cols = np.tile(dofs, (1, 12)).ravel()
    vals = (w[:, None, None] * He).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
