"""Lipschitz-loss training objective of Sec. 4 in float64 (torch on the CPU).

Supervised setting (Sec. 3.2): a linear encoder g(q) = Ew (q - X0) + eb
(reading: the paper uses an autoencoder and gives no encoder form) and the
MLP decoder x(z) = X0 + s f(z) of the solver (ELU hidden layers, linear last
layer, no constraint override during training).

    L_C  = 1/B sum_b ||x(g(q_b)) - q_b||_M^2                          (Eq. 3)
    Ht(z) = d2/dz2 Pt(x(z)),  Pt = sum_{e in S} w_e V_e Psi(F_e)      (Sec. 4.3)
    L_LS = 1/(B(B-1)) sum_{i != j} ||Ht(z_i) - Ht(z_j)||_F^2 / ||z_i - z_j||^2   (Eq. 9)
    L    = L_C + lambda_LS L_LS                                         (Eq. 10)
    Lip ~ max_{i != j} ||Ht(z_i) - Ht(z_j)||_F / ||z_i - z_j||          (Eq. 7)

with z_i = g(q_i) and no gradient through the samples z_i in L_LS
(reading), the elastic term only (Sec. 4.2) and the exact, unprojected
Hessian obtained by automatic differentiation as in the paper (Sec. 5).
Only the rows of the decoder that the cubature tets touch enter Pt, so the
Hessian evaluates the last layer on those rows only (same function).

Unsupervised setting (Eq. 4, Sec. 3.2), over a batch of given samples
z_1..z_B (the caller draws them from N(0, I)):
    L_P   = 1/B sum_b Pt(x(z_b))                                      (potential loss)
    L_R   = 1/(B(B-1)) sum_{i != j} log(||x(z_i) - x(z_j)||_M / (sigma ||z_i - z_j||))^2
    L_U   = L_P + lambda L_R                                            (Eq. 4)
with the same cubature elastic potential Pt as the Lipschitz loss (reading:
the paper's P, with S = every tet as the exact case) and the expectations
taken as batch means over all ordered pairs (reading).  The encoder takes
no part (its gradient is zero).

Parameters are one flat float64 vector, in the order
    Ew (r x n, row-major), eb (r), then per decoder layer W_l (out x in), b_l.

Pins (tests/test_oracle_training.py): the autodiff Hessian equals the closed
form sum_e w_e (J_e^T H_e J_e + sum_k g_{e,k} d2x_k/dz2) assembled from the
numpy oracle; it equals central differences of the numpy reduced elastic
gradient; L_LS equals a brute-force double loop; the gradient of L w.r.t.
parameters equals central differences (8 random entries).
"""
import numpy as np
import torch

from . import fem, snh

torch_dtype = torch.float64


class TrainProblem:
    def __init__(self, X0, tets, widths, scale, youngs, poisson, rho, cub_idx, cub_w):
        self.X0 = np.asarray(X0, np.float64)
        self.nv = self.X0.shape[0]
        self.n = 3 * self.nv
        self.widths = list(widths)
        self.r = widths[0]
        self.scale = float(scale)
        tets = np.asarray(tets, np.int64)
        DmInv, vol = fem.rest_shape(self.X0, tets)
        self.mass = fem.lumped_mass(self.nv, tets, vol, rho)
        self.mu, self.lam = snh.lame(youngs, poisson)
        ci = np.asarray(cub_idx, np.int64)
        self.cw = torch.tensor(np.asarray(cub_w, np.float64) * vol[ci], dtype=torch_dtype)
        self.cDmInv = torch.tensor(DmInv[ci], dtype=torch_dtype)
        ctets = tets[ci]
        # decoder rows touched by the cubature tets, and local vertex slots
        verts = np.unique(ctets)
        self.cverts = verts
        self.rows = (3 * verts[:, None] + np.arange(3)).ravel()
        local = {v: i for i, v in enumerate(verts)}
        self.ctets_local = torch.tensor(np.vectorize(local.get)(ctets), dtype=torch.long)
        self.X0_rows = torch.tensor(self.X0.ravel()[self.rows], dtype=torch_dtype)
        self.massdof = torch.tensor(np.repeat(self.mass, 3), dtype=torch_dtype)
        self.X0t = torch.tensor(self.X0.ravel(), dtype=torch_dtype)
        # parameter layout
        self.shapes = [(self.r, self.n), (self.r,)]
        for a, b in zip(widths[:-1], widths[1:]):
            self.shapes += [(b, a), (b,)]
        self.sizes = [int(np.prod(s)) for s in self.shapes]

    # -- parameters ------------------------------------------------------
    def pack(self, Ew, eb, Ws, bs):
        parts = [np.asarray(Ew, np.float64).ravel(), np.asarray(eb, np.float64).ravel()]
        for W, b in zip(Ws, bs):
            parts += [np.asarray(W, np.float64).ravel(), np.asarray(b, np.float64).ravel()]
        return np.concatenate(parts)

    def unpack(self, theta):
        out, o = [], 0
        for shp, sz in zip(self.shapes, self.sizes):
            out.append(theta[o:o + sz].reshape(shp))
            o += sz
        return out

    # -- maps ------------------------------------------------------------
    def encode(self, P, Q):
        """z for positions Q (B, n)."""
        Ew, eb = P[0], P[1]
        return (Q - self.X0t) @ Ew.T + eb

    def decode(self, P, z, rows=None):
        """Positions x(z) for z of shape (..., r); all rows or the given rows."""
        h = z
        layers = P[2:]
        L = len(layers) // 2
        for l in range(L - 1):
            h = torch.nn.functional.elu(h @ layers[2 * l].T + layers[2 * l + 1])
        W, b = layers[2 * L - 2], layers[2 * L - 1]
        X0 = self.X0t
        if rows is not None:
            W, b, X0 = W[rows], b[rows], X0[rows]
        return X0 + self.scale * (h @ W.T + b)

    def cubature_potential(self, x_rows):
        """Pt for positions of the cubature rows (flat, as self.rows)."""
        xv = x_rows.reshape(-1, 3)[self.ctets_local]             # (S, 4, 3)
        Ds = torch.stack([xv[:, 1] - xv[:, 0], xv[:, 2] - xv[:, 0], xv[:, 3] - xv[:, 0]],
                         dim=2)
        F = Ds @ self.cDmInv
        Ic = (F * F).sum(dim=(1, 2))
        J = torch.linalg.det(F)
        a = 1.0 + 3.0 * self.mu / (4.0 * self.lam)
        psi0 = 0.5 * self.lam * (1.0 - a) ** 2 - self.mu * np.log(2.0)
        psi = (0.5 * self.mu * (Ic - 3.0) + 0.5 * self.lam * (J - a) ** 2
               - 0.5 * self.mu * torch.log(Ic + 1.0) - psi0)
        return (self.cw * psi).sum()

    def hessian(self, P, z, create_graph=False):
        """Ht(z) (r x r) by automatic differentiation."""
        rows = torch.tensor(self.rows, dtype=torch.long)
        f = lambda zz: self.cubature_potential(self.decode(P, zz, rows))
        return torch.autograd.functional.hessian(f, z, create_graph=create_graph)

    # -- losses ----------------------------------------------------------
    def losses(self, theta, Q, lam_ls, create_graph=False, Z_samples=None, order=2):
        """(L_C, L_LS, L, Z, H) for parameters theta (torch, flat) and snapshot
        positions Q (B, n).  The L_LS samples are z_i = g(q_i) without gradient
        (or the given Z_samples, which finite-difference checks hold fixed).
        order 0: the Lipschitz loss of the potential itself (the Supplement's
        order-o family, o = 0), 1/(B(B-1)) sum_{i != j} (Pt_i - Pt_j)^2 /
        ||z_i - z_j||^2; order 1: the same with the reduced gradients
        dPt/dz (squared Euclidean norm of the difference); order 2: Eq. 9."""
        P = self.unpack(theta)
        Z = self.encode(P, Q)
        X = self.decode(P, Z)
        R = X - Q
        Lc = (self.massdof * R * R).sum() / Q.shape[0]
        Zs = Z.detach() if Z_samples is None else Z_samples
        B = Q.shape[0]
        if lam_ls == 0.0 or B < 2:
            return Lc, torch.zeros((), dtype=torch_dtype), Lc, Zs, None
        if order == 0:
            rows = torch.tensor(self.rows, dtype=torch.long)
            Pz = torch.stack([self.cubature_potential(self.decode(P, Zs[b], rows))
                              for b in range(B)])
            dP = Pz[:, None] - Pz[None, :]
            dz = ((Zs[:, None] - Zs[None, :]) ** 2).sum(dim=2)
            off = ~torch.eye(B, dtype=torch.bool)
            L0 = (dP[off] ** 2 / dz[off]).sum() / (B * (B - 1))
            return Lc, L0, Lc + lam_ls * L0, Zs, None
        if order == 1:
            rows = torch.tensor(self.rows, dtype=torch.long)
            G = []
            for b in range(B):
                zb = Zs[b].clone().requires_grad_(True)
                pb = self.cubature_potential(self.decode(P, zb, rows))
                (gb,) = torch.autograd.grad(pb, zb, create_graph=True)
                G.append(gb)
            G = torch.stack(G)
            dG = ((G[:, None] - G[None, :]) ** 2).sum(dim=2)
            dz = ((Zs[:, None] - Zs[None, :]) ** 2).sum(dim=2)
            off = ~torch.eye(B, dtype=torch.bool)
            L1 = (dG[off] / dz[off]).sum() / (B * (B - 1))
            return Lc, L1, Lc + lam_ls * L1, Zs, None
        H = torch.stack([self.hessian(P, Zs[b], create_graph=create_graph) for b in range(B)])
        Lls = lipschitz_loss(H, Zs)
        return Lc, Lls, Lc + lam_ls * Lls, Zs, H


def unsupervised_losses(tp, theta, Z, lam, sigma):
    """(L_P, L_R, L_U) of Eq. 4 for parameters theta (torch, flat) and the
    samples Z (B, r)."""
    P = tp.unpack(theta)
    B = Z.shape[0]
    rows = torch.tensor(tp.rows, dtype=torch.long)
    Lp = sum(tp.cubature_potential(tp.decode(P, Z[b], rows)) for b in range(B)) / B
    X = tp.decode(P, Z)
    dX = X[:, None] - X[None, :]
    dm = (tp.massdof * dX * dX).sum(dim=2)                 # ||x_i - x_j||_M^2
    dz = ((Z[:, None] - Z[None, :]) ** 2).sum(dim=2)
    off = ~torch.eye(B, dtype=torch.bool)
    ell = 0.5 * torch.log(dm[off]) - np.log(sigma) - 0.5 * torch.log(dz[off])
    Lr = (ell * ell).sum() / (B * (B - 1))
    return Lp, Lr, Lp + lam * Lr


def unsupervised_loss_and_grad(tp, theta_np, Z_np, lam, sigma, lam_ls=0.0):
    """float64 losses (L_P, L_R, L_U, L_LS, L = L_U + lam_ls L_LS) and the
    gradient of L; L_LS (Eq. 9) at the same samples, held fixed."""
    theta = torch.tensor(theta_np, dtype=torch_dtype, requires_grad=True)
    Z = torch.tensor(Z_np, dtype=torch_dtype)
    Lp, Lr, Lu = unsupervised_losses(tp, theta, Z, lam, sigma)
    Lls = torch.zeros((), dtype=torch_dtype)
    if lam_ls != 0.0 and Z.shape[0] >= 2:
        P = tp.unpack(theta)
        H = torch.stack([tp.hessian(P, Z[b], create_graph=True) for b in range(Z.shape[0])])
        Lls = lipschitz_loss(H, Z)
    L = Lu + lam_ls * Lls
    (g,) = torch.autograd.grad(L, theta)
    return tuple(float(v.detach()) for v in (Lp, Lr, Lu, Lls, L)), g.numpy()


def lipschitz_loss(H, Z):
    """Eq. 9 with the Frobenius norm: mean over ordered pairs i != j."""
    B = H.shape[0]
    dH = H[:, None] - H[None, :]
    num = (dH * dH).sum(dim=(2, 3))
    dz = Z[:, None] - Z[None, :]
    den = (dz * dz).sum(dim=2)
    off = ~torch.eye(B, dtype=torch.bool)
    return (num[off] / den[off]).sum() / (B * (B - 1))


def lipschitz_estimate(H, Z):
    """Eq. 7: max over pairs of ||Ht_i - Ht_j|| / ||z_i - z_j||."""
    B = H.shape[0]
    best = 0.0
    for i in range(B):
        for j in range(B):
            if i != j:
                best = max(best, float(torch.linalg.norm(H[i] - H[j]) /
                                       torch.linalg.norm(Z[i] - Z[j])))
    return best


def loss_and_grad(tp, theta_np, Q_np, lam_ls, Z_samples=None, order=2):
    """float64 losses and the gradient of L w.r.t. the flat parameters (the
    L_LS samples held fixed, as in training)."""
    theta = torch.tensor(theta_np, dtype=torch_dtype, requires_grad=True)
    Q = torch.tensor(Q_np, dtype=torch_dtype)
    Zf = None if Z_samples is None else torch.tensor(Z_samples, dtype=torch_dtype)
    Lc, Lls, L, Z, H = tp.losses(theta, Q, lam_ls, create_graph=True, Z_samples=Zf,
                                 order=order)
    (g,) = torch.autograd.grad(L, theta)
    return ((float(Lc.detach()), float(Lls.detach()), float(L.detach())), g.numpy(),
            Z.numpy(), None if H is None else H.detach().numpy())


def closed_form_hessian(tp, dec, z):
    """sum_e w_e (J_e^T H_e J_e + sum_k g_{e,k} d2x_k/dz2) from the numpy oracle
    (unprojected element Hessians); used as an independent pin of the autodiff
    Hessian.  `dec` is an oracle.decoder.Decoder with the same weights."""
    o, J, D = dec.out_jac_hess(z, tp.rows)
    x_rows = tp.X0.ravel()[tp.rows] + o
    xv = x_rows.reshape(-1, 3)
    tl = tp.ctets_local.numpy()
    DmInv = tp.cDmInv.numpy()
    w = tp.cw.numpy()
    ones = np.ones(tl.shape[0])
    ge = fem.element_gradient(xv, tl, DmInv, ones, tp.mu, tp.lam)
    He = fem.element_hessian(xv, tl, DmInv, ones, tp.mu, tp.lam, project=False)
    dofs = fem.element_dofs(tl)
    Je, De = J[dofs], D[dofs]                              # (S,12,r), (S,12,r,r)
    H = np.einsum("e,eki,ekl,elj->ij", w, Je, He, Je)
    H += np.einsum("e,ek,ekij->ij", w, ge, De)
    return H
