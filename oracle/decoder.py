"""The neural subspace map f: R^r -> R^n of Sec. 3.1 (Eq. 2) as an MLP
(Sec. 1), with forward-mode derivatives.

Reading: hidden layers h_l = ELU(W_l h_{l-1} + b_l) with ELU(a) = a for
a > 0 and exp(a) - 1 otherwise; a linear last layer; positions
x = X0 + s * out with a fixed output scale s.  Derivatives propagate forward
(tangent propagation):
    first order   T_l = ELU'(a_l) * (W_l T_{l-1}),      T_0 = I_r
    second order  U_l = ELU''(a_l) (W_l T_{l-1}) (x) (W_l T_{l-1})
                        + ELU'(a_l) * (W_l U_{l-1}),     U_0 = 0
with ELU'(a) = 1, ELU''(a) = 0 for a > 0 and ELU'(a) = ELU''(a) = exp(a)
otherwise.  The last layer gives J = s W_L T_{L-1} and
d2x/dz2 = s W_L U_{L-1}.

Pins (tests/test_oracle_decoder.py): J and d2x/dz2 against central finite
differences; f(0) = 0 for zero biases; a one-layer decoder is affine.
"""
import numpy as np


def elu(a):
    return np.where(a > 0, a, np.expm1(np.minimum(a, 0.0)))


def elu_d1(a):
    return np.where(a > 0, 1.0, np.exp(np.minimum(a, 0.0)))


def elu_d2(a):
    return np.where(a > 0, 0.0, np.exp(np.minimum(a, 0.0)))


class Decoder:
    def __init__(self, Ws, bs, scale):
        self.Ws = [np.asarray(W, dtype=np.float64) for W in Ws]
        self.bs = [np.asarray(b, dtype=np.float64) for b in bs]
        self.scale = float(scale)

    @property
    def r(self):
        return self.Ws[0].shape[1]

    def hidden(self, z):
        h = np.asarray(z, dtype=np.float64)
        for W, b in zip(self.Ws[:-1], self.bs[:-1]):
            h = elu(W @ h + b)
        return h

    def out(self, z, rows=None):
        """s * f_raw(z) for the requested output rows (all by default)."""
        h = self.hidden(z)
        W, b = self.Ws[-1], self.bs[-1]
        if rows is not None:
            W, b = W[rows], b[rows]
        return self.scale * (W @ h + b)

    def out_jac(self, z, rows=None):
        """(s f(z), s df/dz) for the requested rows."""
        h = np.asarray(z, dtype=np.float64)
        T = np.eye(h.shape[0])
        for W, b in zip(self.Ws[:-1], self.bs[:-1]):
            a = W @ h + b
            T = elu_d1(a)[:, None] * (W @ T)
            h = elu(a)
        W, b = self.Ws[-1], self.bs[-1]
        if rows is not None:
            W, b = W[rows], b[rows]
        return self.scale * (W @ h + b), self.scale * (W @ T)

    def out_jac_hess(self, z, rows=None):
        """(s f, s df/dz, s d2f/dz2) with the last of shape (rows, r, r)."""
        h = np.asarray(z, dtype=np.float64)
        r = h.shape[0]
        T = np.eye(r)
        U = np.zeros((r, r, r))
        for W, b in zip(self.Ws[:-1], self.bs[:-1]):
            a = W @ h + b
            WT = W @ T
            WU = np.einsum("ij,jab->iab", W, U)
            U = (elu_d2(a)[:, None, None] * np.einsum("ia,ib->iab", WT, WT)
                 + elu_d1(a)[:, None, None] * WU)
            T = elu_d1(a)[:, None] * WT
            h = elu(a)
        W, b = self.Ws[-1], self.bs[-1]
        if rows is not None:
            W, b = W[rows], b[rows]
        return (self.scale * (W @ h + b), self.scale * (W @ T),
                self.scale * np.einsum("ij,jab->iab", W, U))
