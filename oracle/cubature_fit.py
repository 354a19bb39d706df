"""Optimised cubature selection (Sec. 4.3: the cubature set and weights come
from a fit on the initial subspace, after von Tycowicz et al. 2013; the
cubature-count trade-off of Sec. 5.3).

TEST INFRASTRUCTURE: this module is part of the FP64 CPU oracle; only the
tests, the smoke check and the CPU baseline of the benchmark use it.

Readings (the paper names the method, not its details):

  * training forces: at K subspace points z_k the reduced elastic force of
    every tet e, a_{k,e} = J_e(z_k)^T dP_e/dx_e (r values, P_e = V_e Psi(F_e),
    unit weight, constrained rows of J zero), stacked into a column of
    A in R^{Kr x E}; the target is the full force b = sum_e a_{.,e}
    (every weight 1);
  * each snapshot's block of rows is divided by the norm of its b_k, so
    every snapshot counts alike (a block with b_k = 0 is left as it is);
  * the fit is non-negative least squares min ||A w - b||, w >= 0, by the
    Lawson-Hanson active-set method, which moves one column (the one with
    the largest gradient A^T (b - A w)) into the active set per outer
    iteration; it is stopped once S columns are active (or when no column
    has a positive gradient): the active columns are the cubature tets and
    w their weights.

Pins (tests/test_oracle_cubature.py): the columns sum to the reduced
elastic gradient of the assembled model; a consistent system with a sparse
non-negative solution is recovered exactly; a full run meets the KKT
conditions and reaches SciPy's NNLS residual; the residual does not grow
with S.
"""
import numpy as np

from . import fem


def tet_force_matrix(model, Z):
    """A (K r x E) of the per-tet reduced elastic forces at the points Z
    (K x r) for every tet of ``model`` (a ReducedModel; its cubature set is
    ignored: all tets, unit weights)."""
    tets, X0 = model.tets_all, model.X0
    DmInv, vol = fem.rest_shape(X0, tets)
    Z = np.atleast_2d(np.asarray(Z, dtype=np.float64))
    K, r = Z.shape
    E = tets.shape[0]
    A = np.zeros((K * r, E))
    dofs = fem.element_dofs(tets)                      # (E, 12)
    for k in range(K):
        x, J = model.positions_jac(Z[k])
        ge = fem.element_gradient(x.reshape(-1, 3), tets, DmInv, vol, model.mu, model.lam)
        Je = J[dofs]                                   # (E, 12, r)
        A[k * r:(k + 1) * r, :] = np.einsum("eki,ek->ie", Je, ge)
    return A


def normalise_blocks(A, r):
    """Divide each snapshot's r rows of A and of b = A 1 by ||b_k||."""
    A = A.copy()
    b = A.sum(axis=1)
    for k in range(A.shape[0] // r):
        sl = slice(k * r, (k + 1) * r)
        nb = np.linalg.norm(b[sl])
        if nb > 0.0:
            A[sl] /= nb
            b[sl] /= nb
    return A, b


def nnls_active_set(A, b, S=None, tol=None, max_inner=None):
    """Lawson-Hanson NNLS, stopped when S columns are active.  Returns
    (active column indices in the order they entered, their weights,
    relative residual ||A w - b|| / ||b||)."""
    m, n = A.shape
    S = n if S is None else int(S)
    x = np.zeros(n)
    active = []
    w_grad = A.T @ b
    if tol is None:
        tol = 1e-12 * max(1.0, float(np.max(np.abs(w_grad))))
    max_inner = 3 * n if max_inner is None else max_inner
    res = b.copy()
    while len(active) < S:
        w_grad = A.T @ res
        cand = w_grad.copy()
        cand[active] = -np.inf
        j = int(np.argmax(cand))
        if not cand[j] > tol:
            break
        active.append(j)
        for _ in range(max_inner):
            Ap = A[:, active]
            s = np.linalg.lstsq(Ap, b, rcond=None)[0]
            if np.all(s > 0.0):
                x[:] = 0.0
                x[active] = s
                break
            xp = x[active]
            neg = s <= 0.0
            alpha = float(np.min(xp[neg] / (xp[neg] - s[neg])))
            xp = xp + alpha * (s - xp)
            x[active] = xp
            keep = [a for a, v in zip(active, xp) if v > 1e-15]
            x[[a for a in active if a not in keep]] = 0.0
            active = keep
            if not active:
                break
        res = b - A @ x
    nb = float(np.linalg.norm(b))
    return np.array(active, dtype=np.int64), x[active], float(np.linalg.norm(res)) / (nb or 1.0)


def select_cubature(model, Z, S):
    """Cubature tets and weights for the model's decoder at the points Z."""
    r = np.atleast_2d(Z).shape[1]
    A, b = normalise_blocks(tet_force_matrix(model, Z), r)
    return nnls_active_set(A, b, S)
