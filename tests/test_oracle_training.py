"""Pins of the oracle's training objective (Sec. 4: Eq. 3, 7, 9, 10, 11)."""
import numpy as np
import pytest
import torch

from oracle import fem
from oracle.decoder import Decoder
from oracle.training import (TrainProblem, lipschitz_loss, lipschitz_estimate,
                             loss_and_grad, closed_form_hessian)
from workloads import make_bar, xavier_decoder


@pytest.fixture(scope="module")
def setup():
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    widths = [3, 8, 8, n]
    rng = np.random.default_rng(0)
    cub = np.sort(rng.choice(mesh.ne, 10, replace=False))
    w = rng.uniform(0.5, 4.0, 10)
    tp = TrainProblem(mesh.X0, mesh.tets, widths, 0.05, 1e5, 0.45, 1000.0, cub, w)
    Ws, bs = xavier_decoder(widths, 1)
    bs = [0.05 * rng.standard_normal(b.shape) for b in bs]
    Ew = 0.3 * rng.standard_normal((3, n))
    eb = 0.1 * rng.standard_normal(3)
    theta = tp.pack(Ew, eb, Ws, bs)
    Q = mesh.X0.ravel()[None] + 0.02 * rng.standard_normal((4, n))
    return tp, theta, Q, Ws, bs


def test_autodiff_hessian_equals_closed_form(setup):
    tp, theta, Q, Ws, bs = setup
    P = tp.unpack(torch.tensor(theta))
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    for z in np.random.default_rng(1).standard_normal((3, 3)):
        H = tp.hessian(P, torch.tensor(z)).numpy()
        Hc = closed_form_hessian(tp, dec, z)
        assert np.allclose(H, Hc, rtol=1e-9, atol=1e-9 * np.abs(Hc).max())
        assert np.allclose(H, H.T, atol=1e-12 * np.abs(H).max())


def test_hessian_equals_differences_of_reduced_gradient(setup):
    tp, theta, Q, Ws, bs = setup
    P = tp.unpack(torch.tensor(theta))
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    tl = tp.ctets_local.numpy()
    ones = np.ones(tl.shape[0])

    def grad(z):  # sum_e w_e J_e^T g_e (Eq. 11 over the cubature set)
        o, J = dec.out_jac(z, tp.rows)
        xv = (tp.X0.ravel()[tp.rows] + o).reshape(-1, 3)
        ge = fem.element_gradient(xv, tl, tp.cDmInv.numpy(), ones, tp.mu, tp.lam)
        return np.einsum("e,eki,ek->i", tp.cw.numpy(), J[fem.element_dofs(tl)], ge)

    z = np.array([0.3, -0.7, 0.4])
    H = tp.hessian(P, torch.tensor(z)).numpy()
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (grad(z + e) - grad(z - e)) / (2 * h)
        assert np.allclose(fd, H[:, k], rtol=1e-5, atol=1e-6 * np.abs(H).max())


def test_lipschitz_loss_brute_force():
    rng = np.random.default_rng(2)
    H = torch.tensor(rng.standard_normal((3, 4, 4)))
    H = H + H.transpose(1, 2)
    Z = torch.tensor(rng.standard_normal((3, 4)))
    tot = 0.0
    for i in range(3):
        for j in range(3):
            if i != j:
                tot += float(((H[i] - H[j]) ** 2).sum() / ((Z[i] - Z[j]) ** 2).sum())
    assert float(lipschitz_loss(H, Z)) == pytest.approx(tot / 6, rel=1e-14)
    best = max(float(torch.linalg.norm(H[i] - H[j]) / torch.linalg.norm(Z[i] - Z[j]))
               for i in range(3) for j in range(3) if i != j)
    assert lipschitz_estimate(H, Z) == pytest.approx(best, rel=1e-14)
    # two samples: the mean over the two ordered pairs is the single ratio
    assert float(lipschitz_loss(H[:2], Z[:2])) == pytest.approx(
        float(((H[0] - H[1]) ** 2).sum() / ((Z[0] - Z[1]) ** 2).sum()), rel=1e-14)


def test_reconstruction_loss_definition(setup):
    tp, theta, Q, Ws, bs = setup
    (Lc, Lls, L), g, Z, H = loss_and_grad(tp, theta, Q, 0.0)
    P = tp.unpack(torch.tensor(theta))
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    Ew, eb = theta[:3 * tp.n].reshape(3, tp.n), theta[3 * tp.n:3 * tp.n + 3]
    ref = 0.0
    for q in Q:
        z = Ew @ (q - tp.X0.ravel()) + eb
        x = tp.X0.ravel() + dec.out(z)
        ref += np.sum(np.repeat(tp.mass, 3) * (x - q) ** 2)
    assert Lc == pytest.approx(ref / Q.shape[0], rel=1e-12)
    assert Lls == 0.0 and L == Lc


@pytest.mark.parametrize("lam_ls", [0.0, 1e-3])
def test_parameter_gradient_by_central_differences(setup, lam_ls):
    tp, theta, Q, Ws, bs = setup
    (Lc, Lls, L), g, Z, H = loss_and_grad(tp, theta, Q, lam_ls)
    rng = np.random.default_rng(100)
    idx = rng.choice(theta.shape[0], 8, replace=False)
    # include a last-layer weight of a cubature row and a hidden weight
    for k in idx:
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp_, tm_ = theta.copy(), theta.copy()
        tp_[k] += h
        tm_[k] -= h
        # the Lipschitz samples z_i carry no gradient: hold them fixed
        Lp = loss_and_grad(tp, tp_, Q, lam_ls, Z_samples=Z)[0][2]
        Lm = loss_and_grad(tp, tm_, Q, lam_ls, Z_samples=Z)[0][2]
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-8 * max(1.0, abs(L)))


def test_unsupervised_losses_against_independent_sums(setup):
    """Eq. 4: L_P equals the numpy oracle's cubature elastic energy at the
    decoded positions; L_R equals a double loop over ordered pairs."""
    from oracle.training import unsupervised_losses
    tp, theta, Q, Ws, bs = setup
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    Z = np.random.default_rng(5).standard_normal((4, 3))
    lam, sigma = 0.3, 0.02
    Lp, Lr, L = (float(v) for v in unsupervised_losses(tp, torch.tensor(theta), torch.tensor(Z),
                                                       lam, sigma))
    tl = tp.ctets_local.numpy()
    DmInv = tp.cDmInv.numpy()
    cw = tp.cw.numpy()
    Ep = 0.0
    X = []
    for z in Z:
        x = tp.X0.ravel() + dec.out(z)
        X.append(x)
        xv = x[tp.rows].reshape(-1, 3)
        Ep += float(np.sum(cw * fem.element_energy(xv, tl, DmInv, np.ones(len(tl)), tp.mu, tp.lam)))
    assert Lp == pytest.approx(Ep / 4, rel=1e-12)
    m = np.repeat(tp.mass, 3)
    acc = 0.0
    for i in range(4):
        for j in range(4):
            if i != j:
                d = np.sqrt(np.sum(m * (X[i] - X[j]) ** 2))
                acc += np.log(d / (sigma * np.linalg.norm(Z[i] - Z[j]))) ** 2
    assert Lr == pytest.approx(acc / 12, rel=1e-12)
    assert L == pytest.approx(Lp + lam * Lr, rel=1e-14)


def test_unsupervised_gradient_matches_central_differences(setup):
    from oracle.training import unsupervised_loss_and_grad
    tp, theta, Q, Ws, bs = setup
    Z = np.random.default_rng(6).standard_normal((4, 3))
    (Lp, Lr, Lu, Lls, L), g = unsupervised_loss_and_grad(tp, theta, Z, 0.3, 0.02, 1e-3)
    assert L == pytest.approx(Lu + 1e-3 * Lls, rel=1e-14) and Lls > 0.0
    n_enc = tp.sizes[0] + tp.sizes[1]
    assert np.all(g[:n_enc] == 0.0)          # the encoder takes no part
    rng = np.random.default_rng(101)
    for k in rng.choice(np.arange(n_enc, theta.size), 8, replace=False):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp_, tm_ = theta.copy(), theta.copy()
        tp_[k] += h
        tm_[k] -= h
        fd = (unsupervised_loss_and_grad(tp, tp_, Z, 0.3, 0.02, 1e-3)[0][4] -
              unsupervised_loss_and_grad(tp, tm_, Z, 0.3, 0.02, 1e-3)[0][4]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-8 * max(1.0, abs(L)))


def test_zeroth_order_lipschitz_loss(setup):
    """L_LS,0 equals a double loop over the numpy oracle's cubature energies
    at the encoded samples, and its gradient (samples held fixed) central
    differences."""
    tp, theta, Q, Ws, bs = setup
    (Lc, L0, L), g, Z, _ = loss_and_grad(tp, theta, Q, 0.7, order=0)
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    tl, DmInv, cw = tp.ctets_local.numpy(), tp.cDmInv.numpy(), tp.cw.numpy()
    E = []
    for z in Z:
        xv = (tp.X0.ravel() + dec.out(z))[tp.rows].reshape(-1, 3)
        E.append(float(np.sum(cw * fem.element_energy(xv, tl, DmInv, np.ones(len(tl)), tp.mu,
                                                      tp.lam))))
    B = len(E)
    ref = sum((E[i] - E[j]) ** 2 / np.sum((Z[i] - Z[j]) ** 2)
              for i in range(B) for j in range(B) if i != j) / (B * (B - 1))
    assert L0 == pytest.approx(ref, rel=1e-10)
    assert L == pytest.approx(Lc + 0.7 * L0, rel=1e-14)
    rng = np.random.default_rng(102)
    for k in rng.choice(theta.size, 6, replace=False):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp_, tm_ = theta.copy(), theta.copy()
        tp_[k] += h
        tm_[k] -= h
        fd = (loss_and_grad(tp, tp_, Q, 0.7, Z_samples=Z, order=0)[0][2] -
              loss_and_grad(tp, tm_, Q, 0.7, Z_samples=Z, order=0)[0][2]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-8 * max(1.0, abs(L)))


def test_first_order_lipschitz_loss(setup):
    """L_LS,1 equals a double loop over the numpy oracle's reduced elastic
    gradients sum_e w_e J_e^T g_e at the encoded samples; its gradient
    (samples held fixed) central differences."""
    tp, theta, Q, Ws, bs = setup
    (Lc, L1, L), g, Z, _ = loss_and_grad(tp, theta, Q, 0.7, order=1)
    dec = Decoder([np.asarray(W, np.float64) for W in Ws], [np.asarray(b) for b in bs], tp.scale)
    tl, DmInv, cw = tp.ctets_local.numpy(), tp.cDmInv.numpy(), tp.cw.numpy()
    G = []
    for z in Z:
        o, J = dec.out_jac(z, tp.rows)
        xv = (tp.X0.ravel()[tp.rows] + o).reshape(-1, 3)
        ge = fem.element_gradient(xv, tl, DmInv, np.ones(len(tl)), tp.mu, tp.lam)
        G.append(np.einsum("e,eki,ek->i", cw, J[fem.element_dofs(tl)], ge))
    B = len(G)
    ref = sum(np.sum((G[i] - G[j]) ** 2) / np.sum((Z[i] - Z[j]) ** 2)
              for i in range(B) for j in range(B) if i != j) / (B * (B - 1))
    assert L1 == pytest.approx(ref, rel=1e-10)
    rng = np.random.default_rng(103)
    for k in rng.choice(theta.size, 6, replace=False):
        h = 1e-6 * max(1.0, abs(theta[k]))
        tp_, tm_ = theta.copy(), theta.copy()
        tp_[k] += h
        tm_[k] -= h
        fd = (loss_and_grad(tp, tp_, Q, 0.7, Z_samples=Z, order=1)[0][2] -
              loss_and_grad(tp, tm_, Q, 0.7, Z_samples=Z, order=1)[0][2]) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-5, abs=1e-8 * max(1.0, abs(L)))


def test_lipschitz_measures_of_a_linear_hessian_field():
    """For the Hessian field Ht(z) = z_0 A the Lipschitz constant of Eq. 7 is
    ||A||_F: every pair's ratio is at most that, and a pair that differs only
    in z_0 attains it (so its Eq. 9 term is ||A||_F^2)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4, 4))
    A = A + A.T
    nA = np.linalg.norm(A)
    Z = rng.standard_normal((5, 3))
    H = torch.tensor(Z[:, 0, None, None] * A)
    assert lipschitz_estimate(H, torch.tensor(Z)) <= nA * (1 + 1e-12)
    Z[1] = Z[0]
    Z[1, 0] += 0.7
    H = torch.tensor(Z[:, 0, None, None] * A)
    assert lipschitz_estimate(H, torch.tensor(Z)) == pytest.approx(nA, rel=1e-12)
    two = torch.tensor(Z[:2])
    assert float(lipschitz_loss(H[:2], two)) == pytest.approx(nA ** 2, rel=1e-12)


def test_repulsion_of_an_m_isometric_linear_decoder():
    """Eq. 4's repulsion term in closed form.  For a linear decoder
    x = X0 + s W z with W^T M W = c^2 I, every pair has
    ||x_i - x_j||_M = s c ||z_i - z_j||, so L_R = log(s c / sigma)^2, and it
    vanishes at sigma = s c."""
    from oracle.training import unsupervised_losses
    mesh = make_bar(5, 3, 3, 0.05)
    n, r = 3 * mesh.nv, 3
    cub = np.arange(6)
    tp = TrainProblem(mesh.X0, mesh.tets, [r, n], 0.05, 1e5, 0.45, 1000.0, cub, np.ones(6))
    m = np.repeat(tp.mass, 3)
    Qm, _ = np.linalg.qr(np.sqrt(m)[:, None] * np.random.default_rng(1).standard_normal((n, r)))
    c = 3.0
    W = c * Qm / np.sqrt(m)[:, None]                    # W^T M W = c^2 I
    assert np.allclose(W.T @ (m[:, None] * W), c * c * np.eye(r))
    theta = torch.tensor(tp.pack(np.zeros((r, n)), np.zeros(r), [W], [np.zeros(n)]))
    Z = torch.tensor(np.random.default_rng(2).standard_normal((5, r)))
    for sigma in (0.02, 0.05 * c, 1.0):
        _, Lr, _ = unsupervised_losses(tp, theta, Z, 0.1, sigma)
        assert float(Lr) == pytest.approx(np.log(0.05 * c / sigma) ** 2, rel=1e-10, abs=1e-20)
