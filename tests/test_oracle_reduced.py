"""Pins of the oracle's reduced objective (Eq. 2), its Eq. 11-form gradient,
the Gauss-Newton reduced Hessian and the Newton / Armijo solve."""
import numpy as np
import pytest

from oracle import fem
from oracle.decoder import Decoder
from oracle.fullspace import FullModel
from oracle.reduced import (ReducedModel, ReducedSimulator, newton_solve,
                            cholesky_direction, model_from_problem, CONVERGED)
from workloads import build_problem, make_bar, face_nodes, xavier_decoder

G = (0.0, 0.0, -9.8)


def tiny_model(dyn, seed=0, cub=False, gravity=G):
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([4, 16, 16, n], seed)
    dec = Decoder(Ws, bs, 1e-2)
    idx = w = None
    if cub:
        rng = np.random.default_rng(7)
        idx = np.sort(rng.choice(mesh.ne, 20, replace=False))
        w = rng.uniform(0.5, 3.0, 20)
    m = ReducedModel(mesh.X0, mesh.tets, dec, 1e5, 0.45, 1000.0, gravity,
                     idx, w, face_nodes(mesh, 0))
    if dyn:
        rng = np.random.default_rng(8)
        m.set_dynamics(1 / 60, mesh.X0.ravel() + 1e-3 * rng.standard_normal(n))
    return m


@pytest.mark.parametrize("dyn,cub", [(False, False), (True, False), (True, True)])
def test_reduced_gradient_is_J_transpose_full_gradient(dyn, cub):
    m = tiny_model(dyn, cub=cub)
    z = np.random.default_rng(1).standard_normal(4) * 0.5
    E, g, K = m.eval(z)
    x, J = m.positions_jac(z)
    assert np.allclose(g, J.T @ m.full_gradient_x(x), rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("dyn,cub", [(False, False), (True, True)])
def test_reduced_hessian_is_J_transpose_assembled_J(dyn, cub):
    m = tiny_model(dyn, cub=cub)
    z = np.random.default_rng(2).standard_normal(4) * 0.5
    _, _, K = m.eval(z)
    x, J = m.positions_jac(z)
    He = fem.element_hessian(x.reshape(-1, 3), m.tets, m.DmInv, m.vol, m.mu, m.lam)
    H = fem.assemble_hessian(He, m.tets, m.n, m.w).toarray()
    if dyn:
        H += np.diag(np.repeat(m.mass, 3)) / m.dt ** 2
    assert np.allclose(K, J.T @ H @ J, rtol=1e-10, atol=1e-8)


@pytest.mark.parametrize("dyn", [False, True])
def test_gradient_matches_central_differences_of_energy(dyn):
    m = tiny_model(dyn)
    z = np.random.default_rng(3).standard_normal(4) * 0.5
    _, g, _ = m.eval(z)
    h = 1e-6
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        fd = (m.energy(z + e) - m.energy(z - e)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-8)


def test_rest_state_without_load_is_stationary():
    m = tiny_model(False, gravity=(0.0, 0.0, 0.0))
    E, g, _ = m.eval(np.zeros(4))
    assert abs(E) < 1e-10 and np.max(np.abs(g)) < 1e-10
    z, st = newton_solve(m, np.zeros(4), 1e-10)
    assert st.status == CONVERGED and st.newton_iters == 0


def test_linear_decoder_matches_independent_linear_subspace_newton():
    """x = X0 + U z: the reduced solve equals a Newton solve written here from
    the assembled full-space gradient and Hessian projected onto U."""
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    rng = np.random.default_rng(4)
    U = 1e-2 * rng.standard_normal((n, 5))
    cn = face_nodes(mesh, 0)
    cd = (3 * cn[:, None] + np.arange(3)).ravel()
    m = ReducedModel(mesh.X0, mesh.tets, Decoder([U], [np.zeros(n)], 1.0),
                     1e5, 0.45, 1000.0, G, None, None, cn)
    z_red, st = newton_solve(m, np.zeros(5), 1e-10)
    assert st.status == CONVERGED
    fm = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, G, cn)
    Uc = U.copy()
    Uc[cd] = 0.0
    z = np.zeros(5)
    for _ in range(50):
        q = mesh.X0.ravel() + Uc @ z
        g = Uc.T @ fm.gradient(q)
        if np.max(np.abs(g)) < 1e-10:
            break
        K = Uc.T @ (fm.hessian(q) @ Uc)
        d = -np.linalg.solve(K, g)
        a = 1.0
        while fm.energy(mesh.X0.ravel() + Uc @ (z + a * d)) > fm.energy(q) + 1e-4 * a * (g @ d):
            a *= 0.5
        z = z + a * d
    assert np.allclose(z_red, z, rtol=1e-8, atol=1e-10)


def test_linear_decoder_minimiser_matches_torch_transcription():
    """x = X0 + U z: the reduced solve's end point minimises an independent
    torch transcription of the Eq. 2 objective at dt = 0 (stable neo-Hookean
    density of the deformation gradient times rest volume, minus the work of
    gravity on lumped masses), minimised here by autodiff Newton.  Shares no
    code with the oracle's fem module, which the test above relies on."""
    import torch
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    rng = np.random.default_rng(4)
    U = 1e-2 * rng.standard_normal((n, 5))
    cn = face_nodes(mesh, 0)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder([U], [np.zeros(n)], 1.0),
                     1e5, 0.45, 1000.0, G, None, None, cn)
    z_red, st = newton_solve(m, np.zeros(5), 1e-10)
    assert st.status == CONVERGED

    youngs, nu, rho = 1e5, 0.45, 1000.0
    mu = youngs / (2.0 * (1.0 + nu))
    lam = youngs * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    alpha = 1.0 + 0.75 * mu / lam
    X = torch.tensor(mesh.X0, dtype=torch.float64)
    T = torch.tensor(np.asarray(mesh.tets), dtype=torch.long)

    def edge_matrix(P):  # columns P_a - P_0, a = 1..3, per tet
        return torch.stack([P[T[:, a]] - P[T[:, 0]] for a in (1, 2, 3)], dim=2)

    Dm = edge_matrix(X)
    vol = torch.abs(torch.linalg.det(Dm)) / 6.0
    Dm_inv = torch.linalg.inv(Dm)
    mass = torch.zeros(mesh.nv, dtype=torch.float64)
    for a in range(4):  # a quarter of each tet's mass on each of its vertices
        mass.index_add_(0, T[:, a], rho * vol / 4.0)
    keep = torch.ones(n, dtype=torch.float64)
    keep[torch.tensor((3 * cn[:, None] + np.arange(3)).ravel())] = 0.0  # clamped face
    Ut = torch.tensor(U) * keep[:, None]
    grav = torch.tensor(G, dtype=torch.float64)

    def energy(z):
        x = X + (Ut @ z).reshape(-1, 3)
        F = edge_matrix(x) @ Dm_inv
        Ic = (F * F).sum(dim=(1, 2))
        psi = (0.5 * mu * (Ic - 3.0) + 0.5 * lam * (torch.linalg.det(F) - alpha) ** 2
               - 0.5 * mu * torch.log(Ic + 1.0))
        return (vol * psi).sum() - (mass[:, None] * grav[None, :] * x).sum()

    z = torch.zeros(5, dtype=torch.float64)
    for _ in range(60):
        gz = torch.autograd.functional.jacobian(energy, z)
        if gz.abs().max() < 1e-10:
            break
        H = torch.autograd.functional.hessian(energy, z)
        w, V = torch.linalg.eigh(H)
        w = torch.clamp(w, min=1e-8 * w.abs().max())
        d = -(V @ ((V.T @ gz) / w))
        step, e0 = 1.0, energy(z)
        while energy(z + step * d) > e0 + 1e-4 * step * (gz @ d):
            step *= 0.5
        z = z + step * d
    assert gz.abs().max() < 1e-10
    assert np.allclose(z_red, z.numpy(), rtol=1e-8, atol=1e-10), (z_red, z.numpy())


def test_linear_decoder_with_quadratic_energy_converges_in_one_step():
    """Only the inertia term (all cubature weights zero): E is quadratic in z,
    Newton lands on the weighted least-squares solution in one step."""
    mesh = make_bar(5, 3, 3, 0.05)
    n = 3 * mesh.nv
    rng = np.random.default_rng(5)
    U = rng.standard_normal((n, 6))
    b = rng.standard_normal(n)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder([U], [b], 1e-2), 1e5, 0.45,
                     1000.0, G, np.arange(mesh.ne), np.zeros(mesh.ne), None)
    qbar = mesh.X0.ravel() + 0.01 * rng.standard_normal(n)
    m.set_dynamics(0.01, qbar)
    z, st = newton_solve(m, np.zeros(6), 1e-9)
    assert st.status == CONVERGED and st.newton_iters == 1
    W = np.repeat(m.mass, 3)
    A = 1e-2 * U
    rhs = qbar - mesh.X0.ravel() - 1e-2 * b
    z_ls = np.linalg.solve(A.T @ (W[:, None] * A), A.T @ (W * rhs))
    assert np.allclose(z, z_ls, rtol=1e-9, atol=1e-12)


def test_cholesky_shift_gives_descent_direction():
    K = np.diag([1.0, 2.0, -1e-3])
    g = np.array([1.0, -1.0, 0.5])
    d, ok = cholesky_direction(K, g)
    assert ok and g @ d < 0


def test_quasistatic_bar_solve_converges():
    p = build_problem("tiny_quasistatic")
    m = model_from_problem(p)
    sim = ReducedSimulator(m, 0.0, eps=p.config.eps)
    st = sim.step(p.targets(1))
    assert st.status == CONVERGED
    assert np.max(np.abs(m.eval(sim.z)[1])) < p.config.eps
    # gravity pulls the free end down
    assert (sim.q.reshape(-1, 3)[:, 2] - p.X0[:, 2]).mean() < 0


def test_ground_penalty_closed_form_under_rigid_translation():
    """x = X0 + z e_z (one linear layer, a rigid vertical translation: no
    elastic energy, no gravity): E = k/2 N_below (z - h)^2, g = k N_below
    (z - h), K = k N_below, with N_below the bottom layer of nodes (z = 0)
    when 0 < h - z < 0.05."""
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    W = np.zeros((n, 1), np.float32)
    W[2::3, 0] = 100.0                       # output scale 1e-2: dx_z/dz = 1
    dec = Decoder([W], [np.zeros(n, np.float32)], 1e-2)
    m = ReducedModel(mesh.X0, mesh.tets, dec, 1e5, 0.45, 1000.0, (0.0, 0.0, 0.0))
    k, h, z = 3e4, 0.01, -0.025
    m.set_ground(h, k)
    nb = int(np.sum(mesh.X0[:, 2] == 0.0))
    assert nb == 6 * 3
    E, g, K = m.eval(np.array([z]))
    pen = z - h
    assert E == pytest.approx(0.5 * k * nb * pen ** 2, rel=1e-12)
    assert g[0] == pytest.approx(k * nb * pen, rel=1e-12)
    assert K[0, 0] == pytest.approx(k * nb, rel=1e-12)
    # above the plane the penalty vanishes
    E0, g0, K0 = m.eval(np.array([0.02]))
    assert E0 == pytest.approx(0.0, abs=1e-12) and abs(g0[0]) < 1e-9 and K0[0, 0] < 1e-6


@pytest.mark.parametrize("dyn", [False, True])
def test_gradient_with_ground_contact_matches_central_differences(dyn):
    m = tiny_model(dyn)
    m.set_ground(0.06, 2e4)                  # a plane through the bar's second node layer
    z = np.random.default_rng(4).standard_normal(4) * 0.5
    E, g, _ = m.eval(z)
    assert m._ground(m.positions(z))[0] > 0.0
    h = 1e-6
    for k in range(4):
        e = np.zeros(4)
        e[k] = h
        fd = (m.energy(z + e) - m.energy(z - e)) / (2 * h)
        assert fd == pytest.approx(g[k], rel=1e-6, abs=1e-8)


def _affine_model(zero_network, gravity=(0.0, 0.0, 0.0), seed=0):
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([4, 16, 16, n], seed)
    if zero_network:
        Ws[-1] = np.zeros_like(Ws[-1])
    c = mesh.X0.mean(0)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0, gravity,
                     affine_center=c)
    return m, mesh, c


def test_affine_modes_map_closed_form():
    """Network output zero: z_aff = (M, t) moves every vertex to
    X0 + s (M (X0 - c) + t) (s = 1e-2, the output scale), so every tet has
    F = I + s M and the elastic energy is V_total Psi(I + s M); a pure
    translation costs nothing."""
    from oracle import snh
    m, mesh, c = _affine_model(True)
    assert m.r == 4 + 12
    rng = np.random.default_rng(3)
    M = 5.0 * rng.standard_normal((3, 3))
    t = rng.standard_normal(3)
    z = np.concatenate([rng.standard_normal(4), M.ravel(), t])
    x = m.positions(z).reshape(-1, 3)
    assert np.allclose(x, mesh.X0 + 1e-2 * ((mesh.X0 - c) @ M.T + t), rtol=0, atol=1e-14)
    mu, lam = snh.lame(1e5, 0.45)
    vol = fem.rest_shape(mesh.X0, mesh.tets)[1]
    psi = float(snh.psi(np.eye(3) + 1e-2 * M, mu, lam))
    assert m.energy(z) == pytest.approx(vol.sum() * psi, rel=1e-10)
    zt = np.concatenate([np.zeros(4 + 9), t])
    assert abs(m.energy(zt)) < 1e-9


def test_affine_jacobian_columns_match_central_differences():
    m, _, _ = _affine_model(False)
    z = np.random.default_rng(5).standard_normal(16) * 0.3
    _, J = m.positions_jac(z)
    h = 1e-6
    for k in range(16):
        e = np.zeros(16)
        e[k] = h
        fd = (m.positions(z + e) - m.positions(z - e)) / (2 * h)
        assert np.allclose(J[:, k], fd, rtol=1e-6, atol=1e-9), k


def test_affine_free_fall_is_exact_projectile_motion():
    """Network output zero, no contact: one implicit-Euler step from rest with
    a uniform initial velocity v0 lands on x = X0 + dt v0 + dt^2 g (the
    inertial guess is reachable at zero elastic energy), and v becomes
    v0 + dt g."""
    g = np.array([0.0, 0.0, -9.8])
    m, mesh, _ = _affine_model(True, gravity=tuple(g))
    v0 = np.tile([0.3, -0.2, 0.5], mesh.nv)
    dt = 0.01
    sim = ReducedSimulator(m, dt, eps=1e-10, v0=v0)
    st = sim.step(np.zeros((0, 3)))
    assert st.status == CONVERGED
    assert np.allclose(sim.q, mesh.X0.ravel() + dt * v0 + dt * dt * np.tile(g, mesh.nv),
                       rtol=0, atol=1e-11)
    assert np.allclose(sim.v, v0 + dt * np.tile(g, mesh.nv), rtol=0, atol=1e-9)


def test_worker_pool_gives_the_serial_sums_exactly():
    """The chunked element sums evaluated in worker processes are the serial
    loop's, bit for bit (same chunks, added in the same order)."""
    from oracle.pool import ElementPool
    from oracle.reduced import model_from_problem
    from workloads import build_problem
    p = build_problem("small_dyn_full")
    m = model_from_problem(p, chunk=96)
    m.set_targets(p.targets(2))
    m.set_dynamics(p.config.dt, p.X0.ravel() + 1e-3)
    z = np.random.default_rng(5).standard_normal(m.r) * 0.5
    E0, g0, K0 = m.eval(z)
    pool = ElementPool(m, workers=2)
    try:
        m.pool = pool
        E1, g1, K1 = m.eval(z)
    finally:
        m.pool = None
        pool.close()
    assert E0 == E1
    assert np.array_equal(g0, g1) and np.array_equal(K0, K1)


def _fd_hessian(m, z, h=1e-5):
    """Central differences of the reduced gradient g(z)."""
    r = z.shape[0]
    Hfd = np.zeros((r, r))
    for k in range(r):
        e = np.zeros(r)
        e[k] = h
        Hfd[:, k] = (m.energy_grad(z + e)[1] - m.energy_grad(z - e)[1]) / (2 * h)
    return 0.5 * (Hfd + Hfd.T)


@pytest.mark.parametrize("dyn,cub", [(False, False), (True, False), (True, True)])
def test_exact_hessian_matches_central_differences_of_gradient(dyn, cub):
    """With unprojected element Hessians, K + sum_k dE/dx_k d2x_k/dz2 (before
    the r x r projection) is the Hessian of E(z): it equals central
    differences of the reduced gradient, which the Gauss-Newton K alone
    misses by far more."""
    m = tiny_model(dyn, cub=cub)
    z = np.random.default_rng(4).standard_normal(4) * 0.8
    Hfd = _fd_hessian(m, z)
    _, _, Kx = m.eval_exact(z, project=False)
    _, _, Kgn = m.eval(z, project=False)
    scale = np.abs(Hfd).max()
    assert np.abs(Kx - Hfd).max() < 1e-6 * scale
    assert np.abs(Kgn - Hfd).max() > 1e3 * np.abs(Kx - Hfd).max()


def test_exact_hessian_with_affine_modes_matches_central_differences():
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([4, 16, 16, n], 5)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0, G,
                     affine_center=mesh.X0.mean(0))
    rng = np.random.default_rng(9)
    m.set_dynamics(1 / 60, mesh.X0.ravel() + 1e-3 * rng.standard_normal(n))
    z = rng.standard_normal(16) * 0.5
    Hfd = _fd_hessian(m, z)
    _, _, Kx = m.eval_exact(z, project=False)
    assert np.abs(Kx - Hfd).max() < 1e-6 * np.abs(Hfd).max()
    assert np.all(m.curvature_term(z)[4:, :] == 0.0) and np.all(m.curvature_term(z)[:, 4:] == 0.0)


def test_curvature_term_vanishes_for_a_linear_decoder():
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([4, n], 2)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0, G,
                     cnodes=face_nodes(mesh, 0))
    m.set_dynamics(1 / 60, mesh.X0.ravel())
    z = np.random.default_rng(3).standard_normal(4)
    assert np.all(m.curvature_term(z) == 0.0)
    _, _, K = m.eval(z)
    _, _, Kx = m.eval_exact(z)
    assert np.allclose(Kx, K, rtol=1e-12, atol=1e-12 * np.abs(K).max())


def test_exact_hessian_projection():
    """The r x r projection: eigenvalues at least clamp * max |eigenvalue|;
    with clamp = 0 the closest PSD matrix in the Frobenius norm (the
    eigen-clamp, checked against a brute-force search over PSD candidates
    along the clamped directions); a matrix that is already positive definite
    is left alone."""
    from oracle.snh import project_psd
    m = tiny_model(False)
    z = np.random.default_rng(6).standard_normal(4) * 1.5
    _, _, Kraw = m.eval_exact(z, project=False)
    Kraw_p = m.eval(z)[2] + m.curvature_term(z)
    Kraw_p = 0.5 * (Kraw_p + Kraw_p.T)
    lam_ = np.linalg.eigvalsh(Kraw_p)
    _, _, Kx = m.eval_exact(z, clamp=1e-3)
    assert np.linalg.eigvalsh(Kx).min() >= 1e-3 * np.abs(lam_).max() * (1 - 1e-9)
    _, _, K0 = m.eval_exact(z, clamp=0.0)
    assert np.allclose(K0, project_psd(Kraw_p), atol=1e-10 * np.abs(lam_).max())
    # a positive definite sum is kept as it is
    A = Kraw_p + (1.0 - lam_.min()) * np.eye(4)
    w, Q = np.linalg.eigh(A)
    assert np.allclose((Q * np.maximum(w, 1e-10 * np.abs(w).max())) @ Q.T, A)
    if lam_.min() < 0:   # the clamp moved something: distances to PSD matrices are larger
        d0 = np.linalg.norm(K0 - Kraw_p)
        rng = np.random.default_rng(0)
        for _ in range(50):
            B = rng.standard_normal((4, 4))
            C = K0 + 1e-2 * np.abs(lam_).max() * (B @ B.T) / np.linalg.norm(B @ B.T)
            assert np.linalg.norm(C - Kraw_p) >= d0 - 1e-12


def test_exact_newton_reaches_the_same_minimiser():
    """Newton with the exact-form Hessian converges to the minimiser the
    Gauss-Newton solve finds, from the same start."""
    m = tiny_model(True)
    z0 = np.zeros(4)
    zg, sg = newton_solve(m, z0, 1e-8)
    zx, sx = newton_solve(m, z0, 1e-8, exact=True)
    assert sg.status == CONVERGED and sx.status == CONVERGED
    assert np.allclose(zx, zg, atol=1e-6)
