"""Pins of the oracle's element quantities and assembly (Sec. 3.1)."""
import numpy as np
import pytest

from oracle import fem, snh
from workloads import make_bar

MU, LAM = snh.lame(1e5, 0.45)


@pytest.fixture(scope="module")
def bar():
    return make_bar(4, 3, 3, 0.05)


def test_volumes_sum_to_box_and_are_positive(bar):
    _, vol = fem.rest_shape(bar.X0, bar.tets)
    assert np.all(vol > 0)
    assert vol.sum() == pytest.approx(0.15 * 0.1 * 0.1, rel=1e-12)
    big = make_bar(20, 5, 5, 0.05)
    _, vb = fem.rest_shape(big.X0, big.tets)
    assert big.tets.shape[0] == 1824 and big.X0.shape[0] == 500
    assert vb.sum() == pytest.approx(0.95 * 0.2 * 0.2, rel=1e-12)


def test_lumped_mass_total(bar):
    _, vol = fem.rest_shape(bar.X0, bar.tets)
    m = fem.lumped_mass(bar.nv, bar.tets, vol, 1000.0)
    assert m.sum() == pytest.approx(1000.0 * 0.15 * 0.01, rel=1e-12)
    assert np.all(m > 0)


def test_affine_map_gives_constant_F(bar):
    rng = np.random.default_rng(0)
    A = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    x = bar.X0 @ A.T + np.array([0.3, -0.1, 2.0])
    DmInv, vol = fem.rest_shape(bar.X0, bar.tets)
    F = fem.deformation_gradient(x, bar.tets, DmInv)
    assert np.allclose(F, A[None], atol=1e-12)
    P = fem.element_energy(x, bar.tets, DmInv, vol, MU, LAM)
    assert P.sum() == pytest.approx(vol.sum() * snh.psi(A[None], MU, LAM)[0], rel=1e-10)


def test_rigid_motion_has_zero_energy_and_force(bar):
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    x = bar.X0 @ Q.T + 1.0
    DmInv, vol = fem.rest_shape(bar.X0, bar.tets)
    assert np.max(np.abs(fem.element_energy(x, bar.tets, DmInv, vol, MU, LAM))) < 1e-6
    assert np.max(np.abs(fem.element_gradient(x, bar.tets, DmInv, vol, MU, LAM))) < 1e-6


def _perturbed(bar, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    return bar.X0 + amp * rng.standard_normal(bar.X0.shape)


@pytest.mark.parametrize("ntet", [1, None])
def test_element_gradient_and_hessian_by_central_differences(bar, ntet):
    tets = bar.tets[:1] if ntet == 1 else bar.tets
    DmInv, vol = fem.rest_shape(bar.X0, tets)
    x = _perturbed(bar, 2, amp=0.012)
    g = fem.element_gradient(x, tets, DmInv, vol, MU, LAM)
    H = fem.element_hessian(x, tets, DmInv, vol, MU, LAM, project=False)
    h = 1e-7
    for e in range(min(tets.shape[0], 12)):
        for k in range(12):
            v, c = tets[e, k // 3], k % 3
            xp, xm = x.copy(), x.copy()
            xp[v, c] += h
            xm[v, c] -= h
            Pp = fem.element_energy(xp, tets[e:e + 1], DmInv[e:e + 1], vol[e:e + 1], MU, LAM)
            Pm = fem.element_energy(xm, tets[e:e + 1], DmInv[e:e + 1], vol[e:e + 1], MU, LAM)
            assert (Pp - Pm)[0] / (2 * h) == pytest.approx(g[e, k], rel=1e-5, abs=1e-4)
            gp = fem.element_gradient(xp, tets[e:e + 1], DmInv[e:e + 1], vol[e:e + 1], MU, LAM)
            gm = fem.element_gradient(xm, tets[e:e + 1], DmInv[e:e + 1], vol[e:e + 1], MU, LAM)
            assert np.allclose((gp - gm)[0] / (2 * h), H[e, :, k], rtol=1e-5, atol=1e-1)


def test_projected_hessian_is_psd_and_unchanged_near_rest(bar):
    DmInv, vol = fem.rest_shape(bar.X0, bar.tets)
    x_far = _perturbed(bar, 3, amp=0.03)
    Hp = fem.element_hessian(x_far, bar.tets, DmInv, vol, MU, LAM, project=True)
    assert np.min(np.linalg.eigvalsh(Hp)) > -1e-6 * np.max(np.abs(Hp))
    # uniform stretch by 5%: the density Hessian is positive definite there
    # (checked), so projection must leave the element Hessians unchanged
    A = 1.05 * np.eye(3)
    assert np.min(np.linalg.eigvalsh(snh.d2psi_dF2(A[None], MU, LAM)[0])) > 0
    x_s = bar.X0 @ A.T
    Hn = fem.element_hessian(x_s, bar.tets, DmInv, vol, MU, LAM, project=True)
    Hu = fem.element_hessian(x_s, bar.tets, DmInv, vol, MU, LAM, project=False)
    assert np.allclose(Hn, Hu, rtol=1e-9, atol=1e-9 * np.max(np.abs(Hu)))


def test_assembly_matches_element_sums(bar):
    DmInv, vol = fem.rest_shape(bar.X0, bar.tets)
    x = _perturbed(bar, 5)
    w = np.random.default_rng(6).uniform(0.5, 2.0, bar.ne)
    ge = fem.element_gradient(x, bar.tets, DmInv, vol, MU, LAM)
    He = fem.element_hessian(x, bar.tets, DmInv, vol, MU, LAM)
    g = fem.assemble_gradient(ge, bar.tets, 3 * bar.nv, w)
    H = fem.assemble_hessian(He, bar.tets, 3 * bar.nv, w).toarray()
    # brute force: loop over elements and local DOFs
    g_ref = np.zeros(3 * bar.nv)
    H_ref = np.zeros((3 * bar.nv, 3 * bar.nv))
    for e in range(bar.ne):
        d = [3 * bar.tets[e, a] + c for a in range(4) for c in range(3)]
        for i in range(12):
            g_ref[d[i]] += w[e] * ge[e, i]
            for j in range(12):
                H_ref[d[i], d[j]] += w[e] * He[e, i, j]
    assert np.allclose(g, g_ref, atol=1e-12)
    assert np.allclose(H, H_ref, atol=1e-9)
