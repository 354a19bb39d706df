"""Pins of the oracle's Stable Neo-Hookean model (Sec. 5.1) and of the PSD
projection used by projective Newton (Supplement)."""
import numpy as np
import pytest
import torch

from oracle import snh

MU, LAM = snh.lame(1e5, 0.45)


def rand_F(rng, n, scale=0.3, inverted=False):
    F = np.eye(3) + scale * rng.standard_normal((n, 3, 3))
    if inverted:
        F[:, :, 0] *= -1.0
    return F


def rand_rot(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, 3, 3)))
    Q = Q * np.sign(np.diagonal(R, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1.0
    return Q


def test_lame_values():
    # E = 1e5, nu = 0.45: mu = E / 2.9, lam = 0.45 E / (1.45 * 0.1)
    assert MU == pytest.approx(1e5 / 2.9, rel=1e-15)
    assert LAM == pytest.approx(0.45e5 / 0.145, rel=1e-15)


def test_rest_energy_and_stress_vanish():
    I = np.eye(3)[None]
    assert abs(snh.psi(I, MU, LAM)[0]) < 1e-9
    assert np.max(np.abs(snh.dpsi_dF(I, MU, LAM))) < 1e-9


def test_cofactor_is_det_times_inverse_transpose():
    rng = np.random.default_rng(0)
    F = rand_F(rng, 20, inverted=True)
    ref = np.linalg.det(F)[:, None, None] * np.swapaxes(np.linalg.inv(F), 1, 2)
    assert np.allclose(snh.cofactor(F), ref, rtol=1e-12, atol=1e-12)


def test_rotation_and_isotropy_invariance():
    rng = np.random.default_rng(1)
    F = rand_F(rng, 50, scale=0.5)
    R1, R2 = rand_rot(rng, 50), rand_rot(rng, 50)
    p = snh.psi(F, MU, LAM)
    assert np.allclose(snh.psi(R1 @ F, MU, LAM), p, rtol=1e-10, atol=1e-6)
    assert np.allclose(snh.psi(F @ R2, MU, LAM), p, rtol=1e-10, atol=1e-6)


@pytest.mark.parametrize("inverted", [False, True])
def test_first_derivative_matches_central_differences(inverted):
    rng = np.random.default_rng(2)
    F = rand_F(rng, 10, inverted=inverted)
    P = snh.dpsi_dF(F, MU, LAM)
    h = 1e-6
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3))
            E[i, j] = h
            fd = (snh.psi(F + E, MU, LAM) - snh.psi(F - E, MU, LAM)) / (2 * h)
            assert np.allclose(fd, P[:, i, j], rtol=1e-6, atol=1e-3)


@pytest.mark.parametrize("inverted", [False, True])
def test_second_derivative_matches_central_differences(inverted):
    rng = np.random.default_rng(3)
    F = rand_F(rng, 10, inverted=inverted)
    H = snh.d2psi_dF2(F, MU, LAM)
    h = 1e-6
    for k in range(9):
        E = np.zeros(9)
        E[k] = h
        E = E.reshape(3, 3)
        fd = (snh.dpsi_dF(F + E, MU, LAM) - snh.dpsi_dF(F - E, MU, LAM)) / (2 * h)
        assert np.allclose(fd.reshape(-1, 9), H[:, :, k], rtol=1e-6, atol=1e-2)


def test_rest_hessian_hand_derived_closed_form():
    # At F = I: I_C = 3, J = 1, cof = I, d2J/dF_ij dF_kl = d_ij d_kl - d_il d_kj,
    # lam (1 - a) = -3 mu / 4.  Collecting terms gives
    #   (3 mu / 4)(Id + T) + (lam - 5 mu / 8) v v^T,  v = vec(I), T = transpose map.
    v = np.eye(3).ravel()
    T = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            T[3 * i + j, 3 * j + i] = 1.0
    ref = 0.75 * MU * (np.eye(9) + T) + (LAM - 0.625 * MU) * np.outer(v, v)
    H = snh.d2psi_dF2(np.eye(3)[None], MU, LAM)[0]
    assert np.allclose(H, ref, rtol=1e-12, atol=1e-6)


def test_derivatives_match_float64_autodiff():
    # an independent torch transcription of the density, differentiated by
    # autodiff, against the closed-form first and second derivatives
    rng = np.random.default_rng(4)
    a = 1.0 + 3.0 * MU / (4.0 * LAM)
    p0 = 0.5 * LAM * (1 - a) ** 2 - MU * np.log(2.0)

    def psi_t(f):
        F = f.reshape(3, 3)
        Ic = (F * F).sum()
        return (0.5 * MU * (Ic - 3) + 0.5 * LAM * (torch.linalg.det(F) - a) ** 2
                - 0.5 * MU * torch.log(Ic + 1) - p0)

    for F in rand_F(rng, 5, scale=0.4):
        f = torch.tensor(F.ravel(), dtype=torch.float64, requires_grad=True)
        g = torch.autograd.grad(psi_t(f), f)[0].numpy()
        H = torch.autograd.functional.hessian(psi_t, f.detach()).numpy()
        assert np.allclose(g, snh.dpsi_dF(F[None], MU, LAM)[0].ravel(), rtol=1e-10)
        assert np.allclose(H, snh.d2psi_dF2(F[None], MU, LAM)[0], rtol=1e-9, atol=1e-6)


def test_projection_characterisation():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 9, 9))
    A = A + np.swapaxes(A, 1, 2)
    P = snh.project_psd(A)
    # P >= 0, A - P <= 0, complementary slackness P (A - P) = 0
    assert np.min(np.linalg.eigvalsh(P)) > -1e-12
    assert np.max(np.linalg.eigvalsh(A - P)) < 1e-12
    assert np.max(np.abs(P @ (A - P))) < 1e-10


def test_projection_keeps_psd_and_clamps_diagonal():
    rng = np.random.default_rng(6)
    B = rng.standard_normal((5, 9, 9))
    S = B @ np.swapaxes(B, 1, 2)
    assert np.allclose(snh.project_psd(S), S, atol=1e-12)
    D = np.diag([3.0, -1.0, 0.5, -2.0, 0.0, 1.0, -0.1, 4.0, 2.0])
    assert np.allclose(snh.project_psd(D[None])[0], np.diag(np.maximum(np.diag(D), 0)))
