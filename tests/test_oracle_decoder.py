"""Pins of the oracle's MLP subspace map and its forward-mode derivatives."""
import numpy as np
import pytest

from oracle.decoder import Decoder, elu, elu_d1, elu_d2
from workloads import xavier_decoder


@pytest.fixture(scope="module")
def dec():
    Ws, bs = xavier_decoder([5, 12, 12, 12, 30], seed=0)
    rng = np.random.default_rng(1)
    bs = [0.1 * rng.standard_normal(b.shape) for b in bs]
    return Decoder(Ws, bs, 1e-2)


def test_elu_derivatives_by_differences():
    a = np.linspace(-3, 3, 61)
    a = a[np.abs(a) > 1e-3]
    h = 1e-6
    assert np.allclose((elu(a + h) - elu(a - h)) / (2 * h), elu_d1(a), atol=1e-8)
    assert np.allclose((elu_d1(a + h) - elu_d1(a - h)) / (2 * h), elu_d2(a), atol=1e-7)
    assert elu(np.array([0.0]))[0] == 0.0 and elu_d1(np.array([0.0]))[0] == 1.0


def test_zero_bias_decoder_maps_origin_to_zero():
    Ws, bs = xavier_decoder([4, 16, 16, 30], seed=3)
    d = Decoder(Ws, bs, 1e-2)
    assert np.all(d.out(np.zeros(4)) == 0.0)


def test_jacobian_matches_central_differences(dec):
    rng = np.random.default_rng(2)
    z = rng.standard_normal(5)
    o, J = dec.out_jac(z)
    assert np.allclose(o, dec.out(z), atol=1e-15)
    h = 1e-6
    for k in range(5):
        e = np.zeros(5)
        e[k] = h
        fd = (dec.out(z + e) - dec.out(z - e)) / (2 * h)
        assert np.allclose(fd, J[:, k], rtol=1e-6, atol=1e-10)


def test_second_derivative_matches_differences_of_jacobian(dec):
    rng = np.random.default_rng(3)
    z = rng.standard_normal(5)
    o, J, D = dec.out_jac_hess(z)
    assert np.allclose(J, dec.out_jac(z)[1], atol=1e-15)
    assert np.allclose(D, np.swapaxes(D, 1, 2), atol=1e-15)
    h = 1e-6
    for k in range(5):
        e = np.zeros(5)
        e[k] = h
        fd = (dec.out_jac(z + e)[1] - dec.out_jac(z - e)[1]) / (2 * h)
        assert np.allclose(fd, D[:, :, k], rtol=1e-5, atol=1e-9)


def test_rows_subset(dec):
    z = np.random.default_rng(4).standard_normal(5)
    rows = np.array([0, 7, 29])
    o, J, D = dec.out_jac_hess(z, rows)
    oa, Ja, Da = dec.out_jac_hess(z)
    assert np.allclose(o, oa[rows]) and np.allclose(J, Ja[rows]) and np.allclose(D, Da[rows])


def test_single_layer_decoder_is_affine():
    rng = np.random.default_rng(5)
    W = rng.standard_normal((9, 3))
    b = rng.standard_normal(9)
    d = Decoder([W], [b], 0.5)
    z = rng.standard_normal(3)
    o, J, D = d.out_jac_hess(z)
    assert np.allclose(o, 0.5 * (W @ z + b)) and np.allclose(J, 0.5 * W)
    assert np.all(D == 0.0)
