"""Pins of the oracle's optimised cubature selection (Sec. 4.3, after von
Tycowicz et al. 2013): the force matrix against the assembled model, and the
active-set NNLS against facts that do not depend on its code."""
import numpy as np
import pytest

from oracle.cubature_fit import (tet_force_matrix, normalise_blocks, nnls_active_set,
                                 select_cubature)
from oracle.decoder import Decoder
from oracle.reduced import ReducedModel
from workloads import make_bar, face_nodes, xavier_decoder


def _model():
    mesh = make_bar(6, 3, 3, 0.05)
    n = 3 * mesh.nv
    Ws, bs = xavier_decoder([4, 16, 16, n], 0)
    return ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0,
                        (0.0, 0.0, 0.0), cnodes=face_nodes(mesh, 0))


def test_columns_sum_to_the_assembled_elastic_gradient():
    """sum_e a_e(z) = J(z)^T dP/dx (no gravity, no inertia: the reduced
    gradient of the assembled elastic potential)."""
    m = _model()
    Z = np.random.default_rng(1).standard_normal((3, 4)) * 0.5
    A = tet_force_matrix(m, Z)
    for k in range(3):
        x, J = m.positions_jac(Z[k])
        g = J.T @ m.full_gradient_x(x)
        assert np.allclose(A[4 * k:4 * k + 4].sum(axis=1), g, rtol=1e-10, atol=1e-12)


def test_sparse_nonnegative_solution_is_recovered():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((60, 40))
    x = np.zeros(40)
    x[[3, 11, 17, 29, 36]] = rng.uniform(0.5, 2.0, 5)
    idx, w, rel = nnls_active_set(A, A @ x, S=40)
    assert rel < 1e-12
    assert sorted(idx.tolist()) == [3, 11, 17, 29, 36]
    assert np.allclose(w[np.argsort(idx)], x[[3, 11, 17, 29, 36]], rtol=1e-10)


def test_full_run_meets_kkt_and_scipy_residual():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(3)
    A = rng.standard_normal((50, 30))
    b = rng.standard_normal(50)
    idx, w, rel = nnls_active_set(A, b)
    x = np.zeros(30)
    x[idx] = w
    grad = A.T @ (b - A @ x)
    assert np.all(w > 0)
    assert np.all(grad <= 1e-9)                      # no improving direction
    assert np.allclose(grad[idx], 0.0, atol=1e-9)    # stationary on the active set
    xs, rs = scipy_opt.nnls(A, b)
    assert rel * np.linalg.norm(b) == pytest.approx(rs, rel=1e-9)


def test_residual_does_not_grow_with_the_cubature_count():
    m = _model()
    Z = np.random.default_rng(4).standard_normal((6, 4)) * 0.5
    A, b = normalise_blocks(tet_force_matrix(m, Z), 4)
    rels = [nnls_active_set(A, b, S)[2] for S in (2, 4, 8, 16)]
    assert all(r2 <= r1 + 1e-12 for r1, r2 in zip(rels, rels[1:]))
    idx, w, rel = select_cubature(m, Z, 16)
    assert len(idx) <= 16 and np.all(w > 0) and rel == pytest.approx(rels[-1])
