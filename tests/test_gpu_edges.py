"""GPU edge cases and argument checks of the C ABI."""
import numpy as np
import pytest

from oracle.decoder import Decoder
from oracle.reduced import ReducedModel
from workloads import make_bar, face_nodes, xavier_decoder
from tests.gpu_util import rel, assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_03807_gb300.build import build
    build()
    import paper_2409_03807_gb300 as pkg
    pkg.load()
    return pkg


def _setup(pkg, mesh, widths, prec, cub=None, cn=None, seed=0):
    Ws, bs = xavier_decoder(widths, seed)
    ctx = pkg.Context()
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0.0, 0.0, -9.8))
    if cub is not None:
        ctx.set_cubature(*cub)
    if cn is not None:
        ctx.set_constraints(cn, mesh.X0[cn])
    ctx.set_decoder(Ws, bs, 1e-2, prec)
    ctx.set_solver(1e-6)
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Ws, bs, 1e-2), 1e5, 0.45, 1000.0,
                     (0.0, 0.0, -9.8), None if cub is None else cub[0],
                     None if cub is None else cub[1], cn)
    return ctx, m


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_tet_and_r1(pkg, prec):
    X0 = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0.1]], float)
    mesh = type("M", (), {"X0": X0, "tets": np.array([[0, 1, 2, 3]], np.int32)})
    ctx, m = _setup(pkg, mesh, [1, 5, 12], prec, cn=np.array([0], np.int32))
    z = np.array([0.8])
    E, g, K = ctx.eval(z)
    E0, g0, K0 = m.eval(z)
    tol = 1e-10 if prec == "fp64" else 1e-4
    assert abs(E - E0) <= tol * max(1, abs(E0)) and rel(g, g0) < tol * 10 and rel(K, K0) < tol
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ragged_tiles_single_cubature_tet_and_no_constraints(pkg, prec):
    # 5x4x3 nodes: 144 tets (one full element tile + ragged), n = 180 rows
    mesh = make_bar(5, 4, 3, 0.05)
    for cub in [(np.array([7], np.int32), np.array([3.5])),
                (np.arange(0, mesh.ne, 2, dtype=np.int32), np.full((mesh.ne + 1) // 2, 2.0))]:
        ctx, m = _setup(pkg, mesh, [7, 13, 3 * mesh.nv], prec, cub=cub)
        m.set_dynamics(0.02, mesh.X0.ravel() + 1e-3)
        ctx.set_dynamics(0.02, mesh.X0.ravel() + 1e-3)
        z = np.random.default_rng(3).standard_normal(7)
        E, g, K = ctx.eval(z)
        E0, g0, K0 = m.eval(z)
        tol = 1e-10 if prec == "fp64" else 1e-4
        assert abs(E - E0) <= tol * max(1, abs(E0))
        assert_close(g, g0, tol * 10)
        assert_close(K, K0, tol)
        ctx.close()


def test_max_subspace_dimension(pkg):
    mesh = make_bar(6, 3, 3, 0.05)
    ctx, m = _setup(pkg, mesh, [64, 40, 3 * mesh.nv], "fp64",
                    cn=face_nodes(mesh, 0))
    z = 0.1 * np.random.default_rng(4).standard_normal(64)
    E, g, K = ctx.eval(z)
    E0, g0, K0 = m.eval(z)
    assert abs(E - E0) < 1e-10 * abs(E0) and rel(g, g0) < 1e-9 and rel(K, K0) < 1e-9
    ctx.close()


def test_argument_errors(pkg):
    ctx = pkg.Context()
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_material(1e5, 0.45, 1000.0, (0, 0, -9.8))
    assert e.value.code == -4
    mesh = make_bar(3, 2, 2, 0.05)
    bad = mesh.tets.copy()
    bad[0, [1, 2]] = bad[0, [2, 1]]            # inverted rest tet
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_mesh(mesh.X0, bad)
    assert e.value.code == -1
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0, 0, -9.8))
    Ws, bs = xavier_decoder([65, 4, 3 * mesh.nv], 0)
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_decoder(Ws, bs, 1e-2)
    assert e.value.code == -1
    Ws, bs = xavier_decoder([4, 4, 3 * mesh.nv], 0)
    Ws[0][0, 0] = np.nan
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_decoder(Ws, bs, 1e-2)
    assert e.value.code == -3
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_cubature(np.array([0, mesh.ne], np.int32), np.ones(2))
    assert e.value.code == -1
    ctx.close()


def test_argument_errors_of_the_optimiser_cubature_and_training_calls(pkg):
    ctx = pkg.Context()
    mesh = make_bar(4, 3, 3, 0.05)
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0, 0, -9.8))
    # affine modes need a decoder, and fit in r <= 64 with it
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_affine_modes(mesh.X0.mean(0))
    assert e.value.code == -4
    Ws, bs = xavier_decoder([60, 8, 3 * mesh.nv], 0)
    ctx.set_decoder(Ws, bs, 1e-2)
    with pytest.raises(pkg.LsnError) as e:
        ctx.set_affine_modes(mesh.X0.mean(0))     # 60 + 12 > 64
    assert e.value.code == -1
    Ws, bs = xavier_decoder([4, 8, 3 * mesh.nv], 0)
    ctx.set_decoder(Ws, bs, 1e-2)
    for kind, hist in (("lbfgs", 0), ("lbfgs", 33)):
        with pytest.raises(pkg.LsnError) as e:
            ctx.set_optimizer(kind, hist)
        assert e.value.code == -1
    with pytest.raises(KeyError):
        ctx.set_optimizer("sgd", 10)
    ctx.set_state()
    Z = np.random.default_rng(0).standard_normal((2, 4)) * 0.1
    with pytest.raises(pkg.LsnError) as e:
        ctx.select_cubature(Z, mesh.ne + 1)
    assert e.value.code == -1
    # training: unsupported Lipschitz order, repeated unsupervised samples
    for order in (-1, 3):                         # orders 0, 1 and 2 exist
        with pytest.raises(pkg.LsnError) as e:
            ctx.set_lipschitz_order(order)
        assert e.value.code == -1
    ctx.train_init(np.zeros((4, 3 * mesh.nv), np.float32), np.zeros(4, np.float32),
                   np.arange(8, dtype=np.int32), np.ones(8))
    with pytest.raises(pkg.LsnError) as e:
        ctx.train_eval_unsup(np.vstack([Z[0], Z[0]]), 0.1, 0.05)
    assert e.value.code == -1
    with pytest.raises(pkg.LsnError) as e:
        ctx.train_eval_unsup(Z, 0.1, 0.0)           # sigma must be positive
    assert e.value.code == -1
    ctx.close()


def test_bounded_wait_runs_out_and_the_context_stays_usable(pkg):
    """Failure detection without a GPU fault: one mbarrier wait of the
    tensor-core kernels' kind on a barrier that nothing completes (no bulk
    copy or MMA in flight) gives up after its limit (50 ms here) and records
    its error code; the same context then evaluates as before (BF16 form,
    against the FP64 oracle of its rounded weights)."""
    import dataclasses
    import time
    from oracle.reduced import model_from_problem
    from workloads import build_problem
    from tests.gpu_util import round_bf16
    p = build_problem("tiny_quasistatic")
    ctx = pkg.context_from_problem(p, precision="bf16")
    z = np.random.default_rng(3).standard_normal(p.config.r) * 0.4
    E0, g0, K0 = ctx.eval(z)
    t0 = time.perf_counter()
    code = ctx.selftest_bounded_wait(0.05)
    dt = time.perf_counter() - t0
    assert code == 1
    assert 0.05 <= dt < 5.0
    with pytest.raises(Exception):
        ctx.selftest_bounded_wait(0.0)   # argument check, nothing launched
    E1, g1, K1 = ctx.eval(z)
    assert E1 == E0 and np.array_equal(g1, g0) and np.array_equal(K1, K0)
    m = model_from_problem(dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])]))
    m.set_targets(p.targets(0))
    _, g_ref, _ = m.eval(z)
    assert_close(g1, g_ref, 2e-4)
    ctx.close()
