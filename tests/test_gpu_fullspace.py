"""GPU parity of the full-space projective-Newton solve (Eq. 1 over all n
DOFs, every tet at unit weight: the comparison solve of the reduced method)
through the C ABI, against the FP64 oracle's full-space solve
(oracle/fullspace.py: a sparse direct factorisation of the same projected
Hessian).

The GPU solves each Newton system by Jacobi-preconditioned CG.  With
cg_rtol = 1e-12 its directions equal the direct solve's to rounding, so the
FP64 GPU solve follows the oracle's iterates: the same exit, Newton
iterations within one, and the end point to 1e-7.  With FP32 element math
the end point agrees to 1e-4, and the exit is converged or the precision
floor.  A loose CG tolerance changes the iterates but not the end point
(checked to 1e-6 at eps = 1e-7)."""
import numpy as np
import pytest

from oracle.fullspace import FullModel, newton_solve
from oracle.reduced import CONVERGED
from workloads import build_problem, make_bar, face_nodes
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


def _ctx(pkg, X0, tets, grav, cnodes, targets, eps, prec, rtol, youngs=1e5, poisson=0.45,
         max_cg=4096):
    ctx = pkg.Context()
    ctx.set_mesh(X0, tets)
    ctx.set_material(youngs, poisson, 1000.0, grav)
    ctx.set_solver(eps)
    ctx.set_constraints(cnodes, targets)
    ctx.fullspace_setup(prec, rtol, max_cg)
    return ctx


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,eps", [((8, 3, 3), 1e-7), ((9, 4, 3), 1e-6)])
def test_quasistatic_sag_matches_oracle(pkg, prec, dims, eps):
    """Cantilever under gravity from rest (quasi-static); the second mesh
    has a tet count that fills no CTA evenly.  eps is one that the FP64
    oracle reaches: below about 1e-7 (8 x 3 x 3) or 1e-6 (9 x 4 x 3) its
    energy differences no longer resolve the Armijo decrease and it stops at
    the iteration cap."""
    mesh = make_bar(*dims, 0.05)
    cn = face_nodes(mesh, 0)
    fm = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, (0, 0, -9.8), cn)
    q_ref, st_ref = newton_solve(fm, mesh.X0.ravel(), mesh.X0[cn], eps)
    assert st_ref.status == CONVERGED
    ctx = _ctx(pkg, mesh.X0, mesh.tets, (0, 0, -9.8), cn, mesh.X0[cn], eps, prec,
               1e-12 if prec == "fp64" else 1e-6)
    rc, st, q = ctx.fullspace_step(0.0)
    u, u_ref = q - mesh.X0.ravel(), q_ref - mesh.X0.ravel()
    if prec == "fp64":
        assert rc == pkg.LSN_OK, st
        assert abs(st["newton_iters"] - st_ref.newton_iters) <= 1, (st, st_ref.newton_iters)
        assert_close(u, u_ref, 1e-7)
        assert st["energy"] == pytest.approx(st_ref.energy, rel=1e-10, abs=1e-12)
        # the oracle's own gradient test at the GPU's end point
        assert np.max(np.abs(fm.gradient(q)[fm.free])) < 2 * eps
    else:
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
        assert_close(u, u_ref, 1e-4)
    assert np.array_equal(q.reshape(-1, 3)[cn], mesh.X0[cn])
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_implicit_euler_steps_match_oracle(pkg, prec):
    """Six implicit-Euler steps of the rotating bar (tiny_dyn's mesh,
    constraints and dt; every tet), each from the previous state, at
    eps = 1e-6: at tiny_dyn's 1e-7 the FP64 oracle's third step stops at the
    iteration cap with ||g|| = 1.2e-7, at the rounding level of its energy
    differences."""
    p = build_problem("tiny_dyn")
    c = p.config
    eps = 1e-6
    fm = FullModel(p.X0, p.tets, c.youngs, c.poisson, c.density, c.gravity, p.cnodes)
    ctx = _ctx(pkg, p.X0, p.tets, c.gravity, p.cnodes, p.targets(1), eps, prec,
               1e-12 if prec == "fp64" else 1e-6, c.youngs, c.poisson)
    q = p.X0.ravel().copy()
    v = np.zeros_like(q)
    g = np.tile(np.asarray(c.gravity, np.float64), p.X0.shape[0])
    for k in range(1, 7):
        tg = p.targets(k)
        fm.set_dynamics(c.dt, q + c.dt * v + c.dt ** 2 * g)
        q1, st_ref = newton_solve(fm, q, tg, eps)
        assert st_ref.status == CONVERGED
        v = (q1 - q) / c.dt
        q = q1
        ctx.set_constraints(None, tg)
        rc, st, qg = ctx.fullspace_step(c.dt)
        u, u_ref = qg - p.X0.ravel(), q - p.X0.ravel()
        if prec == "fp64":
            assert rc == st_ref.status, (k, st, st_ref.status)
            assert abs(st["newton_iters"] - st_ref.newton_iters) <= 1, (k, st)
            assert_close(u, u_ref, 1e-7)
        else:
            assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
            assert_close(u, u_ref, 1e-4)
        assert st["cg_iters"] >= st["newton_iters"]
        # continue the oracle from the GPU's state so that FP32 rounding does
        # not accumulate into the comparison
        if prec == "fp32":
            v = v + (qg - q) / c.dt
            q = qg.copy()
    ctx.close()


def test_loose_cg_tolerance_keeps_the_end_point(pkg):
    mesh = make_bar(8, 3, 3, 0.05)
    cn = face_nodes(mesh, 0)
    fm = FullModel(mesh.X0, mesh.tets, 1e5, 0.45, 1000.0, (0, 0, -9.8), cn)
    q_ref, _ = newton_solve(fm, mesh.X0.ravel(), mesh.X0[cn], 1e-7)
    its = {}
    for rtol in (1e-2, 1e-4):
        ctx = _ctx(pkg, mesh.X0, mesh.tets, (0, 0, -9.8), cn, mesh.X0[cn], 1e-7, "fp64", rtol)
        rc, st, q = ctx.fullspace_step(0.0)
        assert rc == pkg.LSN_OK, st
        assert_close(q - mesh.X0.ravel(), q_ref - mesh.X0.ravel(), 1e-6)
        its[rtol] = (st["newton_iters"], st["cg_iters"])
        ctx.close()
    # the looser tolerance takes fewer CG iterations per Newton direction
    print(f"\n CG tolerance 1e-2: {its[1e-2]}, 1e-4: {its[1e-4]} (Newton, CG iterations)")
    assert its[1e-2][1] / its[1e-2][0] < its[1e-4][1] / its[1e-4][0]


def test_rest_without_load_and_state_calls(pkg):
    mesh = make_bar(5, 3, 3, 0.05)
    cn = face_nodes(mesh, 0)
    ctx = _ctx(pkg, mesh.X0, mesh.tets, (0, 0, 0), cn, mesh.X0[cn], 1e-9, "fp64", 1e-8)
    rc, st, q = ctx.fullspace_step(0.0)
    assert rc == pkg.LSN_OK and st["newton_iters"] == 0 and st["cg_iters"] == 0
    assert np.array_equal(q, mesh.X0.ravel())
    # a displaced start relaxes back to rest (free DOFs only)
    q0 = mesh.X0.ravel() + 1e-3 * np.random.default_rng(1).standard_normal(3 * mesh.nv)
    ctx.fullspace_set_state(q0)
    rc, st, q = ctx.fullspace_step(0.0)
    assert rc == pkg.LSN_OK and st["newton_iters"] > 0
    assert np.max(np.abs(q - mesh.X0.ravel())) < 1e-6
    ctx.close()


def test_fullspace_argument_errors(pkg):
    mesh = make_bar(5, 3, 3, 0.05)
    ctx = pkg.Context()
    with pytest.raises(pkg.LsnError) as e:
        ctx.fullspace_setup("fp64")                 # no mesh
    assert e.value.code == -4
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0, 0, -9.8))
    with pytest.raises(pkg.LsnError) as e:
        ctx.fullspace_step(0.0)                     # no setup
    assert e.value.code == -4
    for args in (("bf16", 1e-4, 100), ("fp64", 1.0, 100), ("fp64", 1e-4, 0)):
        with pytest.raises(pkg.LsnError) as e:
            ctx.fullspace_setup(*args)
        assert e.value.code == -1
    ctx.fullspace_setup("fp32", 1e-4, 64)
    with pytest.raises(pkg.LsnError) as e:
        ctx.fullspace_step(-1.0)
    assert e.value.code == -1
    ctx.set_ground(0.0, 1e4)
    with pytest.raises(pkg.LsnError) as e:
        ctx.fullspace_step(0.0)
    assert e.value.code == -4
    ctx.close()
