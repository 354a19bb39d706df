"""GPU parity of the optimised cubature selection (Sec. 4.3, after von
Tycowicz et al. 2013; the cubature-count trade-off of Sec. 5.3) through the
C ABI: the per-tet reduced force matrix against the FP64 oracle, the
Lawson-Hanson selection against the oracle's, and the trade-off on the bar
twist (printed with pytest -s)."""
import dataclasses

import numpy as np
import pytest

from oracle.cubature_fit import tet_force_matrix, select_cubature
from oracle.reduced import model_from_problem
from workloads import build_problem, CONFIGS, draw_cubature
from tests.gpu_util import rel, round_bf16, assert_close, UNIT_ROUNDOFF

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


@pytest.mark.parametrize("name", ["tiny_dyn", "tiny_torus_drop"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_tet_forces_match_oracle(pkg, name, prec):
    p = build_problem(name)
    pr = p if prec != "bf16" else dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    m = model_from_problem(pr)
    ctx = pkg.context_from_problem(p, precision=prec)
    tg = p.targets(3)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    Z = np.random.default_rng(6).standard_normal((3, m.r)) * 0.4
    A = ctx.tet_forces(Z)
    A_ref = tet_force_matrix(m, Z)
    assert A.shape == A_ref.shape == (3 * m.r, p.ne)
    assert_close(A, A_ref, (1e-11 if prec == "fp64" else 2e-5), u=UNIT_ROUNDOFF[prec])
    ctx.close()


@pytest.mark.parametrize("S", [8, 24])
def test_selection_matches_oracle(pkg, S):
    """FP64: the same active tets (ascending), weights and residual (S below
    the K r = 36 rows of the fit, where the active columns stay independent)."""
    p = build_problem("tiny_dyn")
    m = model_from_problem(p)
    ctx = pkg.context_from_problem(p, precision="fp64")
    tg = p.targets(4)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    Z = np.random.default_rng(7).standard_normal((6, m.r)) * 0.4
    idx, w, res = ctx.select_cubature(Z, S)
    idx_ref, w_ref, res_ref = select_cubature(m, Z, S)
    order = np.argsort(idx_ref)
    assert np.array_equal(idx, idx_ref[order])
    assert np.allclose(w, w_ref[order], rtol=1e-8)
    assert res == pytest.approx(res_ref, rel=1e-8, abs=1e-14)
    assert len(idx) <= S and np.all(w > 0)
    # the solver's state is untouched
    z_before = ctx.get_state()[0].copy()
    ctx.select_cubature(Z, 4)
    assert np.array_equal(ctx.get_state()[0], z_before)
    ctx.close()


def test_cubature_count_tradeoff_on_the_bar_twist(pkg):
    """Fit residual against S for the optimised cubature and for uniform
    draws of the same size, at 64 subspace points (16 points of the bar-twist
    trajectory, all tets in the solve, and three perturbations of each, so the
    fit has 1,024 equations), and the runtime effect: 12 frames solved with
    each 256-tet cubature against the all-tet solve."""
    c_all = dataclasses.replace(CONFIGS["bar_twist_dyn_14976"], cubature=0)
    p = build_problem(c_all)
    ctx = pkg.context_from_problem(p, precision="fp32")
    Z, Q = [], []
    for k in range(1, 33):
        ctx.set_constraints(None, p.targets(k))
        rc, st, z = ctx.step(dt=p.config.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR, pkg.LSN_NOT_CONVERGED)
        if k % 2 == 0:
            Z.append(z.copy())
        Q.append(ctx.get_positions())
    Z = np.array(Z)
    rng = np.random.default_rng(11)
    Z = np.concatenate([Z] + [Z + 0.2 * rng.standard_normal(Z.shape) for _ in range(3)])
    A = ctx.tet_forces(Z)
    r = p.config.r
    b = A.sum(axis=1)
    # the same per-snapshot normalisation as the fit, for uniform draws
    An, bn = A.copy(), b.copy()
    for k in range(Z.shape[0]):
        nb = np.linalg.norm(b[k * r:(k + 1) * r])
        An[k * r:(k + 1) * r] /= nb
        bn[k * r:(k + 1) * r] /= nb
    rows = []
    sel256 = None
    for S in (32, 64, 128, 256, 512):
        idx, w, res = ctx.select_cubature(Z, S)
        ui, uw = draw_cubature(p.ne, S, 1)
        ures = np.linalg.norm(An[:, ui] @ uw - bn) / np.linalg.norm(bn)
        rows.append((S, len(idx), res, ures))
        if S == 256:
            sel256 = (idx, w)
    print("\n   S  active  fit residual (optimised)  fit residual (uniform)")
    for S, k, res, ures in rows:
        print(f" {S:4d} {k:6d}  {res:12.3e}              {ures:12.3e}")
    res = [x[2] for x in rows]
    assert all(b2 <= b1 + 1e-12 for b1, b2 in zip(res, res[1:]))
    assert all(x[2] < x[3] for x in rows)
    ctx.close()
    # runtime: 12 frames with the optimised and the uniform 256-tet cubature
    errs = {}
    for label, (ci, cw) in (("optimised", sel256), ("uniform", draw_cubature(p.ne, 256, 1))):
        cc = pkg.context_from_problem(p, precision="fp32")
        cc.set_cubature(ci, cw)
        cc.set_state()
        e = []
        for k in range(1, 13):
            cc.set_constraints(None, p.targets(k))
            cc.step(dt=p.config.dt)
            e.append(rel(cc.get_positions() - p.X0.ravel(), Q[k - 1] - p.X0.ravel()))
        errs[label] = max(e)
        cc.close()
    print(f" 12 frames, 256 cubature tets vs every tet: optimised {errs['optimised']:.3e}, "
          f"uniform {errs['uniform']:.3e}")
    assert errs["optimised"] < errs["uniform"]
