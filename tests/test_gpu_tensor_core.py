"""GPU parity of the tensor-core (tcgen05) forms of the decoder output layer
against the FP64 CPU oracle.

BF16 form: the output-layer weights are stored in BF16 and the activations
enter as a two-term BF16 split, so against the oracle evaluated with the
same BF16-rounded weights it agrees like the FP32 form (x, J to 1e-5;
E, g to 2e-4); the inertia part of K is formed from BF16 operands (K to
5e-3, which changes Newton iterates only, not the converged point).  TF32
form: weights and activations both rounded to TF32 (10-bit mantissa), so
x, J, g agree with the FP32-weight oracle to a few 1e-3.  Solves: relative
displacement error 1e-4 for the BF16 form against the oracle of its own
weights and 5e-3 against the FP32-weight oracle (the BF16 rounding of W_L
changes the model by about 2e-3); 1e-3 for the TF32 form against the
FP32-weight oracle."""
import dataclasses

import numpy as np
import pytest

from oracle.reduced import model_from_problem, ReducedSimulator
from workloads import build_problem, CONFIGS
from tests.gpu_util import rel, random_qbar, round_bf16, assert_close, UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

TOL = {"bf16": dict(x=1e-5, J=1e-5, E=2e-4, g=2e-4, K=5e-3),
       "tf32": dict(x=5e-3, J=5e-3, E=5e-3, g=1e-2, K=1e-2)}


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


def oracle_for(p, prec):
    """The BF16 form is checked against the oracle of its own (BF16-rounded)
    output-layer weights; the TF32 form against the FP32 weights."""
    if prec == "bf16":
        p = dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    return model_from_problem(p)


def wide_problem():
    """r = 64 (the largest subspace), 68 decoder columns, every tet."""
    c = dataclasses.replace(CONFIGS["small_dyn_full"], name="wide_r64", dims=(24, 6, 6), r=64,
                            hidden=(128, 128))
    return build_problem(c)


@pytest.mark.parametrize("name", ["tiny_dyn", "bar_quasistatic_1824", "bar_twist_dyn_14976",
                                  "wide_r64"])
@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_positions_jacobian_and_system(pkg, name, prec):
    p = wide_problem() if name == "wide_r64" else build_problem(name)
    m = oracle_for(p, prec)
    ctx = pkg.context_from_problem(p, precision=prec)
    rng = np.random.default_rng(21)
    t = TOL[prec]
    tg = p.targets(3)
    ctx.set_constraints(None, tg)
    m.set_targets(tg)
    if p.config.dt > 0:
        qbar = random_qbar(p, 8)
        ctx.set_dynamics(p.config.dt, qbar)
        m.set_dynamics(p.config.dt, qbar)
    for trial in range(2):
        z = rng.standard_normal(p.config.r) * 0.5
        x, J = ctx.decode(z)
        x_ref, J_ref = m.positions_jac(z)
        assert_close(x - p.X0.ravel(), x_ref - p.X0.ravel(), t["x"], u=UNIT_ROUNDOFF[prec])
        assert_close(J, J_ref, t["J"], u=UNIT_ROUNDOFF[prec])
        cd = (3 * p.cnodes[:, None] + np.arange(3)).ravel()
        assert np.all(J[cd] == 0.0)
        E, g, K = ctx.eval(z)
        E_ref, g_ref, K_ref = m.eval(z)
        assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref)), (E, E_ref)
        assert_close(g, g_ref, t["g"], u=UNIT_ROUNDOFF[prec])
        assert_close(K, K_ref, t["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
        assert np.allclose(K, K.T)
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_quasistatic_solve(pkg, prec):
    p = build_problem("bar_quasistatic_1824")
    ctx = pkg.context_from_problem(p, precision=prec)
    ctx.set_constraints(None, p.targets(1))
    rc, st, z = ctx.step(dt=0.0)
    assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), st
    u = ctx.get_positions() - p.X0.ravel()
    # (oracle weights, bound): the BF16 form against the oracle of its own
    # BF16-rounded weights, and every form against the FP32-weight oracle;
    # rounding W_L to BF16 changes the model itself by a few 1e-3
    checks = [("bf16", 1e-4), ("tf32", 5e-3)] if prec == "bf16" else [("tf32", 1e-3)]
    for ref_prec, bound in checks:
        m = oracle_for(p, ref_prec)
        sim = ReducedSimulator(m, 0.0, eps=p.config.eps)
        assert sim.step(p.targets(1)).status == 0
        err = rel(u, sim.q - p.X0.ravel())
        print(f"{prec} solve vs {ref_prec}-weight oracle: rel. displacement error {err:.3e}")
        assert err < bound, (ref_prec, err)
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_dynamics_trajectory(pkg, prec):
    p = build_problem("tiny_dyn")
    m = oracle_for(p, prec)
    sim = ReducedSimulator(m, p.config.dt, eps=p.config.eps)
    ctx = pkg.context_from_problem(p, precision=prec, tol=1e-5)
    for k in range(1, p.config.steps + 1):
        sim.step(p.targets(k))
        ctx.set_constraints(None, p.targets(k))
        rc, st, z = ctx.step(dt=p.config.dt)
        assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
        err = rel(ctx.get_positions() - p.X0.ravel(), sim.q - p.X0.ravel())
        assert err < (1e-3 if prec == "bf16" else 3e-3), (k, err)
    ctx.close()


def _ctx_and_oracle(pkg, mesh, widths, prec, cub=None, cn=None, round_last=True):
    from oracle.decoder import Decoder
    from oracle.reduced import ReducedModel
    from workloads import xavier_decoder
    Ws, bs = xavier_decoder(widths, 0)
    ctx = pkg.Context()
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(1e5, 0.45, 1000.0, (0.0, 0.0, -9.8))
    if cub is not None:
        ctx.set_cubature(*cub)
    if cn is not None:
        ctx.set_constraints(cn, mesh.X0[cn])
    ctx.set_decoder(Ws, bs, 1e-2, prec)
    Wo = [*Ws[:-1], round_bf16(Ws[-1])] if (prec == "bf16" and round_last) else Ws
    m = ReducedModel(mesh.X0, mesh.tets, Decoder(Wo, bs, 1e-2), 1e5, 0.45, 1000.0,
                     (0.0, 0.0, -9.8), None if cub is None else cub[0],
                     None if cub is None else cub[1], cn)
    return ctx, m


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_single_tet_and_r1(pkg, prec):
    """One tet, one constrained vertex, r = 1 (N padded to 16 in the MMAs)."""
    X0 = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0.1]], float)
    mesh = type("M", (), {"X0": X0, "tets": np.array([[0, 1, 2, 3]], np.int32)})
    ctx, m = _ctx_and_oracle(pkg, mesh, [1, 8, 12], prec, cn=np.array([0], np.int32))
    t = TOL[prec]
    for z in (np.array([0.8]), np.array([-1.3])):
        E, g, K = ctx.eval(z)
        E0, g0, K0 = m.eval(z)
        assert abs(E - E0) <= t["E"] * max(1.0, abs(E0))
        assert_close(g, g0, t["g"], u=UNIT_ROUNDOFF[prec])
        assert_close(K, K0, t["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
    ctx.close()


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_tc_ragged_tiles_and_fp32_output_layer_fallback(pkg, prec):
    """Hidden width 13 (TMA row pitch not a multiple of 16 bytes): the output
    layer runs on the FP32 CUDA-core kernel with the FP32 weights, the element
    contraction on the tensor cores; one cubature tet and a ragged half set."""
    from workloads import make_bar
    mesh = make_bar(5, 4, 3, 0.05)
    for cub in [(np.array([7], np.int32), np.array([3.5])),
                (np.arange(0, mesh.ne, 2, dtype=np.int32), np.full((mesh.ne + 1) // 2, 2.0))]:
        ctx, m = _ctx_and_oracle(pkg, mesh, [7, 13, 3 * mesh.nv], prec, cub=cub,
                                 round_last=False)
        m.set_dynamics(0.02, mesh.X0.ravel() + 1e-3)
        ctx.set_dynamics(0.02, mesh.X0.ravel() + 1e-3)
        z = np.random.default_rng(3).standard_normal(7)
        x, J = ctx.decode(z)
        x0, J0 = m.positions_jac(z)
        assert_close(J, J0, 1e-5)  # FP32 output layer
        E, g, K = ctx.eval(z)
        E0, g0, K0 = m.eval(z)
        assert abs(E - E0) <= 1e-4 * max(1.0, abs(E0))
        assert_close(g, g0, 2e-3, u=UNIT_ROUNDOFF[prec])
        assert_close(K, K0, TOL[prec]["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
        ctx.close()
