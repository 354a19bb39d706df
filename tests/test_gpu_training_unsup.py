"""GPU parity of the unsupervised construction (Eq. 4: potential loss plus
the M-weighted repulsion loss, lsn_train_*_unsup, optionally with the
Lipschitz loss of Eq. 9 at the same Gaussian samples) against the float64
autodiff oracle, and the two trainings compared on the free torus: vanilla
unsupervised against unsupervised with the Lipschitz term, in the
subspace-Hessian Lipschitz estimate (Eq. 7) and Newton iterations per
implicit-Euler step of the reduced FP64 solve.

Tolerances: FP64 trainer 1e-8 (losses, every gradient block); FP32 trainer
losses 1e-4 and gradient 2e-3 relative (the Lipschitz term's gradient blocks
as in test_gpu_training.py: 0.2); TF32 trainer losses 2e-3 and gradient
3e-2 (Lipschitz blocks 0.2)."""
import dataclasses

import numpy as np
import pytest

from oracle.training import unsupervised_loss_and_grad
from workloads import build_problem, CONFIGS, draw_cubature, xavier_decoder
from tests.gpu_util import rel, assert_close, UNIT_ROUNDOFF
from tests.test_gpu_training import make_case, gpu_ctx

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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("lam,lam_ls", [(0.0, 0.0), (0.5, 0.0), (0.5, 1e-3)])
def test_unsupervised_losses_and_gradient_match_oracle(pkg, lam, lam_ls, prec):
    mesh, widths, cub, w, Ws, bs, Ew, eb, Q, tp, theta = make_case(B=6)
    ctx = gpu_ctx(pkg, mesh, Ws, bs, Ew, eb, cub, w, prec)
    th = ctx.train_get_params()
    Z = np.random.default_rng(9).standard_normal((6, widths[0]))
    sigma = 0.02
    losses, g = ctx.train_eval_unsup(Z, lam, sigma, lam_ls)
    losses0, g0 = unsupervised_loss_and_grad(tp, th, Z, lam, sigma, lam_ls)
    # BF16 operands: eight times the TF32 bands (the ratio of the unit roundoffs)
    tl, tg = {"fp64": (1e-8, 1e-8), "fp32": (1e-4, 2e-3), "tf32": (2e-3, 3e-2),
              "bf16": (2e-2, 0.25)}[prec]
    if lam_ls > 0.0 and prec != "fp64":
        tg = max(tg, 0.2)
    for a, b in zip(losses, losses0):
        assert a == pytest.approx(b, rel=tl, abs=1e-12)
    o = 0
    for shp in tp.shapes:
        sz = int(np.prod(shp))
        gb, g0b = g[o:o + sz], g0[o:o + sz]
        if np.linalg.norm(g0b) > 1e-10 * np.linalg.norm(g0):
            assert_close(gb, g0b, tg, u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16"
                                                      else prec])
        else:
            assert np.linalg.norm(gb) <= 1e-6 * np.linalg.norm(g0) + 1e-30
        o += sz
    ctx.close()


def test_unsupervised_training_on_the_torus(pkg):
    """Decoders of the tiny torus (6 network coordinates + 12 affine modes)
    trained on Gaussian samples only (Eq. 4, 1,500 Adam steps, batch 16,
    lambda 0.1, sigma 0.05), without and with the Lipschitz term at the same
    samples (lambda_LS = 1): both lower the potential loss, and the
    Lipschitz-trained subspace needs no more Newton iterations per step of
    the reduced FP64 solve of the dropped, spinning torus than the vanilla
    one.  The losses, the Lipschitz estimate on held-out samples and the
    iterations (with the untrained decoder's) are printed (pytest -s)."""
    import torch
    from oracle.training import lipschitz_estimate
    c = dataclasses.replace(CONFIGS["tiny_torus_drop"], eps=1e-6)
    p = build_problem(c)
    r = c.r
    cub, cw = draw_cubature(p.ne, 256, 1)
    Zh = np.random.default_rng(17).standard_normal((16, r))

    def train(lam_ls, steps=1500):
        ctx = pkg.Context()
        ctx.set_mesh(p.X0, p.tets)
        ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
        ctx.set_decoder(p.Ws, p.bs, c.out_scale, "fp32")
        ctx.train_init(np.zeros((r, p.n), np.float32), np.zeros(r, np.float32), cub, cw)
        rng = np.random.default_rng(3)
        l0 = ctx.train_eval_unsup(Zh, 0.1, 0.05, lam_ls, want_grad=False)[0]
        for _ in range(steps):
            ctx.train_step_unsup(rng.standard_normal((16, r)), 0.1, 0.05, 1e-3, lam_ls)
        l1 = ctx.train_eval_unsup(Zh, 0.1, 0.05, lam_ls, want_grad=False)[0]
        lip = lipschitz_estimate(torch.tensor(ctx.train_hessians(Zh)), torch.tensor(Zh))
        th = ctx.train_get_params()
        ctx.close()
        o = r * p.n + r
        Ws, bs = [], []
        for a, b in zip(p.widths[:-1], p.widths[1:]):
            Ws.append(th[o:o + a * b].reshape(b, a).astype(np.float32))
            o += a * b
            bs.append(th[o:o + b].astype(np.float32))
            o += b
        return l0, l1, lip, Ws, bs

    def solve(Ws_, bs_):
        pp = dataclasses.replace(p, Ws=Ws_, bs=bs_)
        sc = pkg.context_from_problem(pp, precision="fp64")
        its = []
        for k in range(1, c.steps + 1):
            rc, st, _ = sc.step(dt=c.dt)
            assert rc == pkg.LSN_OK, (k, st)
            its.append(st["newton_iters"])
        sc.close()
        return float(np.mean(its))

    lam_ls = 1.0
    van = train(0.0)
    lip = train(lam_ls)
    it_u = solve(p.Ws, p.bs)
    it_v, it_l = solve(van[3], van[4]), solve(lip[3], lip[4])
    print(f"\n lambda_LS {lam_ls:.3e}")
    for name, t, it in (("vanilla", van, it_v), ("lipschitz", lip, it_l)):
        print(f" {name:9s} L_P {t[0][0]:.3e} -> {t[1][0]:.3e}  L_R {t[0][1]:.3e} -> {t[1][1]:.3e}"
              f"  Lip {t[2]:.3e}  Newton iters/step {it:.2f}")
    print(f" untrained Newton iters/step {it_u:.2f}")
    assert van[1][0] < van[0][0] and lip[1][0] < lip[0][0]
    assert it_l <= it_v


def test_unsupervised_training_at_the_full_torus(pkg):
    """torus_drop_200k (200,928 tets, n = 119,268, r = 32 + 12 affine modes,
    decoder 32-512x3-n, its 1,024 cubature tets): 300 Adam steps of the
    unsupervised loss (batch 16, lambda 0.1, sigma 0.05) without and with
    the Lipschitz term (lambda_LS = 1) on the FP32 trainer, then 24 frames of
    the FP32 reduced solve (free fall and the first contacts) with the
    untrained and the two trained decoders.  Printed: losses and Newton
    iterations per step; checked: the potential loss drops and every solve
    step ends converged or at the FP32 form's precision floor."""
    p = build_problem("torus_drop_200k")
    c = p.config
    r = c.r

    def train(lam_ls, steps=300):
        ctx = pkg.Context()
        ctx.set_mesh(p.X0, p.tets)
        ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
        ctx.set_decoder(p.Ws, p.bs, c.out_scale, "fp32")
        ctx.train_init(np.zeros((r, p.n), np.float32), np.zeros(r, np.float32), p.cub_idx,
                       p.cub_w)
        rng = np.random.default_rng(3)
        Zt = rng.standard_normal((16, r))
        l0 = ctx.train_eval_unsup(Zt, 0.1, 0.05, lam_ls, want_grad=False)[0]
        for _ in range(steps):
            ctx.train_step_unsup(rng.standard_normal((16, r)), 0.1, 0.05, 1e-3, lam_ls)
        l1 = ctx.train_eval_unsup(Zt, 0.1, 0.05, lam_ls, want_grad=False)[0]
        th = ctx.train_get_params()
        ctx.close()
        o = r * p.n + r
        Ws, bs = [], []
        for a, b in zip(p.widths[:-1], p.widths[1:]):
            Ws.append(th[o:o + a * b].reshape(b, a).astype(np.float32))
            o += a * b
            bs.append(th[o:o + b].astype(np.float32))
            o += b
        return l0, l1, Ws, bs

    def solve(Ws_, bs_):
        pp = dataclasses.replace(p, Ws=Ws_, bs=bs_)
        sc = pkg.context_from_problem(pp, precision="fp32")
        its = []
        for k in range(1, 25):
            rc, st, _ = sc.step(dt=c.dt)
            assert rc in (pkg.LSN_OK, pkg.LSN_PRECISION_FLOOR), (k, st)
            its.append(st["newton_iters"])
        sc.close()
        return float(np.mean(its))

    van = train(0.0)
    lip = train(1.0)
    it_u, it_v, it_l = solve(p.Ws, p.bs), solve(van[2], van[3]), solve(lip[2], lip[3])
    print(f"\n full torus: untrained {it_u:.2f} Newton iterations / step")
    for name, t, it in (("vanilla", van, it_v), ("lipschitz", lip, it_l)):
        print(f" {name:9s} L_P {t[0][0]:.3e} -> {t[1][0]:.3e}  L_R {t[0][1]:.3e} -> "
              f"{t[1][1]:.3e}  L_LS {t[1][3]:.3e}  Newton iterations / step {it:.2f}")
    assert van[1][0] < van[0][0] and lip[1][0] < lip[0][0]
