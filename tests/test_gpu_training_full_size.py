"""The training workload at full size (bar 30x17x17 nodes, 44,544 tets,
n = 26,010; decoder 16-256x3-26010; 512 cubature tets; batch 64): the GPU
gradient of L = L_C + lambda L_LS checked by central differences of the GPU
loss itself on 8 random parameters (FP64 trainer, step 1e-6 max(1, |theta|)),
and one FP32 Adam step that lowers the loss.  The BF16 trainer form (BF16
operands in every product, FP32 master weights) against that central-
difference-checked FP64 gradient at full size, every decoder block (the
oracle's autodiff at this size is too slow for a test; the two forms agree
with the oracle at the small size in test_gpu_training.py), and BF16 Adam steps
that lower the loss.  At this size the Lipschitz loss and its gradient cancel
more than at the small size, so the BF16 form's bands are wider there.  The snapshots are seeded smooth displacement fields (the
oracle's 1,024 full-space solves at this size are far too slow for a test; the
gradient check does not depend on them)."""
import numpy as np
import pytest

from workloads import build_problem, draw_cubature

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


def _setup(pkg, prec):
    p = build_problem("bar_train_44544")
    c = p.config
    rng = np.random.default_rng(2)
    X = p.X0
    L = X[:, 0].max()
    # smooth fields: twist and bend of random amplitude along the bar axis
    Q = []
    for _ in range(64):
        tw, bd = rng.uniform(0, 0.3), rng.uniform(0, 0.05)
        s = X[:, 0] / L
        d = np.zeros_like(X)
        yc, zc = X[:, 1] - X[:, 1].mean(), X[:, 2] - X[:, 2].mean()
        d[:, 1] = (np.cos(tw * s) - 1) * yc - np.sin(tw * s) * zc
        d[:, 2] = np.sin(tw * s) * yc + (np.cos(tw * s) - 1) * zc - bd * s * s * L
        Q.append((X + d).ravel())
    Q = np.array(Q)
    cub, w = draw_cubature(p.ne, c.cubature, c.cubature_seed)
    r, n = c.r, p.n
    Ew = (rng.standard_normal((r, n)) / np.sqrt(n)).astype(np.float32)
    eb = np.zeros(r, np.float32)
    ctx = pkg.Context()
    ctx.set_mesh(p.X0, p.tets)
    ctx.set_material(c.youngs, c.poisson, c.density, c.gravity)
    ctx.set_decoder(p.Ws, p.bs, c.out_scale, prec)
    ctx.train_init(Ew, eb, cub, w)
    return p, ctx, Q


def test_full_size_gradient_by_central_differences(pkg):
    p, ctx, Q = _setup(pkg, "fp64")
    lam = 1e-3
    (_, lls, L), g = ctx.train_eval(Q, lam)
    assert np.isfinite(L) and lls > 0.0
    th = ctx.train_get_params()
    r, n = p.config.r, p.n
    rng = np.random.default_rng(100)
    cand = np.arange(r * n + r, th.shape[0])  # decoder parameters
    for k in rng.choice(cand, 8, replace=False):
        h = 1e-6 * max(1.0, abs(float(th[k])))
        tp_, tm_ = th.copy(), th.copy()
        tp_[k] += h
        tm_[k] -= h
        ctx.train_set_params(tp_)
        Lp = ctx.train_eval(Q, lam, want_grad=False)[0][2]
        ctx.train_set_params(tm_)
        Lm = ctx.train_eval(Q, lam, want_grad=False)[0][2]
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(float(g[k]), rel=1e-5, abs=1e-7 * np.abs(g).max()), k
    ctx.close()


def test_full_size_fp32_adam_steps_lower_the_loss(pkg):
    p, ctx, Q = _setup(pkg, "fp32")
    l0 = ctx.train_eval(Q, 1e-3, want_grad=False)[0][2]
    for _ in range(20):
        ctx.train_step(Q, 1e-3, 1e-4)
    l1 = ctx.train_eval(Q, 1e-3, want_grad=False)[0][2]
    assert np.isfinite(l1) and l1 < l0
    ctx.close()


def test_full_size_bf16_gradient_against_fp64(pkg):
    """Losses and per-block gradient of the BF16 form against the FP64 form at
    the same parameters.  L_C 1e-3.  L_LS sums squared differences of the
    subspace Hessians of 64 smooth, similar fields, which cancel: the BF16
    rounding of every product reaches it at 10.3 % here (3 % at the small
    size), so 0.2.  Gradient blocks 0.2 relative and 0.99 cosine (measured:
    the encoder 2.7e-3, the decoder blocks 0.04-0.12 with cosines above
    0.993).  The measured values are printed (pytest -s)."""
    from tests.gpu_util import rel
    lam = 1e-3
    p, c64, Q = _setup(pkg, "fp64")
    (lc0, lls0, _), g0 = c64.train_eval(Q, lam)
    th = c64.train_get_params()
    c64.close()
    _, c16, _ = _setup(pkg, "bf16")
    c16.train_set_params(th)
    (lc, lls, _), g = c16.train_eval(Q, lam)
    r, n = p.config.r, p.n
    sizes = [r * n, r] + [sz for a, b in zip(p.widths[:-1], p.widths[1:]) for sz in (a * b, b)]
    o, blocks = 0, []
    for sz in sizes:  # encoder W, b, then every decoder layer's W, b
        gb, g0b = g[o:o + sz], g0[o:o + sz]
        blocks.append((sz, rel(gb, g0b), gb @ g0b / (np.linalg.norm(gb) * np.linalg.norm(g0b))))
        o += sz
    assert o == g.shape[0]
    print(f"\nBF16 vs FP64 at full size: L_C {abs(lc / lc0 - 1):.2e}, L_LS {abs(lls / lls0 - 1):.2e}")
    for sz, rl, cs in blocks:
        print(f"  block of {sz}: rel {rl:.3e}, cos {cs:.6f}")
    assert lc == pytest.approx(lc0, rel=1e-3)
    assert lls == pytest.approx(lls0, rel=0.2)
    for sz, rl, cs in blocks:
        assert rl < 0.2 and cs > 0.99, (sz, rl, cs)
    l0 = c16.train_eval(Q, lam, want_grad=False)[0][2]
    for _ in range(20):
        c16.train_step(Q, lam, 1e-4)
    l1 = c16.train_eval(Q, lam, want_grad=False)[0][2]
    assert np.isfinite(l1) and l1 < l0
    c16.close()
