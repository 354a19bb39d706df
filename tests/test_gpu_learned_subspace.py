"""What the learned subspace gains (Sec. 3.2, Sec. 4): a decoder trained on the
GPU by the project's own kernels (lsn_train_step: reconstruction loss Eq. 3,
optionally with the cubature Lipschitz loss Eq. 9 / Eq. 10) against the same
decoder untrained and trained without the Lipschitz term.

Snapshots are quasi-static full-space solutions of the FP64 oracle (a bar of
10x4x4 nodes, the x = 0 face fixed, the x = L face twisted by U[0, 1.5] rad
and bent by U[0, 0.3] rad about its centre).  Checked:
  * training reproduces the snapshots (reconstruction 1e3x below the
    untrained decoder's), and the Lipschitz term costs at most 3x of it;
  * the Lipschitz term lowers the subspace Hessian's Lipschitz estimate
    (Eq. 7 over the snapshot codes) by more than 10x;
  * on held-out loads the reduced FP64 solve with a trained decoder lands
    within a few percent of the full-space solution, far closer than the
    untrained subspace, and the Lipschitz-trained decoder needs no more
    Newton iterations than the vanilla one (within 25 %).
The measured numbers are printed (pytest -s)."""
import numpy as np
import pytest

from oracle.fullspace import FullModel, newton_solve as full_solve
from oracle.training import lipschitz_estimate
from workloads import make_bar, face_nodes, xavier_decoder
from tests.gpu_util import rel

pytestmark = pytest.mark.gpu

E_, NU, RHO, GRAV = 1e5, 0.45, 1000.0, (0.0, 0.0, -9.8)
SCALE = 0.05


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


def _rot(tw, bd):
    cx, sx, cy, sy = np.cos(tw), np.sin(tw), np.cos(bd), np.sin(bd)
    return (np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]]) @
            np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]]))


@pytest.fixture(scope="module")
def data():
    mesh = make_bar(10, 4, 4, 0.05)
    f0, f1 = face_nodes(mesh, 0), face_nodes(mesh, 1)
    cn = np.concatenate([f0, f1])

    def targets(tw, bd):
        P = mesh.X0[f1]
        c = P.mean(0)
        return np.concatenate([mesh.X0[f0], (P - c) @ _rot(tw, bd).T + c])

    fm = FullModel(mesh.X0, mesh.tets, E_, NU, RHO, GRAV, cn)
    rng = np.random.default_rng(2)
    loads = np.stack([rng.uniform(0, 1.5, 40), rng.uniform(0, 0.3, 40)], 1)
    loads = loads[np.argsort(loads[:, 0])]
    q = mesh.X0.ravel().copy()
    Q = []
    for tw, bd in loads:  # load continuation
        q, st = full_solve(fm, q, targets(tw, bd), 1e-6)[:2]
        assert st.status == 0
        Q.append(q.copy())
    rt = np.random.default_rng(7)
    held = np.stack([rt.uniform(0.1, 1.4, 4), rt.uniform(0, 0.3, 4)], 1)
    Qh = []
    for tw, bd in held:
        qh, st = full_solve(fm, mesh.X0.ravel().copy(), targets(tw, bd), 1e-6)[:2]
        assert st.status == 0
        Qh.append(qh)
    return mesh, cn, targets, np.array(Q), held, np.array(Qh)


def _unpack(th, widths, n):
    r = widths[0]
    Ew, eb = th[:r * n].reshape(r, n), th[r * n:r * n + r]
    o, Ws, bs = r * n + r, [], []
    for a, b in zip(widths[:-1], widths[1:]):
        Ws.append(th[o:o + a * b].reshape(b, a).astype(np.float32))
        o += a * b
        bs.append(th[o:o + b].astype(np.float32))
        o += b
    return Ew, eb, Ws, bs


def _train_and_measure(pkg, data, lam, steps, r=8, order=2):
    import torch
    mesh, cn, targets, Q, held, Qh = data
    n = 3 * mesh.nv
    widths = [r, 64, 64, n]
    Ws, bs = xavier_decoder(widths, 0)
    D = Q - mesh.X0.ravel()
    _, s, Vt = np.linalg.svd(D, full_matrices=False)  # PCA initial encoder
    Ew = (Vt[:r] / s[:r, None] * np.sqrt(Q.shape[0])).astype(np.float32)
    eb = np.zeros(r, np.float32)
    rng = np.random.default_rng(1)
    cub = np.sort(rng.choice(mesh.ne, 64, replace=False)).astype(np.int32)
    ctx = pkg.Context()
    ctx.set_mesh(mesh.X0, mesh.tets)
    ctx.set_material(E_, NU, RHO, GRAV)
    ctx.set_decoder(Ws, bs, SCALE, "fp32")
    ctx.train_init(Ew, eb, cub, np.full(64, mesh.ne / 64))
    ctx.set_lipschitz_order(order)
    rs = np.random.default_rng(3)
    for _ in range(steps):
        ctx.train_step(Q[rs.choice(Q.shape[0], 16, replace=False)], lam, 1e-3)
    (lc, _, _), _ = ctx.train_eval(Q, 0.0, want_grad=False)
    th = ctx.train_get_params()
    Ew_t, eb_t, Ws_t, bs_t = _unpack(th, widths, n)
    Z = (Q - mesh.X0.ravel()) @ Ew_t.T + eb_t
    lip = lipschitz_estimate(torch.tensor(ctx.train_hessians(Z)), torch.tensor(Z))
    ctx.close()
    # reduced FP64 solves of the held-out loads from the rest code
    sc = pkg.Context()
    sc.set_mesh(mesh.X0, mesh.tets)
    sc.set_material(E_, NU, RHO, GRAV)
    sc.set_constraints(cn, targets(0.0, 0.0))
    sc.set_decoder(Ws_t, bs_t, SCALE, "fp64")
    sc.set_solver(1e-7, 1024, 128, 1e-4)
    iters, errs = 0, []
    for (tw, bd), qh in zip(held, Qh):
        sc.set_state(eb_t.astype(np.float64))
        sc.set_constraints(None, targets(tw, bd))
        rc, st, _ = sc.step(dt=0.0)
        assert rc == pkg.LSN_OK, st
        iters += st["newton_iters"]
        errs.append(rel(sc.get_positions() - mesh.X0.ravel(), qh - mesh.X0.ravel()))
    sc.close()
    return dict(Lc=lc, lip=lip, iters=iters, err=max(errs), Ws=Ws_t, bs=bs_t, eb=eb_t)


@pytest.fixture(scope="module")
def trained(pkg, data):
    return {"untrained": _train_and_measure(pkg, data, 0.0, 0),
            "vanilla": _train_and_measure(pkg, data, 0.0, 3000),
            "lipschitz": _train_and_measure(pkg, data, 1e-6, 3000)}


def test_learned_subspace_gains(trained):
    untrained, vanilla, lipschitz = (trained[k] for k in ("untrained", "vanilla", "lipschitz"))
    for name, m in (("untrained", untrained), ("vanilla", vanilla), ("lipschitz", lipschitz)):
        print(f"{name:10s} L_C {m['Lc']:.3e}  Lip {m['lip']:.3e}  Newton iters {m['iters']:4d}"
              f"  max subspace error vs full space {m['err']:.3e}")
    assert vanilla["Lc"] < 1e-3 * untrained["Lc"]
    assert lipschitz["Lc"] < 3.0 * vanilla["Lc"]
    assert lipschitz["lip"] < 0.1 * vanilla["lip"]
    assert vanilla["err"] < 0.1 and lipschitz["err"] < 0.1
    assert max(vanilla["err"], lipschitz["err"]) < 0.2 * untrained["err"]
    assert lipschitz["iters"] <= 1.25 * vanilla["iters"]


def test_lbfgs_exit_shares_per_tolerance(pkg, data, trained):
    """The Supplement's exit table: L-BFGS (FP32 form, the paper's optimiser)
    on 40 implicit-Euler frames of the bar (far face twisted 0 -> 1.2 rad and
    bent 0 -> 0.15 rad over 30 frames, then held), for each tolerance and for
    the vanilla and the Lipschitz-trained decoder: the share of frames ending
    with each exit (I converged, II saddle, III line search, IV iteration
    cap, and the FP32 form's precision floor), the mean ||g||_inf at exit and
    the mean iterations per frame.  Printed (pytest -s); checked: every frame
    ends with one of these exits and every trajectory stays finite."""
    mesh, cn, targets, Q, held, Qh = data
    names = {0: "I", 5: "II", 2: "III", 1: "IV", 4: "floor"}
    rows = []
    for eps in (1e-4, 1e-5, 1e-6):
        for which in ("lipschitz", "vanilla"):
            t = trained[which]
            sc = pkg.Context()
            sc.set_mesh(mesh.X0, mesh.tets)
            sc.set_material(E_, NU, RHO, GRAV)
            sc.set_constraints(cn, targets(0.0, 0.0))
            sc.set_decoder(t["Ws"], t["bs"], SCALE, "fp32")
            sc.set_solver(eps, 1024, 128, 1e-4)
            sc.set_optimizer("lbfgs", 10)
            sc.set_state(t["eb"].astype(np.float64))
            exits, gs, its = {}, [], []
            for k in range(1, 41):
                a = min(k / 30.0, 1.0)
                sc.set_constraints(None, targets(1.2 * a, 0.15 * a))
                rc, st, _ = sc.step(dt=1.0 / 60.0)
                assert rc in names, (k, rc, st)
                assert np.all(np.isfinite(sc.get_positions()))
                exits[names[rc]] = exits.get(names[rc], 0) + 1
                gs.append(st["grad_inf"])
                its.append(st["newton_iters"])
            sc.close()
            share = {n: 100.0 * exits.get(n, 0) / 40 for n in ("I", "II", "III", "IV", "floor")}
            rows.append((eps, which, share, float(np.mean(gs)), float(np.mean(its))))
    print("\n eps     subspace    I      II     III    IV   floor   mean|g|exit  iters/frame")
    for eps, which, sh, g, it in rows:
        print(f" {eps:.0e}  {which:9s} " + " ".join(f"{sh[n]:5.1f}%" for n in
                                                   ("I", "II", "III", "IV", "floor")) +
              f"   {g:.2e}   {it:7.1f}")


def test_lipschitz_order_ablation(pkg, data, trained):
    """The Supplement's ablation of the Lipschitz loss's order: training with
    the zeroth- and first-order losses (potential and reduced-gradient
    differences) against the paper's second-order one (Hessian differences,
    Eq. 9) and no Lipschitz term.  lambda_0 and lambda_1 put the lower-order
    terms at the weight the second-order term has at the untrained decoder.  Printed: L_C, the Hessian Lipschitz
    estimate (Eq. 7) and Newton iterations on the held-out loads; checked:
    the second-order loss gives the lowest Hessian Lipschitz estimate."""
    import torch
    mesh, cn, targets, Q, held, Qh = data
    r = 8
    n = 3 * mesh.nv
    widths = [r, 64, 64, n]
    Ws, bs = xavier_decoder(widths, 0)
    _, sv, Vt = np.linalg.svd(Q - mesh.X0.ravel(), full_matrices=False)
    Ew = (Vt[:r] / sv[:r, None] * np.sqrt(Q.shape[0])).astype(np.float32)
    eb = np.zeros(r, np.float32)
    rng = np.random.default_rng(1)
    cub = np.sort(rng.choice(mesh.ne, 64, replace=False)).astype(np.int32)
    scale = {}
    for order in (0, 1, 2):
        ctx = pkg.Context()
        ctx.set_mesh(mesh.X0, mesh.tets)
        ctx.set_material(E_, NU, RHO, GRAV)
        ctx.set_decoder(Ws, bs, SCALE, "fp32")
        ctx.train_init(Ew, eb, cub, np.full(64, mesh.ne / 64))
        ctx.set_lipschitz_order(order)
        scale[order] = ctx.train_eval(Q[:16], 1.0, want_grad=False)[0][1]
        ctx.close()
    lam0 = 1e-6 * scale[2] / scale[0]
    lam1 = 1e-6 * scale[2] / scale[1]
    zeroth = _train_and_measure(pkg, data, lam0, 3000, order=0)
    first = _train_and_measure(pkg, data, lam1, 3000, order=1)
    van, second = trained["vanilla"], trained["lipschitz"]
    print(f"\n lambda_0 {lam0:.3e}  lambda_1 {lam1:.3e}")
    for name, m in (("vanilla", van), ("order 0", zeroth), ("order 1", first),
                    ("order 2", second)):
        print(f" {name:8s} L_C {m['Lc']:.3e}  Lip[Hessian] {m['lip']:.3e}  "
              f"Newton iters {m['iters']:4d}  max error {m['err']:.3e}")
    assert second["lip"] < min(van["lip"], zeroth["lip"], first["lip"])
