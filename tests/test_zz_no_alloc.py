"""Allocation-free entry point: lsn_element_system_noalloc.

For callers that must not allocate device memory while they run (a fixed
memory budget handed to the library up front, a pool or arena that must not
grow, a real-time loop where cudaMalloc / cudaFree is not allowed), the
library evaluates the elastic reduced system with its partial sums in a
fixed device array instead of cudaMalloc'd scratch.  This file checks that
entry point through the C ABI against the regular one (lsn_eval with
gravity off, so that only the elastic term remains), on two calls in a row
with different inputs.  It is kept last in collection order.
"""
import numpy as np
import pytest

from oracle import fem
from oracle.reduced import model_from_problem
from workloads import build_problem
from tests.gpu_util import rel, close_elementwise

pytestmark = pytest.mark.gpu

TOL = dict(E=1e-4, g=2e-4, K=1e-4)   # the FP32 parity tolerances of the solver tests


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


@pytest.mark.parametrize("name", ["bar_twist_dyn_14976", "bar_quasistatic_1824"])
def test_noalloc_element_system_matches_eval(pkg, name):
    import torch
    p = build_problem(name)
    c = p.config
    r, n = c.r, p.n
    ctx = pkg.Context()
    ctx.set_mesh(p.X0, p.tets)
    ctx.set_material(c.youngs, c.poisson, c.density, (0.0, 0.0, 0.0))
    if c.cubature > 0:
        ctx.set_cubature(p.cub_idx, p.cub_w)
    ctx.set_constraints(p.cnodes, p.targets(3))
    ctx.set_decoder(p.Ws, p.bs, c.out_scale, "fp32")
    ctx.set_dynamics(0.0)
    mu = c.youngs / (2 * (1 + c.poisson))
    lam = c.youngs * c.poisson / ((1 + c.poisson) * (1 - 2 * c.poisson))
    # per-tet inputs of the cubature set (structure-of-arrays Dm^-1, w V)
    DmInv, vol = fem.rest_shape(p.X0, p.tets)
    idx = p.cub_idx
    S = idx.shape[0]
    dev = torch.device("cuda", 0)
    tets = torch.tensor(p.tets[idx], dtype=torch.int32, device=dev).contiguous()
    dminv = torch.tensor(DmInv[idx].reshape(S, 9).T.copy(), dtype=torch.float32, device=dev)
    wvol = torch.tensor(p.cub_w * vol[idx], dtype=torch.float32, device=dev)
    ns = 2 + 2 * r + r * (r + 1) // 2
    # the oracle's model with gravity off and no inertia: its E, g, K are the
    # elastic cubature sums alone
    om = model_from_problem(p)
    om.gravity = np.zeros(3)
    om.set_targets(p.targets(3))
    om.set_dynamics(0.0, None)
    out = torch.zeros(ns, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(17)
    first = None
    for call in range(2):
        z = rng.standard_normal(r) * 0.6
        E_ref, g_ref, K_ref = ctx.eval(z)
        x, J = ctx.decode(z)
        u_d = torch.tensor(x - p.X0.ravel(), dtype=torch.float32, device=dev)
        J_d = torch.tensor(J, dtype=torch.float32, device=dev).contiguous()
        rc = pkg._native.element_system_noalloc(S, r, n, tets, dminv, wvol, u_d, J_d, mu, lam,
                                                out)
        assert rc == 0
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        E, g = o[0], o[2:2 + r]
        Ku = o[2 + 2 * r:]
        K = np.zeros((r, r))
        K[np.triu_indices(r)] = Ku
        K = K + np.triu(K, 1).T
        assert abs(E - E_ref) <= TOL["E"] * max(1.0, abs(E_ref))
        assert rel(g, g_ref) < TOL["g"]
        assert rel(K, K_ref) < TOL["K"]
        # and against the FP64 oracle's elastic system at the same z
        Eo, go, Ko = om.eval(z)
        assert abs(E - Eo) <= TOL["E"] * max(1.0, abs(Eo))
        assert rel(g, go) < TOL["g"] and rel(K, Ko) < TOL["K"]
        assert close_elementwise(g, go, TOL["g"]) and close_elementwise(K, Ko, TOL["K"])
        if first is not None:
            assert not np.array_equal(o, first)  # a new input really was evaluated
        first = o.copy()
    ctx.close()


def _noalloc_rows(S, sms):
    """CTAs of the solver's element launch shape for S tets (one per 64 tets
    when S <= 128 * SMs, else one per 128, at most two per SM)."""
    et = 64 if S <= 64 * 2 * sms else 128
    return max(1, min((S + et - 1) // et, 2 * sms))


def test_noalloc_rejects_oversize_and_bad_arguments(pkg):
    import torch
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r, S, n = 64, 960000, 12
    nst = 2 + 2 * r + r * (r + 1) // 2 + 6
    if (_noalloc_rows(S, sms) + 1) * nst <= 524288:
        pytest.skip(f"{sms} SMs: 960,000 tets at r = 64 fit the scratch array here")
    # buffers of the full size with every index 0 < n / 3, so that the call
    # would stay in bounds even if it launched
    tets = torch.zeros((S, 4), dtype=torch.int32, device=dev)
    dminv = torch.zeros(9 * S, dtype=torch.float32, device=dev)
    wvol = torch.zeros(S, dtype=torch.float32, device=dev)
    u = torch.zeros(n, dtype=torch.float32, device=dev)
    J = torch.zeros((n, r), dtype=torch.float32, device=dev)
    out = torch.zeros(2 + 2 * r + r * (r + 1) // 2, dtype=torch.float64, device=dev)
    # r beyond the supported maximum (rejected before anything is read)
    rc = pkg._native.element_system_noalloc(1, 65, n, tets, dminv, wvol, u, J, 1.0, 1.0, out)
    assert rc == -1
    # partial sums beyond the fixed scratch size: 960,000 tets at r = 64
    rc = pkg._native.element_system_noalloc(S, r, n, tets, dminv, wvol, u, J, 1.0, 1.0, out)
    assert rc == -1
