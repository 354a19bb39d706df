"""GPU parity of E, g, K for free bodies with affine modes across subspace
and decoder shapes, up to the full torus_drop_200k workload (sampled-free:
the oracle evaluates the whole reduced system at one point)."""
import dataclasses

import numpy as np
import pytest

from oracle.reduced import model_from_problem
from workloads import build_problem, CONFIGS
from tests.gpu_util import rel, random_qbar, round_bf16, assert_close, UNIT_ROUNDOFF

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(E=1e-10, g=1e-8, K=1e-8), "fp32": dict(E=1e-4, g=1e-3, K=1e-3),
       "bf16": dict(E=1e-4, g=1e-3, K=2e-3)}


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


def _case(name):
    if name == "full":
        return build_problem("torus_drop_200k")
    r, hidden, h = {"r32_h512": (32, (512, 512), 0.06), "r6_h512": (6, (512,), 0.06),
                    "r32_h24": (32, (24, 24), 0.06)}[name]
    c = dataclasses.replace(CONFIGS["tiny_torus_drop"], r=r, hidden=hidden, h=h)
    return build_problem(c)


@pytest.mark.parametrize("name", ["r6_h512", "r32_h24", "r32_h512", "full"])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_system_parity_across_shapes(pkg, name, prec):
    p = _case(name)
    c = p.config
    pr = p if prec != "bf16" else dataclasses.replace(p, Ws=[*p.Ws[:-1], round_bf16(p.Ws[-1])])
    m = model_from_problem(pr)
    ctx = pkg.context_from_problem(p, precision=prec)
    qbar = p.X0.ravel() + c.dt * p.v0 + c.dt ** 2 * np.tile(c.gravity, p.nv)
    ctx.set_dynamics(c.dt, qbar)
    m.set_dynamics(c.dt, qbar)
    r = m.r
    z = np.random.default_rng(3).standard_normal(r) * 0.05
    E, g, K = ctx.eval(z)
    E_ref, g_ref, K_ref = m.eval(z)
    t = TOL[prec]
    print(name, prec, "E", abs(E - E_ref) / max(1, abs(E_ref)), "g", rel(g, g_ref),
          "g_nn", rel(g[:c.r], g_ref[:c.r]), "g_aff", rel(g[c.r:], g_ref[c.r:]), "K", rel(K, K_ref))
    assert abs(E - E_ref) <= t["E"] * max(1.0, abs(E_ref)), (E, E_ref)
    assert_close(g, g_ref, t["g"], u=UNIT_ROUNDOFF[prec])
    assert_close(K, K_ref, t["K"], u=UNIT_ROUNDOFF["bf16_operands" if prec == "bf16" else prec])
    ctx.close()
