"""Parity at the largest workload's full size, in the launch configuration
bench.py times (BF16 form): block_twist_960k (101x41x41 nodes, 960,000
tets, n = 509,343, r = 64, decoder 64-1024x3-509343).

The decoder output (x, J) is compared on 4,096 sampled rows, which the FP64
oracle computes one by one (rows of the last layer); the reduced system
(E, g, K) is compared with the elastic part restricted to 4,096 sampled
tets (a cubature set) while the inertia term still runs over all 509,343
rows.  The oracle uses the BF16-rounded output-layer weights that the BF16
form stores (tolerances as in test_gpu_tensor_core.py)."""
import dataclasses

import numpy as np
import pytest

from oracle.decoder import Decoder
from oracle.reduced import ReducedModel
from workloads import build_problem
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


def test_block_960k_sampled_rows_and_sampled_cubature_system(pkg):
    p = build_problem("block_twist_960k")
    c = p.config
    rng = np.random.default_rng(31)
    tets = np.sort(rng.choice(p.ne, 4096, replace=False)).astype(np.int32)
    w = np.ones(tets.shape[0])
    ctx = pkg.context_from_problem(p, precision="bf16")
    ctx.set_cubature(tets, w)
    tg = p.targets(40)
    ctx.set_constraints(None, tg)
    qbar = p.X0.ravel() + 1e-3 * rng.standard_normal(p.n)
    ctx.set_dynamics(c.dt, qbar)
    z = 0.3 * rng.standard_normal(c.r)
    x, J = ctx.decode(z)
    E, g, K = ctx.eval(z)
    ctx.close()

    Wb = [*p.Ws[:-1], round_bf16(p.Ws[-1])]
    dec = Decoder(Wb, p.bs, c.out_scale)
    rows = np.sort(rng.choice(p.n, 4096, replace=False))
    o, Jr = dec.out_jac(z, rows)
    cd = set((3 * p.cnodes[:, None] + np.arange(3)).ravel().tolist())
    free = np.array([k not in cd for k in rows])
    assert_close(x[rows][free] - p.X0.ravel()[rows][free], o[free], 1e-5)
    assert_close(J[rows][free], Jr[free], 1e-5)
    assert np.all(J[rows][~free] == 0.0)

    m = ReducedModel(p.X0, p.tets, dec, c.youngs, c.poisson, c.density, c.gravity,
                     tets, w, p.cnodes)
    m.set_targets(tg)
    m.set_dynamics(c.dt, qbar)
    E0, g0, K0 = m.eval(z)
    assert abs(E - E0) <= 2e-4 * max(1.0, abs(E0)), (E, E0)
    assert_close(g, g0, 2e-4)
    assert_close(K, K0, 5e-3, u=UNIT_ROUNDOFF["bf16_operands"])  # BF16 Gram operands
