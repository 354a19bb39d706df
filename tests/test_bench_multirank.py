"""The N > 1 path of bench.py (independent replicas, one per rank): the job
time is the maximum over ranks and the value counts every rank's steps.
Two gloo ranks on the CPU stand in for two GPUs; rendezvous on 127.0.0.1."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 * (rank + 1)  # the second rank is the slower replica
    job_ms = bench.aggregate_time(local_ms, world)
    value = bench.job_value(world, 10, job_ms)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{job_ms} {value}")
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_steps(tmp_path):
    world, port = 2, _free_port()
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for rank in range(world):
        job_ms, value = map(float, (tmp_path / f"r{rank}.txt").read_text().split())
        assert job_ms == pytest.approx(200.0)
        assert value == pytest.approx(2 * 10 / 0.2)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_time(123.0, 1) == 123.0
    assert bench.job_value(1, 50, 1000.0) == pytest.approx(50.0)


def test_bench_lipschitz_estimate_is_eq7():
    """bench.py's Eq. 7 estimate (measurement code of the learned-subspace
    comparison) against the oracle's pair loop, and against the closed form of
    an affine Hessian field Ht(z) = z_0 A (the estimate is ||A||_F)."""
    import numpy as np
    import torch
    sys.path.insert(0, ROOT)
    import bench
    from oracle.training import lipschitz_estimate
    rng = np.random.default_rng(5)
    Z = rng.standard_normal((12, 4))
    H = rng.standard_normal((12, 4, 4))
    H = H + np.swapaxes(H, 1, 2)
    ref = lipschitz_estimate(torch.tensor(H), torch.tensor(Z))
    assert bench.lipschitz_estimate(H, Z) == pytest.approx(ref, rel=1e-12)
    A = rng.standard_normal((4, 4))
    Z1 = np.zeros((6, 4))
    Z1[:, 0] = rng.standard_normal(6)
    H1 = Z1[:, 0, None, None] * A[None]
    assert bench.lipschitz_estimate(H1, Z1) == pytest.approx(np.linalg.norm(A), rel=1e-12)
