"""The multi-GPU partition's host logic on CPU: two gloo ranks shard a
monostatic sweep (disjoint angles that together form the denser sweep) and
reduce their unit counts (sum) and times (max) into the job's throughput, as
bench.py does under torchrun.  Also the one-rank path."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import scenes  # noqa: E402
from paper_2408_15583_gb300 import shard  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sw = scenes.workload_sphere(n_points=2000, W=64, view_W=64, n_angles=360, n_freq=2).sweep
        th, ph = shard.rank_angles(sw.theta_deg, sw.phi_deg, rank, world)
        units = 1000.0 * (rank + 1)          # ranks count different work
        t_ms = 10.0 + 5.0 * rank             # the slowest rank decides
        u, t, v = shard.job_throughput(units, t_ms)
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), th=th, ph=ph, u=u, t=t, v=v)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_main, args=(world, _free_port(), d), nprocs=world, join=True)
        r = [np.load(os.path.join(d, f"r{k}.npz")) for k in range(world)]
        sw = scenes.workload_sphere(n_points=2000, W=64, view_W=64, n_angles=360, n_freq=2).sweep
        # each rank keeps the one-GPU angle count (weak scaling), angles are
        # disjoint and together form the sweep at half the phi step
        for k in range(world):
            assert r[k]["ph"].shape == sw.phi_deg.shape
            assert np.array_equal(r[k]["th"], sw.theta_deg)
        allp = np.sort(np.concatenate([r[k]["ph"] for k in range(world)]))
        assert len(np.unique(allp)) == world * len(sw.phi_deg)
        step = shard.phi_step(sw.phi_deg)
        assert np.allclose(np.diff(allp), step / world)
        # reductions: sum of units, max of times, identical on every rank
        for k in range(world):
            assert float(r[k]["u"]) == 1000.0 + 2000.0
            assert float(r[k]["t"]) == 15.0
            assert float(r[k]["v"]) == pytest.approx(3000.0 / 0.015)


def test_one_rank_is_the_plain_sweep():
    sw = scenes.workload_composite(n_points=3000).sweep
    th, ph = shard.rank_angles(sw.theta_deg, sw.phi_deg, 0, 1)
    assert np.array_equal(th, sw.theta_deg) and np.array_equal(ph, sw.phi_deg)
    u, t, v = shard.job_throughput(500.0, 250.0)
    assert (u, t) == (500.0, 250.0) and v == pytest.approx(2000.0)
    with pytest.raises(ValueError):
        shard.rank_angles(sw.theta_deg, sw.phi_deg, 2, 2)
    assert shard.phi_step([45.0]) == 1.0
    assert shard.phi_step(np.arange(0.0, 360.0, 5.0)) == 5.0
