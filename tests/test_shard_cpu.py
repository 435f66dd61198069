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


def _rank_oracle_main(rank, world, port, out_dir):
    # each rank builds the fused geometry from the same points (the shared
    # read-only input) and runs the CPU oracle's sweep over its own angles;
    # the ranks' fields are gathered over gloo
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, sw0 = _tiny_sweep()
        th, ph = shard.rank_angles(sw0.theta_deg, sw0.phi_deg, rank, world)
        sw = scenes.Sweep(theta_deg=th, phi_deg=ph, W=sw0.W, H=sw0.H, centre=sw0.centre,
                          extent=sw0.extent, freqs_hz=sw0.freqs_hz, max_bounces=sw0.max_bounces)
        S, gv, _, _ = oracle.build_geometry(sc, scenes.aggregation_views(sc, 48, 48), "fp32")
        eps = oracle.default_eps(gv)
        res = oracle.rcs_sweep(sc, sw, S, eps, eps, mode="fp32")
        mine = torch.from_numpy(np.stack([res.E.real, res.E.imag], -1).copy())
        parts = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(parts, mine)
        angs = torch.from_numpy(np.stack([th, ph], 1).copy())
        aparts = [torch.empty_like(angs) for _ in range(world)]
        dist.all_gather(aparts, angs)
        if rank == 0:
            np.savez(os.path.join(out_dir, "gathered.npz"),
                     E=np.concatenate([p.numpy() for p in parts]),
                     ang=np.concatenate([a.numpy() for a in aparts]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _tiny_sweep():
    sc = scenes.dihedral(1500, seed=19)
    sw = scenes._sweep_over(sc, [90.0, 90.0, 90.0], [0.0, 30.0, 60.0], 24, [3e9, 3.3e9], 2)
    return sc, sw


def test_two_gloo_ranks_run_the_oracle_on_their_shards():
    # the union of the ranks' fields, gathered, equals one process's sweep
    # over the union of their angles, bit for bit (angles are independent
    # problems over the same fused geometry)
    import torch.multiprocessing as mp
    import oracle
    world = 2
    with tempfile.TemporaryDirectory() as d:
        mp.spawn(_rank_oracle_main, args=(world, _free_port(), d), nprocs=world, join=True)
        g = np.load(os.path.join(d, "gathered.npz"))
    sc, sw0 = _tiny_sweep()
    ang = g["ang"]
    assert len(np.unique(ang[:, 1])) == world * sw0.n_angles
    sw = scenes.Sweep(theta_deg=ang[:, 0], phi_deg=ang[:, 1], W=sw0.W, H=sw0.H,
                      centre=sw0.centre, extent=sw0.extent, freqs_hz=sw0.freqs_hz,
                      max_bounces=sw0.max_bounces)
    S, gv, _, _ = oracle.build_geometry(sc, scenes.aggregation_views(sc, 48, 48), "fp32")
    eps = oracle.default_eps(gv)
    ref = oracle.rcs_sweep(sc, sw, S, eps, eps, mode="fp32")
    E = g["E"][..., 0] + 1j * g["E"][..., 1]
    assert np.abs(ref.E).max() > 0
    assert np.array_equal(E, ref.E)
