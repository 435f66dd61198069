"""Continuous batching on the GPU: requests overlap on the device, and each
request's result in the mix equals its result alone (the kernels and their
reductions are deterministic, so equality is exact; the stated field
tolerance is checked too)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import scenes  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return [("dihedral", scenes.dihedral(3000, seed=2)), ("sphere", scenes.sphere(5000)),
            ("trihedral", scenes.trihedral(3000, a=0.3))]


def _field_err(E, Eref):
    d = np.sqrt((np.abs(E - Eref) ** 2).sum(axis=-1))
    r = np.sqrt((np.abs(Eref) ** 2).sum(axis=-1))
    return d / np.maximum(r, 1e-3 * r.max())


def test_results_identical_alone_and_in_the_mix(pool):
    from paper_2408_15583_gb300 import serve
    reqs = serve.make_requests(pool, 10, rate_hz=1e6, seed=3, max_angles=6, max_freqs=4,
                               screens=(32, 64), max_bounces=3, view_W=64)
    mix = serve.Scheduler(serve.GpuExecutor(n_slots=4), hbm_budget=8 << 30, n_slots=4)
    res_mix = {r.rid: r for r in mix.run(reqs)}
    assert all(r.ok for r in res_mix.values()), [r.error for r in res_mix.values()]
    assert mix.max_running > 1                      # requests overlapped on the GPU
    for rq in reqs:
        alone = serve.Scheduler(serve.GpuExecutor(n_slots=1), hbm_budget=8 << 30, n_slots=1)
        r = alone.run([rq])[0]
        assert r.ok, r.error
        m = res_mix[rq.rid]
        assert np.array_equal(r.E, m.E)
        assert _field_err(m.E, r.E).max() < 1e-3
        assert np.all(np.isfinite(m.sigma))


def test_budget_respected_with_resident_geometry(pool):
    from paper_2408_15583_gb300 import serve
    reqs = serve.make_requests(pool, 8, rate_hz=1e6, seed=4, max_angles=4, max_freqs=2,
                               screens=(32,), max_bounces=2, view_W=64)
    one = max(serve.estimate_bytes(r, False) for r in reqs)
    s = serve.Scheduler(serve.GpuExecutor(n_slots=3), hbm_budget=2 * one, n_slots=3)
    res = s.run(reqs)
    assert all(r.ok for r in res)
    assert s.peak_in_use <= s.budget


def test_c5_requests_device_radii_and_policies():
    # requests that bring no radii (the server computes them on the device,
    # pe_point_attributes), served one at a time, in plain batches and
    # continuously: every policy gives every request the same field, bit for
    # bit, as the direct library calls on the same inputs
    from paper_2408_15583_gb300 import api, pipeline, serve
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = serve.make_c5_requests(6, rate_hz=1e6, seed=7, max_points=60_000, view_W=64)
    for r in reqs:          # keep the screens and sweeps small
        r.W = min(r.W, 128)
        r.theta_deg, r.phi_deg = r.theta_deg[:5], r.phi_deg[:5]
        r.freqs_hz = r.freqs_hz[:6]
    runs = {}
    for name, slots, policy in (("one", 1, "continuous"), ("static", 3, "static"),
                                ("cont", 3, "continuous")):
        s = serve.Scheduler(serve.GpuExecutor(n_slots=slots), hbm_budget=40 << 30, n_slots=slots,
                            policy=policy)
        res = {r.rid: r for r in s.run(reqs)}
        assert all(r.ok for r in res.values()), [r.error for r in res.values()]
        runs[name] = res
    for rq in reqs:
        dev = "cuda:0"
        pos = torch.from_numpy(rq.pos).to(dev)
        nrm = torch.from_numpy(rq.nrm).to(dev)
        rad, _ = api.point_attributes(pos, 8, 16, None, radius=True, normal=False)
        c, r = serve._bounding_sphere(rq.pos)
        gv = pipeline.views_from_angles(serve.AGG_THETA, serve.AGG_PHI, c, r * 1.02, rq.view_W,
                                        rq.view_W)
        prm = pipeline.default_params(rq.pos, gv)
        geom, _ = pipeline.build_geometry(pos, nrm, rad, gv, prm)
        args = api.SweepArgs(rq.theta_deg, rq.phi_deg, rq.W, rq.W, c, r * 1.02, rq.freqs_hz,
                             rq.max_bounces)
        E, _ = api.rcs_sweep(args, pos, nrm, rad, geom if rq.max_bounces > 1 else None, prm)
        api.stream_check()
        Eh = E.cpu().numpy()
        Eh = Eh[..., 0] + 1j * Eh[..., 1]
        for name in runs:
            assert np.array_equal(runs[name][rq.rid].E, Eh), (name, rq.rid)


def test_admission_charge_bounds_the_devices_allocations():
    # the charge the scheduler admits a request with (the library's sizes)
    # covers what the executor actually allocates for it
    from paper_2408_15583_gb300 import serve
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = serve.make_c5_requests(3, rate_hz=1e6, seed=11, max_points=300_000, view_W=128)
    for rq in reqs:
        rq.theta_deg, rq.phi_deg = rq.theta_deg[:40], rq.phi_deg[:40]
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        ex = serve.GpuExecutor(n_slots=1)
        s = serve.Scheduler(ex, hbm_budget=100 << 30, n_slots=1)
        res = s.run([rq])
        assert res[0].ok, res[0].error
        torch.cuda.synchronize()
        used = torch.cuda.max_memory_allocated() - base
        t, r = serve.estimate(rq, False)
        assert used <= t + r, (rq.rid, used, t + r)
