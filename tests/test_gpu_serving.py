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
