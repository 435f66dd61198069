"""Host logic of the continuous-batching server, with a fake executor: no GPU.

Failures are injected on the host (a start that raises, a poll that raises,
malformed requests, cancellation); nothing here touches a device.
"""
import numpy as np
import pytest

from paper_2408_15583_gb300.serve import (RcsRequest, RcsResult, Scheduler, estimate_bytes,
                                          geometry_bytes, latency_stats, validate)


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each request 'runs' for 1 + N/1e5 fake seconds; geometry is cached."""

    def __init__(self, clock, fail_start=(), fail_poll=()):
        self.clock = clock
        self.geo = {}
        self.fail_start = set(fail_start)
        self.fail_poll = set(fail_poll)
        self.started = []
        self.max_concurrent = 0
        self.live = 0

    def geometry_cached(self, key):
        return key in self.geo

    def resident_bytes(self):
        return sum(self.geo.values())

    def evict(self, need):
        freed = 0
        for k in list(self.geo):
            if freed >= need:
                break
            freed += self.geo.pop(k)
        return freed

    def start(self, req, slot):
        if req.rid in self.fail_start:
            raise RuntimeError("injected start failure")
        self.geo.setdefault(req.scene_key, geometry_bytes(req.view_W))
        self.started.append((req.rid, slot, self.clock()))
        self.live += 1
        self.max_concurrent = max(self.max_concurrent, self.live)
        return {"req": req, "end": self.clock() + 1.0 + req.n_points / 1e5}

    def poll(self, h):
        if h["req"].rid in self.fail_poll:
            raise RuntimeError("injected device error")
        return self.clock() >= h["end"]

    def finish(self, h):
        self.live -= 1
        r = h["req"]
        return RcsResult(r.rid, True, E=np.full((1,), float(r.rid)), ray_bounces=r.n_points)


def req(rid, n=1000, key="a", W=64, A=2, F=2, mb=2, arrival=0.0, nan=False):
    pos = np.random.default_rng(rid).normal(size=(n, 3)).astype(np.float32)
    if nan:
        pos[0, 0] = np.nan
    return RcsRequest(rid, key, pos, np.tile(np.float32([0, 0, 1]), (n, 1)),
                      np.full(n, 0.01, np.float32), np.full(A, 90.0), np.linspace(0, 90, A),
                      W, np.linspace(1e9, 2e9, F), mb, view_W=64, arrival=arrival)


def drive(s, clock, requests, dt=0.05, t_end=200.0):
    pending = sorted(requests, key=lambda r: r.arrival)
    i = 0
    budget_ok = True
    while clock.t < t_end and (i < len(pending) or not s.idle()):
        while i < len(pending) and pending[i].arrival <= clock.t:
            s.submit(pending[i])
            i += 1
        s.step()
        budget_ok &= s.in_use + s.ex.resident_bytes() <= s.budget
        clock.t += dt
    return budget_ok


def test_validation_rejects_malformed():
    assert validate(req(0)) is None
    assert "non-finite" in validate(req(1, nan=True))
    r = req(2)
    r.freqs_hz = np.array([0.0])
    assert "frequencies" in validate(r)


def test_continuous_admission_under_budget_and_slots():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    one = estimate_bytes(req(0), False)
    s = Scheduler(ex, hbm_budget=3 * one, n_slots=4, clock=clock)
    reqs = [req(i, arrival=0.3 * i, key=f"s{i % 3}") for i in range(12)]
    assert drive(s, clock, reqs)
    assert sorted(r.rid for r in s.results if r.ok) == list(range(12))
    # at most as many concurrent requests as the budget allows (3 fit), never more slots
    assert 1 < ex.max_concurrent <= 3
    # FIFO admission order
    assert [rid for rid, _, _ in ex.started] == sorted(rid for rid, _, _ in ex.started)
    # requests that arrived while others ran were admitted before those finished
    first_end = min(r.finished for r in s.results)
    assert sum(1 for _, _, t in ex.started if t < first_end) >= 2


def test_oversized_and_malformed_requests_fail_cleanly():
    clock = FakeClock()
    s = Scheduler(FakeExecutor(clock), hbm_budget=estimate_bytes(req(0), False), n_slots=2,
                  clock=clock)
    big = req(1, W=4096, A=64)
    assert not s.submit(big)
    assert not s.submit(req(2, nan=True))
    assert s.submit(req(3))
    drive(s, clock, [])
    res = {r.rid: r for r in s.results}
    assert not res[1].ok and "budget" in res[1].error
    assert not res[2].ok and "non-finite" in res[2].error
    assert res[3].ok


def test_cancel_and_injected_device_failures():
    clock = FakeClock()
    ex = FakeExecutor(clock, fail_start={1}, fail_poll={2})
    s = Scheduler(ex, hbm_budget=1 << 40, n_slots=1, clock=clock)
    for i in range(5):
        s.submit(req(i))
    assert s.cancel(4)
    assert not s.cancel(99)
    drive(s, clock, [])
    res = {r.rid: r for r in s.results}
    assert res[0].ok and res[3].ok
    assert not res[1].ok and "start failed" in res[1].error
    assert not res[2].ok and "injected device error" in res[2].error
    assert not res[4].ok and res[4].error == "cancelled"
    assert s.in_use == 0 and s.idle()


def test_resident_geometry_is_evicted_for_new_work():
    clock = FakeClock()
    ex = FakeExecutor(clock)
    one = estimate_bytes(req(0), False)
    s = Scheduler(ex, hbm_budget=one + geometry_bytes(64) * 2, n_slots=1, clock=clock)
    reqs = [req(i, key=f"scene{i}", arrival=float(i) * 3) for i in range(6)]
    assert drive(s, clock, reqs)
    assert all(r.ok for r in s.results)
    assert ex.resident_bytes() <= s.budget


def test_latency_stats():
    rs = [RcsResult(i, True, arrival=0.0, finished=0.1 * (i + 1), ray_bounces=10) for i in range(10)]
    st = latency_stats(rs)
    assert abs(st["p50_ms"] - 550.0) < 1e-6 and st["n"] == 10


def test_static_batches_wait_for_the_whole_batch():
    # plain batching: a new batch of up to n_slots requests starts only when
    # every request of the previous batch has completed
    clock = FakeClock()
    ex = FakeExecutor(clock)
    s = Scheduler(ex, hbm_budget=100 * estimate_bytes(req(0), False), n_slots=3, clock=clock,
                  policy="static")
    reqs = [req(i, n=1000 * (1 + i % 4), arrival=0.1 * i, key=f"s{i}") for i in range(9)]
    assert drive(s, clock, reqs)
    done = {r.rid: r for r in s.results if r.ok}
    assert sorted(done) == list(range(9))
    starts = sorted(t for _, _, t in ex.started)
    for rid, _, t in ex.started:
        # every request that started before this one's batch has finished by then
        earlier = [r for r in done.values() if r.admitted < t]
        assert all(r.finished <= t + 1e-9 for r in earlier)
    assert ex.max_concurrent <= 3
    with pytest.raises(ValueError):
        Scheduler(ex, 1, policy="greedy")


def test_admission_charge_is_the_librarys_own_sizes():
    # the sweep term of a 4096^2, 720-angle request is the library's
    # pe_rcs_sweep_workspace; an uncached target adds its fusion workspace and
    # the resident geometry blob (pe_geom_bytes)
    from paper_2408_15583_gb300 import _lib, api
    from paper_2408_15583_gb300 import serve
    lib = _lib.load()
    big = req(0, W=4096, A=720, F=128, mb=5)
    big.rad = None
    t_c, r_c = serve.estimate(big, True)
    t_u, r_u = serve.estimate(big, False)
    args = api.SweepArgs(big.theta_deg, big.phi_deg, 4096, 4096, [0, 0, 0], 1.0, big.freqs_hz, 5)
    assert t_c >= args.workspace_bytes() and r_c == 0
    assert t_c >= lib.pe_point_attributes_workspace(big.n_points)
    arr = api.views_to_array(serve._agg_views(big.view_W))
    assert r_u == lib.pe_geom_bytes(8, arr) + 256 == geometry_bytes(big.view_W) + 256
    assert t_u - t_c >= lib.pe_aggregate_workspace(8, arr, 256)
    assert t_c < 20 << 30          # the sweep's angle batch keeps it near 16 GB


def test_c5_request_mix():
    from paper_2408_15583_gb300.serve import make_c5_requests
    reqs = make_c5_requests(40, rate_hz=10.0, seed=3, max_points=200_000)
    assert len({r.scene_key for r in reqs}) == 40          # every request its own target
    for r in reqs:
        assert validate(r) is None and r.rad is None
        assert 9_990 <= r.n_points <= 200_000
        assert r.W in (128, 256, 512, 1024, 2048, 4096)
        assert 1 <= len(r.theta_deg) <= 720 and 1 <= len(r.freqs_hz) <= 128
        assert 1 <= r.max_bounces <= 5
    arr = [r.arrival for r in reqs]
    assert arr == sorted(arr) and arr[0] > 0
