"""Continuous-batching server for monostatic RCS requests.

Requests of uneven size (point count, ray screen, angles, frequencies, bounce
limit) arrive over time.  The scheduler admits them, in arrival order, as soon
as an execution slot (a CUDA stream) and enough of the HBM budget are free, so
requests that arrive while others run join the GPU immediately and their
kernels overlap ("continuous").  The "static" policy is plain batching: it
admits a batch of up to n_slots queued requests only when the previous batch
has completed.  Each admitted request: points to the device, surfel radii
computed on the device when the request brings none, fused splat geometry
(reused from a resident cache when the same target was seen before), the
whole sweep, results back to pinned host memory, a completion event.
Latency = completion - arrival.  A request's device memory (the admission
charge) is the sum of the library's own workspace and buffer queries for its
sizes.

The scheduler (admission, queue, bookkeeping) is host logic independent of the
GPU; `GpuExecutor` is the device side, built only from the C-ABI calls.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass
class RcsRequest:
    rid: int
    scene_key: str
    pos: np.ndarray          # float32 [N,3]
    nrm: np.ndarray          # float32 [N,3]
    rad: Optional[np.ndarray]  # float32 [N], or None: computed on the device
    theta_deg: np.ndarray
    phi_deg: np.ndarray
    W: int
    freqs_hz: np.ndarray
    max_bounces: int
    view_W: int = 512
    arrival: float = 0.0

    @property
    def n_points(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class RcsResult:
    rid: int
    ok: bool
    error: str = ""
    E: Optional[np.ndarray] = None
    sigma: Optional[np.ndarray] = None
    arrival: float = 0.0
    admitted: float = 0.0
    finished: float = 0.0
    ray_bounces: int = 0
    host_ms: float = 0.0      # host time to issue the request's device work
    device_ms: float = 0.0    # device time from its first to its last operation

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def validate(req: RcsRequest) -> Optional[str]:
    """Reject malformed requests before they reach the device."""
    if req.pos.ndim != 2 or req.pos.shape[1] != 3 or req.pos.shape[0] < 1:
        return "points must be a non-empty [N,3] array"
    if req.nrm.shape != req.pos.shape or (req.rad is not None and
                                          req.rad.shape != (req.pos.shape[0],)):
        return "normals/radii do not match the points"
    if not (np.isfinite(req.pos).all() and np.isfinite(req.nrm).all() and
            (req.rad is None or np.isfinite(req.rad).all())):
        return "non-finite point data"
    if req.rad is None and req.pos.shape[0] < 17:
        return "radii computed on the device need at least 17 points"
    if len(req.theta_deg) < 1 or len(req.theta_deg) != len(req.phi_deg):
        return "angles"
    f = np.asarray(req.freqs_hz)
    if f.size < 1 or not np.all(np.isfinite(f)) or not np.all(f > 0):
        return "frequencies must be finite and > 0"
    if not (1 <= req.max_bounces <= 64) or req.W < 1 or req.view_W < 8:
        return "screen size or bounce limit out of range"
    return None


# The 8 aggregation views (theta 60/120 deg x phi 45/135/225/315 deg).
AGG_THETA = [60.0] * 4 + [120.0] * 4
AGG_PHI = [45.0, 135.0, 225.0, 315.0] * 2


def _agg_views(view_W: int):
    from . import api
    return [api.view_from_angles(t, p, [0.0, 0.0, 0.0], 1.0, view_W, view_W)
            for t, p in zip(AGG_THETA, AGG_PHI)]


def geometry_bytes(view_W: int, n_views: int = 8) -> int:
    """Resident fused geometry (splat planes, pyramids, slabs, view grid):
    the library's pe_geom_bytes for the aggregation views."""
    from . import _lib, api
    return int(_lib.load().pe_geom_bytes(n_views, api.views_to_array(_agg_views(view_W)[:n_views])))


def estimate(req: RcsRequest, geometry_cached: bool):
    """(transient, new_resident) device bytes of a request: what it holds
    while it runs, and the fused geometry it leaves resident if not cached.
    Every term is the library's own query for the request's sizes: the
    sweep's workspace (pe_rcs_sweep_workspace), the surfel attributes'
    (pe_point_attributes_workspace), the GFBs' and the fusion's
    (pe_build_gfb_workspace, pe_aggregate_workspace), the geometry blob
    (pe_geom_bytes); plus the points, the GFB buffers, the field and sigma,
    256 bytes of alignment per buffer and 64 KB for the allocator's
    rounding of a request's ~20 buffers (512-byte blocks)."""
    from . import _lib, api
    lib = _lib.load()
    n = req.n_points
    args = api.SweepArgs(req.theta_deg, req.phi_deg, req.W, req.W, [0.0, 0.0, 0.0], 1.0,
                         req.freqs_hz, req.max_bounces)
    A, F = len(req.theta_deg), len(req.freqs_hz)
    b = 28 * n + 3 * 256 + (64 << 10)                     # points, normals, radii; rounding
    if req.rad is None:
        b += int(lib.pe_point_attributes_workspace(n)) + 256
    b += int(args.workspace_bytes()) + 256                # the sweep
    b += A * F * (12 + 4) * 8 + 8 * 8 + 3 * 256           # field, sigma, counters
    resident = 0
    if not geometry_cached:
        vs = _agg_views(req.view_W)
        arr = api.views_to_array(vs)
        pix = 8 * req.view_W * req.view_W
        b += int(lib.pe_build_gfb_workspace(8, arr)) + pix * (16 + 1) + 3 * 256
        b += int(lib.pe_aggregate_workspace(8, arr, 256)) + 256
        resident = int(lib.pe_geom_bytes(8, arr)) + 256
    return int(b), int(resident)


def estimate_bytes(req: RcsRequest, geometry_cached: bool) -> int:
    """Total admission charge of a request (transient + new resident)."""
    t, r = estimate(req, geometry_cached)
    return t + r


class Scheduler:
    """FIFO admission under an HBM budget and a slot limit.

    executor must provide: start(req, slot) -> handle, poll(handle) -> bool,
    finish(handle) -> RcsResult, geometry_cached(scene_key) -> bool,
    evict(bytes_needed) -> bytes_freed (resident geometry), resident_bytes().
    """

    def __init__(self, executor, hbm_budget: int, n_slots: int = 4,
                 clock: Callable[[], float] = time.perf_counter, policy: str = "continuous"):
        if policy not in ("continuous", "static"):
            raise ValueError("policy: continuous or static")
        self.policy = policy
        self.ex = executor
        self.budget = int(hbm_budget)
        self.n_slots = int(n_slots)
        self.clock = clock
        self.queue: List[RcsRequest] = []
        self.running: Dict[int, tuple] = {}      # slot -> (req, handle, charge, admitted)
        self.results: List[RcsResult] = []
        self.in_use = 0
        self.cancelled: set = set()
        self.peak_in_use = 0
        self.max_running = 0

    # ---- submission -------------------------------------------------------
    def submit(self, req: RcsRequest) -> bool:
        err = validate(req)
        if err is None and estimate_bytes(req, False) > self.budget:
            err = "request needs more device memory than the whole budget"
        if err is not None:
            now = self.clock()
            self.results.append(RcsResult(req.rid, False, err, arrival=req.arrival,
                                          admitted=now, finished=now))
            return False
        self.queue.append(req)
        return True

    def cancel(self, rid: int) -> bool:
        """Cancel a queued request (running ones complete)."""
        for i, r in enumerate(self.queue):
            if r.rid == rid:
                del self.queue[i]
                now = self.clock()
                self.results.append(RcsResult(rid, False, "cancelled", arrival=r.arrival,
                                              admitted=now, finished=now))
                return True
        return False

    # ---- loop -------------------------------------------------------------
    def _free_slot(self) -> Optional[int]:
        for s in range(self.n_slots):
            if s not in self.running:
                return s
        return None

    def _admit(self):
        # plain batching admits a new batch only once the last one is done
        if self.policy == "static" and self.running:
            return
        while self.queue:
            slot = self._free_slot()
            if slot is None:
                return
            req = self.queue[0]
            charge, new_res = estimate(req, self.ex.geometry_cached(req.scene_key))
            resident = self.ex.resident_bytes()
            if self.in_use + resident + charge + new_res > self.budget:
                need = self.in_use + resident + charge + new_res - self.budget
                self.ex.evict(need)
                # the eviction may have taken this request's own (idle)
                # geometry: charge it again as the executor now holds it
                charge, new_res = estimate(req, self.ex.geometry_cached(req.scene_key))
                resident = self.ex.resident_bytes()
                if self.in_use + resident + charge + new_res > self.budget:
                    return          # wait for running requests to finish (FIFO)
            self.queue.pop(0)
            now = self.clock()
            try:
                h = self.ex.start(req, slot)
            except Exception as e:  # the device side refused this request
                self.results.append(RcsResult(req.rid, False, f"start failed: {e}",
                                              arrival=req.arrival, admitted=now, finished=now))
                continue
            self.running[slot] = (req, h, charge, now)
            self.in_use += charge
            self.max_running = max(self.max_running, len(self.running))
            self.peak_in_use = max(self.peak_in_use, self.in_use + self.ex.resident_bytes())

    def _reap(self):
        for slot in list(self.running):
            req, h, charge, adm = self.running[slot]
            try:
                done = self.ex.poll(h)
            except Exception as e:
                done = True
                h = ("failed", str(e))
            if not done:
                continue
            now = self.clock()
            if isinstance(h, tuple) and h and h[0] == "failed":
                res = RcsResult(req.rid, False, h[1])
            else:
                try:
                    res = self.ex.finish(h)
                except Exception as e:
                    res = RcsResult(req.rid, False, f"finish failed: {e}")
            res.arrival, res.admitted, res.finished = req.arrival, adm, now
            self.results.append(res)
            del self.running[slot]
            self.in_use -= charge

    def step(self):
        self._reap()
        self._admit()

    def idle(self) -> bool:
        return not self.queue and not self.running

    def run(self, requests: List[RcsRequest], t0: Optional[float] = None,
            poll_s: float = 2e-4) -> List[RcsResult]:
        """Replay requests at their arrival offsets (seconds after t0)."""
        t0 = self.clock() if t0 is None else t0
        pending = sorted((dataclasses.replace(r) for r in requests), key=lambda r: r.arrival)
        i = 0
        while i < len(pending) or not self.idle():
            now = self.clock() - t0
            while i < len(pending) and pending[i].arrival <= now:
                r = pending[i]
                r.arrival = t0 + r.arrival
                self.submit(r)
                i += 1
            self.step()
            if i < len(pending) and self.idle():
                time.sleep(max(0.0, min(poll_s * 10, pending[i].arrival - (self.clock() - t0))))
            else:
                time.sleep(poll_s)
        return self.results


# ----------------------------------------------------------------------------
# device side
# ----------------------------------------------------------------------------

class GpuExecutor:
    """Runs requests on CUDA streams through the C ABI, keeping fused
    geometry resident (LRU) by scene key."""

    def __init__(self, device="cuda:0", n_slots: int = 4):
        import torch
        from . import api, pipeline
        self.torch, self.api, self.pipe = torch, api, pipeline
        self.dev = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(n_slots)]
        self.geo: "OrderedDict[str, dict]" = OrderedDict()
        # the bounding sphere depends on the scene alone: computed once per
        # scene key (it is the largest host-side cost of a request)
        self.spheres: Dict[str, tuple] = {}

    def _sphere(self, req: RcsRequest):
        sp = self.spheres.get(req.scene_key)
        if sp is None:
            sp = _bounding_sphere(req.pos)
            self.spheres[req.scene_key] = sp
        return sp

    # geometry cache
    def geometry_cached(self, key: str) -> bool:
        return key in self.geo

    def resident_bytes(self) -> int:
        return sum(g["bytes"] for g in self.geo.values())

    def evict(self, need: int) -> int:
        freed = 0
        for key in list(self.geo):
            if freed >= need:
                break
            g = self.geo[key]
            if g["users"] == 0:
                freed += g["bytes"]
                del self.geo[key]
        return freed

    def start(self, req: RcsRequest, slot: int):
        torch, api, pipe = self.torch, self.api, self.pipe
        s = self.streams[slot]
        hp = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
              for a in ((req.pos, req.nrm) if req.rad is None else (req.pos, req.nrm, req.rad))]
        t_host = time.perf_counter()
        t0 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            t0.record(s)
            pos, nrm = [t.to(self.dev, non_blocking=True) for t in hp[:2]]
            if req.rad is None:
                rad, _ = api.point_attributes(pos, 8, 16, None, radius=True, normal=False,
                                              stream=s)
            else:
                rad = hp[2].to(self.dev, non_blocking=True)
            g = self.geo.get(req.scene_key)
            c, r = self._sphere(req)
            if g is None:
                gv = pipe.views_from_angles(AGG_THETA, AGG_PHI, c, r * 1.02, req.view_W,
                                            req.view_W)
                prm = pipe.default_params(req.pos, gv)
                geom, _ = pipe.build_geometry(pos, nrm, rad, gv, prm, stream=s)
                ready = torch.cuda.Event()
                ready.record(s)
                g = {"geom": geom, "prm": prm, "ready": ready, "users": 0,
                     "bytes": geometry_bytes(req.view_W)}
                self.geo[req.scene_key] = g
            else:
                s.wait_event(g["ready"])
                self.geo.move_to_end(req.scene_key)
            g["users"] += 1
            args = api.SweepArgs(req.theta_deg, req.phi_deg, req.W, req.W, c, r * 1.02,
                                 req.freqs_hz, req.max_bounces)
            stats = torch.zeros(8, dtype=torch.int64, device=self.dev)
            E, sig = api.rcs_sweep(args, pos, nrm, rad, g["geom"] if req.max_bounces > 1 else None,
                                   g["prm"], stream=s, stats=stats)
            hE = torch.empty(E.shape, dtype=E.dtype).pin_memory()
            hS = torch.empty(sig.shape, dtype=sig.dtype).pin_memory()
            hst = torch.empty(8, dtype=torch.int64).pin_memory()
            hE.copy_(E, non_blocking=True)
            hS.copy_(sig, non_blocking=True)
            hst.copy_(stats, non_blocking=True)
            done = torch.cuda.Event(enable_timing=True)
            done.record(s)
        return {"req": req, "done": done, "t0": t0, "host_ms": (time.perf_counter() - t_host) * 1e3,
                "keep": (pos, nrm, rad, E, sig, stats, args, hp),
                "hE": hE, "hS": hS, "hst": hst, "g": g}

    def poll(self, h) -> bool:
        return h["done"].query()

    def finish(self, h) -> RcsResult:
        h["g"]["users"] -= 1
        E = h["hE"].numpy()
        st = h["hst"].numpy()
        return RcsResult(h["req"].rid, True, E=E[..., 0] + 1j * E[..., 1],
                         sigma=h["hS"].numpy().copy(), ray_bounces=int(st[0] + st[1]),
                         host_ms=h["host_ms"], device_ms=h["t0"].elapsed_time(h["done"]))


def _bounding_sphere(pos: np.ndarray):
    p = pos.astype(np.float64)
    c = 0.5 * (p.min(axis=0) + p.max(axis=0))
    return c, float(np.sqrt(((p - c) ** 2).sum(axis=1).max()))


# ----------------------------------------------------------------------------
# workloads and statistics
# ----------------------------------------------------------------------------

def loguniform(rng, lo, hi):
    return float(math.exp(rng.uniform(math.log(lo), math.log(hi))))


def make_requests(scene_pool: List, n: int, rate_hz: float, seed: int = 5,
                  max_angles: int = 32, max_freqs: int = 16, screens=(128, 256, 512),
                  max_bounces: int = 3, view_W: int = 256) -> List[RcsRequest]:
    """Poisson arrivals; per request a target from the pool, a power-of-two
    screen, log-uniform angle and frequency counts, uniform bounce limit."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        key, sc = scene_pool[int(rng.integers(0, len(scene_pool)))]
        A = max(1, int(round(loguniform(rng, 1, max_angles))))
        F = max(1, int(round(loguniform(rng, 1, max_freqs))))
        W = int(screens[int(rng.integers(0, len(screens)))])
        mb = int(rng.integers(1, max_bounces + 1))
        th = np.full(A, float(rng.uniform(30.0, 150.0)))
        ph = np.sort(rng.uniform(0.0, 360.0, size=A))
        f0 = rng.uniform(2e9, 10e9)
        freqs = f0 * (1.0 + 0.2 * np.arange(F) / max(F - 1, 1))
        out.append(RcsRequest(i, key, sc.pos, sc.nrm, sc.rad, th, ph, W, freqs, mb,
                              view_W=view_W, arrival=t))
    return out


def make_c5_requests(n: int, rate_hz: float, seed: int = 5, max_points: int = 4_000_000,
                     view_W: int = 256) -> List[RcsRequest]:
    """The serving mix: Poisson arrivals; per request its own target
    (scenes.c5_target: one of the standard workloads' shapes at a random
    size) of N ~ logU(10k, max_points) points with exact normals and no
    radii (the server computes them), a power-of-two screen of 128^2 to
    4096^2 rays (log-uniform), A ~ logU(1, 720) azimuths at one elevation,
    F ~ logU(1, 128) frequencies on a uniform grid over 20 % of a band
    starting at 2-12 GHz, mb ~ U{1..5}."""
    import scenes
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_hz)
        N = int(round(loguniform(rng, 10_000, max_points)))
        pos, nrm, kind = scenes.c5_target(seed * 100_003 + i, N)
        W = int(2 ** int(rng.integers(7, 13)))
        A = max(1, int(round(loguniform(rng, 1, 720))))
        F = max(1, int(round(loguniform(rng, 1, 128))))
        mb = int(rng.integers(1, 6))
        th = np.full(A, float(rng.uniform(30.0, 150.0)))
        ph = float(rng.uniform(0.0, 360.0)) + np.arange(A) * (360.0 / A)
        f0 = float(rng.uniform(2e9, 12e9))
        freqs = f0 * (1.0 + 0.2 * np.arange(F) / max(F - 1, 1))
        out.append(RcsRequest(i, f"c5-{seed}-{i}-{kind}", pos, nrm, None, th, ph, W, freqs, mb,
                              view_W=view_W, arrival=t))
    return out


def latency_stats(results: List[RcsResult]) -> dict:
    ok = [r for r in results if r.ok]
    if not ok:
        return {"n": 0}
    lat = np.array([r.latency for r in ok])
    span = max(r.finished for r in ok) - min(r.arrival for r in ok)
    return {"n": len(ok), "failed": len(results) - len(ok),
            "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3),
            "requests_per_s": len(ok) / span if span > 0 else None,
            "ray_bounces_per_s": sum(r.ray_bounces for r in ok) / span if span > 0 else None,
            "host_ms_p50": float(np.percentile([r.host_ms for r in ok], 50)),
            "device_ms_p50": float(np.percentile([r.device_ms for r in ok], 50))}
