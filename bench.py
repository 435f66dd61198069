#!/usr/bin/env python3
"""Benchmark of the SBR-on-points hot path on GB300.

One step = the whole path for one synthetic target: splat the points into
the 8 aggregation views (GFBs), fuse them into splats, then the full
monostatic sweep (per angle: incidence screen, splat for bounce 1, bounces
2..mb through the splats, visibility, PO field over all frequencies, sigma).

Printed (rank 0): one JSON line with ray-bounces/s (executed intersection
queries, shadow rays included) as `value`, RCS samples/s beside it, the
end-to-end figure through the C ABI with host buffers, the roofline of the
dominant kernel, the CPU oracle's rate on a bounded sample, clocks and the
number of kernels launched.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload sphere|dihedral|composite]
  python bench.py --impl reference ...   (the CPU oracle, timed on the host)
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def make_workload(name):
    if name == "sphere":
        wl = scenes.workload_sphere()
        desc = dict(workload="PEC sphere a=1 m, 200k Fibonacci points, 1024^2 rays, 64 freqs "
                             "8-12 GHz, 360 azimuths, mb=2, 8 GFB views 512^2",
                    points=200_000, rays=1024 * 1024, freqs=64, angles=360, max_bounces=2)
    elif name == "dihedral":
        wl = scenes.workload_dihedral()
        desc = dict(workload="PEC dihedral 0.5 m, 10k points, 128^2 rays, 3 GHz, 91 azimuths, "
                             "mb=2, 8 GFB views 512^2",
                    points=10_000, rays=128 * 128, freqs=1, angles=91, max_bounces=2)
    elif name == "composite":
        wl = scenes.workload_composite()
        desc = dict(workload="composite trihedral+plate+cylinder, 1M points (noise lambda/50, "
                             "PCA normals), 2048^2 rays, 10 GHz, 72 azimuths, mb=5, "
                             "8 GFB views 512^2",
                    points=1_000_000, rays=2048 * 2048, freqs=1, angles=72, max_bounces=5)
    elif name == "octar":
        wl = scenes.workload_octar()
        W = wl.sweep.W
        desc = dict(workload=f"OctAR (three orthogonal 20 m plates = 8 trihedrals), 50k points, "
                             f"{W}^2 rays (lambda/10), 500 MHz, theta 60 deg, 360 azimuths, mb=3, "
                             "8 GFB views 512^2",
                    points=wl.scene.n, rays=W * W, freqs=1, angles=360, max_bounces=3,
                    paper_context="3-bounce MBC about 30 ms per angle, EM field under 1 ms per "
                                  "angle, GFB preprocessing 2.44 s (hardware not stated)")
    else:
        raise SystemExit(f"unknown workload {name}")
    return wl, desc


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"pe_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_gpu(args, rank, world, local_rank):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_15583_gb300 import _lib, api, pipeline, shard

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    lib = _lib.load()
    wl, desc = make_workload(args.workload)
    sc, sw, vd = wl.scene, wl.sweep, wl.views
    if world > 1:
        # weak scaling: this rank's interleave of a sweep `world` times
        # denser in phi (angles are independent; nothing is exchanged)
        import dataclasses
        th, ph = shard.rank_angles(sw.theta_deg, sw.phi_deg, rank, world)
        sw = dataclasses.replace(sw, theta_deg=th, phi_deg=ph)
    stream = torch.cuda.current_stream()

    pos, nrm, rad = pipeline.scene_to_device(sc, dev)
    gv = pipeline.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, vd.W, vd.H)
    prm = pipeline.default_params(sc.pos, gv)
    sargs = api.SweepArgs.from_sweep(sw)
    ws = api.workspace(sargs.workspace_bytes(), dev)
    geom = api.alloc_geom(gv, dev)
    A, F = sw.n_angles, sw.n_freq
    E = torch.empty((A, F, 2, 3, 2), dtype=torch.float64, device=dev)
    sig = torch.empty((A, F, 2, 2), dtype=torch.float64, device=dev)
    stats = torch.zeros(8, dtype=torch.int64, device=dev)
    gfb_ws = None

    # the incidence splat takes the points in a spatially coherent order,
    # computed from the step's points inside the step
    order = torch.empty(sc.n, dtype=torch.int32, device=dev)
    sargs.set_point_order(order)

    def step(p, n, r, st=None):
        g = api.build_gfb(gv, p, n, r, 0, 0.0, outputs=("nd", "mask"))
        api.aggregate_views(gv, g["nd"], g["mask"], prm, geom=geom)
        api.order_points(p, out=order)
        api.rcs_sweep(sargs, p, n, r, geom, prm, ws=ws, E=E, sigma=sig, stats=st)

    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    # warm-up
    for _ in range(args.warmup):
        step(pos, nrm, rad)
    api.stream_check()

    # one counted step for the ray-bounce count (device counters)
    stats.zero_()
    step(pos, nrm, rad, stats)
    api.stream_check()
    st = stats.cpu().numpy()
    bounces_per_step = int(st[0] + st[1])

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K steps, L2 flushed between steps (outside the events);
    # the library also records events around every PO field launch on the
    # launching stream (the step's dominant kernel on this workload) for the
    # roofline; the march kernel's launches are timed the same way in the
    # end-to-end steps below.
    max_pairs = 512
    mev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * max_pairs)]
    for e in mev:          # torch creates the CUDA event on its first record
        e.record(stream)
    torch.cuda.synchronize()
    mev_ptrs = (ctypes.c_void_p * (2 * max_pairs))(*[e.cuda_event for e in mev])
    clk = ClockSampler(local_rank)
    clk.start()
    l0 = lib.pe_kernel_launches()
    barrier()
    lib.pe_set_kernel_events(b"po_kernel", mev_ptrs, max_pairs)
    total_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        # the same call as a user's (no diagnostic counters: the units of a
        # step were counted once above, on the device)
        step(pos, nrm, rad)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    barrier()
    n_po = lib.pe_set_kernel_events(None, None, 0)
    launches = lib.pe_kernel_launches() - l0
    clocks = clk.stop()
    api.stream_check()
    po_ms = [mev[2 * k].elapsed_time(mev[2 * k + 1]) for k in range(n_po)]
    po_terms = int(st[7])                                 # Eq. 14 terms per step
    po_launches_per_step = max(1, n_po // args.steps)
    march_queries = int(st[0]) - A * sw.W * sw.H          # bounce >= 2 queries per step

    # end to end through the C ABI with host buffers: pinned H2D of the
    # points each step, D2H of the field and sigma
    hp = torch.from_numpy(np.ascontiguousarray(sc.pos)).pin_memory()
    hn = torch.from_numpy(np.ascontiguousarray(sc.nrm)).pin_memory()
    hr = torch.from_numpy(np.ascontiguousarray(sc.rad)).pin_memory()
    hE = torch.empty(E.shape, dtype=E.dtype).pin_memory()
    hS = torch.empty(sig.shape, dtype=sig.dtype).pin_memory()
    dp, dn, dr = torch.empty_like(pos), torch.empty_like(nrm), torch.empty_like(rad)
    barrier()
    lib.pe_set_kernel_events(b"march_kernel", mev_ptrs, max_pairs)
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dp.copy_(hp, non_blocking=True)
        dn.copy_(hn, non_blocking=True)
        dr.copy_(hr, non_blocking=True)
        step(dp, dn, dr)
        hE.copy_(E, non_blocking=True)
        hS.copy_(sig, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    barrier()
    n_march = lib.pe_set_kernel_events(None, None, 0)
    march_ms = [mev[2 * k].elapsed_time(mev[2 * k + 1]) for k in range(n_march)]
    march_launches_per_step = max(1, n_march // args.steps)
    h2d = int(hp.numel() * 4 + hn.numel() * 4 + hr.numel() * 4)
    d2h = int(hE.numel() * 8 + hS.numel() * 8)

    # phase split (outside the timed steps): GFB views + fusion vs the sweep
    def _time(fn, reps=2):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def _geometry():
        g = api.build_gfb(gv, pos, nrm, rad, 0, 0.0, outputs=("nd", "mask"))
        api.aggregate_views(gv, g["nd"], g["mask"], prm, geom=geom)

    geom_ms = _time(_geometry)
    # surfel radius (8 nearest) and PCA normal (16 nearest) of every point
    pattr_ms = _time(lambda: api.point_attributes(pos, 8, 16, nrm))
    sweep_ms = _time(lambda: api.rcs_sweep(sargs, pos, nrm, rad, geom, prm, ws=ws, E=E, sigma=sig))
    api.stream_check()
    phases = {"point_attributes_ms": pattr_ms, "gfb_views_and_fusion_ms": geom_ms,
              "sweep_ms": sweep_ms, "sweep_ms_per_angle": sweep_ms / A}

    # rooflines of the two largest kernels, each timed per launch with CUDA
    # events on the launching stream inside timed steps; `roofline` is the
    # one with more device time per step
    roof_po = roofline_po(po_ms, po_terms / po_launches_per_step,
                          "po_rot_kernel" if F >= 2 else "po_kernel",
                          clocks.get("sm_mhz") if isinstance(clocks, dict) else None,
                          A * sw.W * sw.H / po_launches_per_step)
    roof_march = roofline_march(march_ms, march_queries / march_launches_per_step,
                                int(st[1]) / march_launches_per_step)
    for r, n in ((roof_po, n_po), (roof_march, n_march)):
        if r:
            r["ms_per_step"] = r["ms_per_launch"] * n / args.steps
    cands = [r for r in (roof_po, roof_march) if r]
    roof = max(cands, key=lambda r: r["ms_per_step"]) if cands else None
    others = {("roofline_march" if r is roof_march else "roofline_po"): r
              for r in cands if r is not roof}
    # the incidence splats of one sweep: 64-bit key updates per second
    # against the measured fire-and-forget atomicMin rate of this device
    roof_splat = roofline_splat(lib, api, sargs, pos, nrm, rad, geom, prm, ws, E, sig, dev,
                                stream)

    # the job: units of all ranks over the slowest rank's time
    job_units, t_ms, value = shard.job_throughput(bounces_per_step * args.steps, total_ms, dev)
    _, e2e_ms, e2e_value = shard.job_throughput(bounces_per_step * args.steps, e2e_ms, dev)
    samples = A * F * 2 * args.steps * world
    out = {
        "metric": "ray-bounces/s",
        "value": value,
        "unit": "ray-bounces/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": dict(desc, l2="flushed between steps (512 MB write outside the timed events)",
                       ray_bounces_per_step=bounces_per_step,
                       shadow_queries_per_step=int(st[1]), splat_tests_per_step=int(st[2]),
                       node_tests_per_step=int(st[3]),
                       parallelism=(f"angles sharded over {world} GPUs (rank r: phi + r/{world} step)"
                                    if world > 1 else "1 GPU")),
        "rcs_samples_per_s": samples / (t_ms / 1e3),
        "e2e": {"value": e2e_value, "unit": "ray-bounces/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "rcs_samples_per_s": samples / (e2e_ms / 1e3)},
        "phases": phases,
        "roofline": roof,
        **others,
        "roofline_splat": roof_splat,
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    # the sweep's field and sigma (every step computes the same ones), for
    # the per-angle comparison with the CPU oracle after the timed work
    Eh = E.cpu().numpy()
    out["_fields"] = (Eh[..., 0] + 1j * Eh[..., 1], sig.cpu().numpy())
    return out


# Algorithmic bytes of the sweep's march: a bounce-2 query reads its pixel's
# GFB key (8 bytes) and the key point's normal (12 bytes; its bounce-1 record
# is implicit in them) and writes the pixel's bounce count and Psi (5 bytes);
# a hit writes a record (hit point, normal, direction, tube vectors: 15
# floats; path length: 8 bytes; 76 bytes with the count and the id).  Hits at
# bounces >= 2 per step = the shadow queries (each ray with two or more hits
# takes one).  With more than two bounces the later queries also read a
# stored record (76 bytes), which this count leaves out: a lower bound there.
MARCH_BYTES_PER_QUERY = 25
MARCH_BYTES_PER_HIT = 76


# DRAM bytes (read + write) per bounce query of march_kernel from one ncu
# capture of the sweep's march on a smaller case (one 8-angle batch of the
# sphere workload through pe_rcs_sweep; profiles/march_kernel_sphere_batch.md:
# 91.1 MB over 6,332,964 queries), valid only for the sources it was taken on
# (their SHA-256 prefixes); scaled to a full launch by the number of queries.
_SWEEP_SOURCES = {"include/pointemray.h": "867cc444e32855cc",
                  "paper_2408_15583_gb300/csrc/pe_internal.cuh": "2dc3ec4e588ae1ce",
                  "paper_2408_15583_gb300/csrc/sweep.cu": "9f2bcf7b228eaa30"}
MARCH_NCU_TRAFFIC = {"bytes_per_query": 14.39,
                     "sources": dict(_SWEEP_SOURCES, **{
                         "paper_2408_15583_gb300/csrc/trace.cu": "04fbdf628ec696d9",
                         "paper_2408_15583_gb300/csrc/aggregate.cu": "a2f21815ee049028"})}

# DRAM bytes (read + write) per ray slot of po_rot_kernel from one ncu capture
# of the sweep's field sum on one 8-angle sphere batch
# (profiles/po_kernel_sphere_batch.md: 115.9 MB over 8 x 1024^2 slots), valid
# for the sources it was taken on; scaled to a full launch by its slots
# (angles x W x H).
PO_NCU_TRAFFIC = {"bytes_per_slot": 13.81,
                  "sources": dict(_SWEEP_SOURCES, **{
                      "paper_2408_15583_gb300/csrc/po.cu": "4eb889207db41b89"})}


def _traffic_valid(rec):
    import hashlib
    for path, sha in rec["sources"].items():
        try:
            h = hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest()
        except OSError:
            return False
        if not h.startswith(sha):
            return False
    return True


def roofline_march(ms_list, queries_per_launch, hits_per_launch=0.0):
    if not ms_list:
        return None
    ms = float(np.mean(ms_list))
    nbytes = queries_per_launch * MARCH_BYTES_PER_QUERY + hits_per_launch * MARCH_BYTES_PER_HIT
    achieved = nbytes / (ms / 1e3) / 1e9
    peak, src = hbm_peak()
    traffic = None
    if _traffic_valid(MARCH_NCU_TRAFFIC):
        traffic = MARCH_NCU_TRAFFIC["bytes_per_query"] * queries_per_launch
    return {"kernel": "march_kernel", "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_note": "bytes per launch, scaled by queries from a smaller ncu capture",
            "peak_source": src, "bytes_per_query": MARCH_BYTES_PER_QUERY,
            "bytes_per_hit": MARCH_BYTES_PER_HIT, "queries_per_launch": queries_per_launch,
            "hits_per_launch": hits_per_launch, "ms_per_launch": ms,
            "launches_timed": len(ms_list)}


def roofline_splat(lib, api, sargs, pos, nrm, rad, geom, prm, ws, E, sig, dev, stream):
    """The sweep's incidence splats (both passes, every angle batch), timed
    per launch with CUDA events on the launching stream, against the
    device's measured rate of fire-and-forget 64-bit atomicMin (the
    splat's key update; pe_probe_units).  Counters: exact per-pixel tests
    and key updates (pe_rcs_sweep stats words 5 and 6).  The sweep runs
    here with one frequency: the same angles, screens and batches, so the
    same splat launches, but one set of batch buffers, so no field sum of a
    previous batch shares the SMs with a splat launch being timed."""
    import torch
    from paper_2408_15583_gb300 import peaks
    n_ev = 256
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_ev)]
    for e in ev:
        e.record(stream)
    torch.cuda.synchronize()
    ptrs = (ctypes.c_void_p * len(ev))(*[e.cuda_event for e in ev])
    st = torch.zeros(8, dtype=torch.int64, device=dev)
    c = sargs.c
    one = api.SweepArgs(sargs.theta, sargs.phi, c.W, c.H, list(c.centre), c.extent,
                        sargs.freqs[:1], c.max_bounces, c.angle_batch)
    one.set_point_order(sargs.order)
    ws1 = api.workspace(one.workspace_bytes(), dev)
    E1 = torch.empty((E.shape[0], 1) + tuple(E.shape[2:]), dtype=E.dtype, device=dev)
    api.rcs_sweep(one, pos, nrm, rad, geom, prm, ws=ws1, E=E1)      # warm
    lib.pe_set_kernel_events(b"splat_kernel", ptrs, n_ev)
    api.rcs_sweep(one, pos, nrm, rad, geom, prm, ws=ws1, E=E1, stats=st)
    n = lib.pe_set_kernel_events(None, None, 0)
    torch.cuda.synchronize()
    api.stream_check()
    ms = sum(ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n))
    s = st.cpu().numpy()
    tests, updates = int(s[5]), int(s[6])
    probe = peaks.measure(str(dev), reps=3, only=("atomic_min_u64",))["atomic_min_u64"]["value"]
    achieved = updates / (ms / 1e3) / 1e9
    return {"kernel": "splat_kernel (both passes)", "bound": "l2_atomics", "achieved": achieved,
            "peak": probe, "unit": "G atomics/s", "frac": achieved / probe, "traffic": None,
            "peak_source": "pe_probe_units fire-and-forget 64-bit atomicMin, measured in this run",
            "launches": n, "ms_per_sweep": ms, "key_updates_per_sweep": updates,
            "exact_tests_per_sweep": tests}


def hbm_peak():
    try:
        m = json.load(open(MEASURED))
        return float(m["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy bandwidth)"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback 6.8 TB/s"


def roofline_po(ms_list, terms_per_launch, name="po_rot_kernel", sm_mhz=None,
                slots_per_launch=None):
    """The PO field kernel of the sweep (po_rot_kernel on uniform frequency
    grids, po_kernel otherwise), timed per launch inside the timed steps;
    terms = the Eq. 14 terms of a step (device counter, stats word 7) over
    its PO launches.  ALU roofline at PO_FLOPS_PER_TERM flops per term."""
    if not ms_list or terms_per_launch <= 0:
        return None
    ms = float(np.mean(ms_list))
    achieved = terms_per_launch * PO_FLOPS_PER_TERM / (ms / 1e3) / 1e12
    peak, src = alu_peak(sm_mhz)
    traffic = None
    if slots_per_launch and name == "po_rot_kernel" and _traffic_valid(PO_NCU_TRAFFIC):
        traffic = PO_NCU_TRAFFIC["bytes_per_slot"] * slots_per_launch
    return {"kernel": name, "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
            "traffic_note": "bytes per launch, scaled by ray slots from a smaller ncu capture",
            "peak_source": src, "flops_per_term": PO_FLOPS_PER_TERM,
            "terms_per_launch": terms_per_launch, "ms_per_launch": ms,
            "launches_timed": len(ms_list)}


PO_FLOPS_PER_TERM = 64


def alu_peak(sm_mhz=None):
    """FP32 peak = 152 SMs x 128 FP32 lanes x 2 (FMA) x SM clock, at the SM
    clock sampled during this run's timed region (the kernel runs at that
    clock; the slower median clock in MEASURED_PEAKS.json is the power-capped
    GEMM's), else at the maximum clock, 2070 MHz."""
    if sm_mhz and sm_mhz > 0:
        mhz, how = float(sm_mhz), "median SM clock sampled during the timed region"
    else:
        mhz, how = 2070.0, "maximum SM clock"
    return 152 * 128 * 2 * mhz * 1e6 / 1e12, f"152 SM x 128 FP32 lanes x 2 x {mhz:.0f} MHz ({how})"


# ----------------------------------------------------------------------------
# CPU oracle arm (cpu_baseline leg and --impl reference)
# ----------------------------------------------------------------------------

def _angle_queries(M, mb, per):
    """Intersection queries of one angle, counted as the device counters
    count them: every screen ray's primary lookup, one query per live ray at
    each bounce b = 2..mb (its last one a miss unless it reached mb), and a
    shadow ray for every ray that ended after two or more bounces."""
    M = np.asarray(M)
    q = per + int(sum(int((M >= b - 1).sum()) for b in range(2, mb + 1)))
    return q + int((M >= 2).sum())


def oracle_workload(wl, angles, threads=None, E_gpu=None, sig_gpu=None):
    """The CPU oracle (FP32-geometry mode: the GPU path's bit-exact target,
    FP64 field sums) on the workload itself: its own 8 GFBs at full size and
    their fusion, then for each listed angle the whole screen (Alg. 1 GFB,
    bounces, Psi, Eq. 14 over every frequency, sigma).  Returns the timings,
    the query counts and, given the GPU's field and sigma for the whole
    sweep, the per-angle parity (c24: field error, |delta sigma| in dB where
    sigma_ref >= peak - 40 dB)."""
    import oracle
    sc, sw, vd = wl.scene, wl.sweep, wl.views
    used = oracle.set_threads(threads or (os.cpu_count() or 1))
    t0 = time.perf_counter()
    S, gv, _, _ = oracle.build_geometry(sc, vd, "fp32")
    t_geom = time.perf_counter() - t0
    eps = oracle.default_eps(gv)
    per = sw.W * sw.H
    t_ang, q_ang, rows = [], [], []
    for a in angles:
        t1 = time.perf_counter()
        ref = oracle.rcs_sweep(sc, sw, S, eps, eps, mode="fp32", angles=[a])
        t_ang.append(time.perf_counter() - t1)
        q_ang.append(_angle_queries(ref.traces[0].M, sw.max_bounces, per))
        if E_gpu is not None:
            Eg = E_gpu[a:a + 1]
            d = np.sqrt((np.abs(Eg - ref.E) ** 2).sum(axis=-1))
            r = np.sqrt((np.abs(ref.E) ** 2).sum(axis=-1))
            fe = float((d / np.maximum(r, 1e-3 * r.max())).max()) if r.max() > 0 else \
                float(d.max())
            de = 0.0
            for p in (0, 1):
                sd, so = oracle.db(sig_gpu[a:a + 1, :, p, p]), oracle.db(ref.sigma[..., p, p])
                keep = so >= so.max() - 40.0
                de = max(de, float(np.abs(sd - so)[keep].max()))
            rows.append({"angle": int(a), "phi_deg": float(sw.phi_deg[a]),
                         "theta_deg": float(sw.theta_deg[a]), "field_err": fe,
                         "dsigma_db": de})
        del ref
    oracle.set_threads(os.cpu_count() or 1)
    # the step's composition: one geometry for the whole sweep of n angles
    n = sw.n_angles
    t_step = t_geom + n * float(np.mean(t_ang))
    q_step = n * float(np.mean(q_ang))
    return {"threads": used, "t_geometry_s": t_geom, "t_angles_s": t_ang, "queries": q_ang,
            "t_step_s": t_step, "queries_step": q_step, "rate": q_step / t_step,
            "parity": rows}


# ----------------------------------------------------------------------------
# serving (continuous batching vs one request at a time)
# ----------------------------------------------------------------------------

def run_serving(n_requests=48, slots=4, budget_gb=150.0, seed=5):
    """The serving mix (serve.make_c5_requests): Poisson arrivals; per
    request its own target of 10k-4M points (radii computed on the device),
    a 128^2-4096^2 screen, 1-720 azimuths, 1-128 frequencies, 1-5 bounces,
    fused geometry from 8 views at 256^2; HBM budget 150 GB.  The one-at-a-
    time service rate is measured first on the same requests; arrivals then
    come at 70 % of it, served one at a time, in plain batches of `slots`
    (a batch starts when the previous one is done) and continuously (a
    request starts as soon as a slot and memory are free)."""
    import torch
    from paper_2408_15583_gb300 import serve
    budget = int(budget_gb * (1 << 30))
    reqs = serve.make_c5_requests(n_requests, rate_hz=1e9, seed=seed)
    cal = serve.Scheduler(serve.GpuExecutor(n_slots=1), budget, n_slots=1)
    t0 = time.perf_counter()
    cal.run(reqs)
    torch.cuda.synchronize()
    busy = time.perf_counter() - t0
    rate = 0.7 * n_requests / busy
    for r in reqs:
        r.arrival = 0.0
    import dataclasses
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    t = 0.0
    timed = []
    for r in reqs:
        t += rng.exponential(1.0 / rate)
        timed.append(dataclasses.replace(r, arrival=t))
    shapes = {(r.n_points, r.W, len(r.theta_deg), len(r.freqs_hz), r.max_bounces) for r in reqs}
    out = {"requests": n_requests, "rate_hz": rate, "slots": slots, "hbm_budget_gb": budget_gb,
           "one_at_a_time_service_s": busy,
           "distinct_shapes": len(shapes),
           "workload": "Poisson arrivals at 70% of the one-at-a-time service rate; per request "
                       "its own target (dihedral / sphere / trihedral / composite / OctAR shape) "
                       "of N ~ logU(10k, 4M) points, radii computed on the device, screen "
                       "128^2-4096^2 (log-uniform powers of two), A ~ logU(1, 720) azimuths, "
                       "F ~ logU(1, 128) frequencies, mb ~ U{1..5}, fused geometry 8 x 256^2"}
    for name, n_slots, policy in (("one_at_a_time", 1, "continuous"),
                                  ("plain_batched", slots, "static"),
                                  ("continuous", slots, "continuous")):
        sch = serve.Scheduler(serve.GpuExecutor(n_slots=n_slots), budget, n_slots=n_slots,
                              policy=policy)
        res = sch.run(timed)
        torch.cuda.synchronize()
        st = serve.latency_stats(res)
        st["max_concurrent"] = sch.max_running
        st["peak_device_gb"] = sch.peak_in_use / (1 << 30)
        ok = [r for r in res if r.ok]
        st["host_exceeds_device"] = sum(1 for r in ok if r.host_ms > r.device_ms)
        out[name] = st
    return out


# ----------------------------------------------------------------------------
# learned GFB completion (training throughput, inference vs plain splatting)
# ----------------------------------------------------------------------------

def run_learned(W=256, batch=64, steps=8, warmup=2):
    """Training steps of the U-Net at the C4 shape (256^2 coarse depth,
    batch 64, widths 32-256), timed with CUDA events; per-view time of the
    learned path (tube splat of the sparse cloud + inference) vs plain surfel
    splatting of the dense cloud."""
    import torch
    from paper_2408_15583_gb300 import learned_train as lt
    from paper_2408_15583_gb300.learned import UNet
    widths, blocks = (32, 64, 128, 256), (2, 2, 2, 2)
    data = lt.dataset(4, 16, W, seed=21, keep_scenes=True)
    net = UNet(scenes.unet_init(0, widths, blocks), widths, blocks, "cuda:0")
    P = W * W
    x = torch.cat([d["x"] for d in data]).view(-1, P)[:batch].reshape(-1).contiguous()
    dg = torch.cat([d["d_gt"] for d in data]).view(-1, P)[:batch].reshape(-1).contiguous()
    ng = torch.cat([d["n_gt"] for d in data]).view(-1, P, 3)[:batch].reshape(-1, 3).contiguous()
    mg = torch.cat([d["m_gt"] for d in data]).view(-1, P)[:batch].reshape(-1).contiguous()
    for _ in range(warmup):
        net.train_step(x, dg, ng, mg, batch, W, W, 1e-4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        loss = net.train_step(x, dg, ng, mg, batch, W, W, 1e-4)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # the same steps replayed as a captured CUDA graph (forward, losses,
    # backward) plus the AdamW update
    from paper_2408_15583_gb300.learned import GraphedUNet
    gnet = GraphedUNet(net, batch, W, W)
    for _ in range(warmup):
        gnet.train_step(x, dg, ng, mg, 1e-4)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        loss = gnet.train_step(x, dg, ng, mg, 1e-4)
    e1.record()
    e1.synchronize()
    ms_graphed = e0.elapsed_time(e1) / steps
    ms_eager = ms
    ms = min(ms, ms_graphed)
    flops = 3.0 * lt.forward_flops(widths, blocks, W, W) * batch
    hbm_bytes = 3.0 * lt.forward_bytes(widths, blocks, W, W) * batch
    peak = 1708.8
    try:
        peak = float(json.load(open(MEASURED))["bf16_tflops_sustained"])
    except (OSError, ValueError, KeyError):
        pass
    t = lt.time_paths(net, data[0]["sparse"], data[0]["dense"], data[0]["vs"])
    fk = lt.finite_k_study(data)
    return {"workload": f"U-Net widths 32-256, {W}^2 coarse depth, batch {batch}, BF16 "
                        "activations, FP32 accumulation; pairs from the surfel tracer",
            "train_ms_per_step": ms, "train_ms_per_step_eager": ms_eager,
            "train_ms_per_step_graphed": ms_graphed, "train_images_per_s": batch / (ms / 1e3),
            "train_tflops": flops / (ms / 1e3) / 1e12,
            "tensor_roofline": {"bound": "tensor", "achieved": flops / (ms / 1e3) / 1e12,
                                "peak": peak, "unit": "TFLOP/s",
                                "frac": flops / (ms / 1e3) / 1e12 / peak,
                                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained"},
            # widths 32-256 make most layers stream activations (1x1 GEMMs
            # with K <= 256, depthwise, LayerNorm, GELU): the same step
            # against HBM, with layer-wise algorithmic bytes (each layer
            # reads its inputs and writes its outputs once; a training step
            # taken as 3 forward passes, like its FLOPs)
            "hbm_roofline": {"bound": "hbm", "achieved": hbm_bytes / (ms / 1e3) / 1e9,
                             "peak": hbm_peak()[0], "unit": "GB/s",
                             "frac": hbm_bytes / (ms / 1e3) / 1e9 / hbm_peak()[0],
                             "bytes_per_step": hbm_bytes,
                             "peak_source": hbm_peak()[1]},
            "last_loss": float(loss.cpu()[0]),
            "ms_per_view_learned_path": t["learned"] * 1e3,
            "ms_per_view_learned_path_graphed": t["learned_graphed"] * 1e3,
            "ms_per_view_plain_splatting": t["plain_splatting"] * 1e3,
            "alg1_finite_k_vs_unbounded": fk}


# angles of the sweep the CPU oracle runs beside the bench (spread over the
# library's angle batches); the first one alone for the one-core leg
CPU_ANGLES = {"sphere": [0, 45, 90, 135, 180, 225, 270, 315], "dihedral": [0, 22, 45, 90],
              "composite": [0, 18], "octar": [0, 45, 90, 180]}


def cpu_baseline(wl, name, E_gpu=None, sig_gpu=None):
    angles = CPU_ANGLES[name]
    allc = oracle_workload(wl, angles, None, E_gpu, sig_gpu)
    one = oracle_workload(wl, angles[:1], 1)
    sw, vd = wl.sweep, wl.views
    sample = (f"CPU oracle (FP32 geometry, FP64 field sums, uniform-grid searches) on the "
              f"workload itself: its 8 GFBs at {vd.W}x{vd.H} over all {wl.scene.n} points and "
              f"their fusion, then {len(angles)} of the {sw.n_angles} angles, every one of the "
              f"{sw.W}x{sw.H} rays, {sw.max_bounces} bounces, {sw.n_freq} frequencies; rate "
              f"projected to the whole step (geometry + {sw.n_angles} x the mean angle time): "
              f"{allc['t_geometry_s']:.1f} s geometry + {np.mean(allc['t_angles_s']):.2f} s per "
              f"angle on {allc['threads']} threads")
    out = {"value": allc["rate"], "unit": "ray-bounces/s", "cores": allc["threads"],
           "kind": "oracle", "sample": sample,
           "one_core": {"value": one["rate"], "cores": 1,
                        "sample": f"geometry {one['t_geometry_s']:.1f} s + angle "
                                  f"{angles[0]} {one['t_angles_s'][0]:.1f} s on one thread"}}
    parity = None
    if allc["parity"]:
        rows = allc["parity"]
        parity = {"vs": "CPU oracle, every ray of each listed angle, all frequencies, both "
                        "polarisations (c24 field error; |d sigma| where sigma_ref >= peak - 40 dB)",
                  "max_field_err": max(r["field_err"] for r in rows),
                  "max_dsigma_db": max(r["dsigma_db"] for r in rows),
                  "per_angle": rows}
    return out, parity


def run_reference(args):
    """The CPU oracle timed as the reference arm: each step is the
    workload's geometry (8 GFBs at full size + fusion) and one angle of its
    sweep (every ray, all frequencies), on every host core; the rate is
    projected to the whole step like the GPU arm's (geometry once + every
    angle)."""
    wl, desc = make_workload(args.workload)
    sw = wl.sweep
    for k in range(args.warmup):
        oracle_workload(wl, [k % sw.n_angles])
    t_geom, t_ang, q_ang, threads = [], [], [], 1
    for k in range(args.steps):
        a = (k * 37) % sw.n_angles
        r = oracle_workload(wl, [a])
        t_geom.append(r["t_geometry_s"])
        t_ang += r["t_angles_s"]
        q_ang += r["queries"]
        threads = r["threads"]
    t_step = float(np.mean(t_geom)) + sw.n_angles * float(np.mean(t_ang))
    q_step = sw.n_angles * float(np.mean(q_ang))
    v = q_step / t_step
    sample = (f"each step: the CPU oracle's 8 GFBs at {wl.views.W}x{wl.views.H} + fusion and one "
              f"angle of the sweep (every one of the {sw.W}x{sw.H} rays, {sw.n_freq} "
              f"frequencies), on {threads} threads; rate projected to the whole step "
              f"(geometry + {sw.n_angles} angles)")
    return {
        "impl": "reference", "metric": "ray-bounces/s", "value": v, "unit": "ray-bounces/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": desc,
        "cpu_baseline": {"value": v, "unit": "ray-bounces/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "ray-bounces/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="sphere", choices=["sphere", "dihedral", "composite", "octar"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_gpu(args, rank, world, local_rank)
    _gpu_fields = out.pop("_fields")
    if rank == 0 and world == 1 and not args.no_serving:
        out["serving"] = run_serving()
    if rank == 0 and world == 1 and not args.no_learned:
        out["learned"] = run_learned()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        wl, _ = make_workload(args.workload)
        out["cpu_baseline"], out["parity"] = cpu_baseline(wl, args.workload, *_gpu_fields)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
