"""Small, representative cases of the hot kernels for profiling (ncu).

    python -m paper_2408_15583_gb300.profile_case march [reps] [workload]  # one traced batch
    python -m paper_2408_15583_gb300.profile_case po [reps] [workload]     # PO over that batch
    python -m paper_2408_15583_gb300.profile_case splat [reps] [workload]  # incidence splats
    python -m paper_2408_15583_gb300.profile_case sweep [reps] [workload]  # pe_rcs_sweep of the batch
    python -m paper_2408_15583_gb300.profile_case unet [reps] [batch] [mma]  # U-Net training steps

By default each case is the sphere workload's geometry (200k points, 8 fused
512^2 views) with one batch of 8 incidence angles at 1024^2 rays and 64
frequencies: a few GB on the device, inputs larger than L2, a handful of
launches -- small enough for a full ncu capture of one launch.  `workload`
= dihedral, composite or octar takes that workload's scene, screen and bounce
count instead (for timing; the composite batch holds ~3 GB of ray records).
"""
from __future__ import annotations

import ctypes
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv):
    import torch

    import scenes
    from paper_2408_15583_gb300 import api, build, pipeline

    build()
    case = argv[0] if argv else "march"
    reps = int(argv[1]) if len(argv) > 1 else 3
    if case == "unet":
        if len(argv) > 3 and argv[3] == "mma":     # the mma.sync contraction kernel only
            from paper_2408_15583_gb300 import _lib
            _lib.load().pe_nn_gemm_path(1)
        return unet_case(reps, int(argv[2]) if len(argv) > 2 else 64)
    name = argv[2] if len(argv) > 2 else "sphere"
    wl = {"sphere": scenes.workload_sphere, "dihedral": scenes.workload_dihedral,
          "composite": scenes.workload_composite, "octar": scenes.workload_octar}[name]()
    sc, sw, vd = wl.scene, wl.sweep, wl.views
    dev = "cuda:0"
    pos, nrm, rad = pipeline.scene_to_device(sc, dev)
    gv = pipeline.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, vd.W, vd.H)
    prm = pipeline.default_params(sc.pos, gv)
    geom, _ = pipeline.build_geometry(pos, nrm, rad, gv, prm)
    nb = 8
    na = len(sw.phi_deg)
    mb = max(2, sw.max_bounces)
    views = [api.view_from_angles(sw.theta_deg[a * na // nb], sw.phi_deg[a * na // nb], sw.centre,
                                  sw.extent, sw.W, sw.H) for a in range(nb)]
    keys = api.build_gfb(views, pos, nrm, rad, 0, outputs=("keys",))["keys"]
    stats = torch.zeros(8, dtype=torch.int64, device=dev)
    h = api.trace_bounces(views, keys, nrm, geom, mb, prm, ids=False, stats=stats)
    ks = [[-x for x in v.d] for v in views]
    if case == "sweep":
        import numpy as np
        sub = [a * na // nb for a in range(nb)]
        sargs = api.SweepArgs(theta_deg=np.asarray(sw.theta_deg, np.float64)[sub],
                              phi_deg=np.asarray(sw.phi_deg, np.float64)[sub], W=sw.W, H=sw.H,
                              centre=sw.centre, extent=sw.extent,
                              freqs_hz=np.asarray(sw.freqs_hz, np.float64), max_bounces=mb,
                              angle_batch=nb)
        sargs.set_point_order(api.order_points(pos))   # as the bench's step does
        sws = api.workspace(sargs.workspace_bytes(), dev)
        sE = torch.empty((nb, len(sw.freqs_hz), 2, 3, 2), dtype=torch.float64, device=dev)
        sS = torch.empty((nb, len(sw.freqs_hz), 2, 2), dtype=torch.float64, device=dev)
        api.rcs_sweep(sargs, pos, nrm, rad, geom, prm, ws=sws, E=sE, sigma=sS)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        if case == "march":
            api.trace_bounces(views, keys, nrm, geom, mb, prm, hits=h, ids=False)
        elif case == "po":
            api.po_field(h, nb, sw.W * sw.H, ks, sw.freqs_hz)
        elif case == "splat":
            api.build_gfb(views, pos, nrm, rad, 0, outputs=("keys",))
        elif case == "sweep":
            # the same 8 angles through the whole sweep (one batch: its march
            # and field sum keep the bounce-1 records implicit in the keys)
            api.rcs_sweep(sargs, pos, nrm, rad, geom, prm, ws=sws, E=sE, sigma=sS)
        else:
            raise SystemExit(f"unknown case {case}")
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / reps
    api.stream_check()
    st = stats.cpu().numpy()
    print(f"{case}: {dt * 1e3:.2f} ms per call; batch queries {st[0]} shadow {st[1]} "
          f"exact splat tests {st[2]} node tests {st[3]} views walked {st[4]}")
    if case == "march":
        # per-launch times of the trace's kernels (CUDA events on the stream)
        from paper_2408_15583_gb300 import _lib
        lib = _lib.load()
        for kname in ("primary_kernel", "march_kernel", "shadow_kernel"):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * 16)]
            for e in ev:       # torch creates the CUDA event on its first record
                e.record()
            torch.cuda.synchronize()
            ptrs = (ctypes.c_void_p * len(ev))(*[e.cuda_event for e in ev])
            lib.pe_set_kernel_events(kname.encode(), ptrs, 16)
            api.trace_bounces(views, keys, nrm, geom, mb, prm, hits=h, ids=False)
            n = lib.pe_set_kernel_events(None, None, 0)
            torch.cuda.synchronize()
            ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(n)]
            print(f"  {kname}: " + " ".join(f"{m:.3f}" for m in ms) + " ms")


def unet_case(reps, batch, W=256):
    """Training steps of the completion U-Net (widths 32-256, two blocks per
    level) at W x W on seeded random maps (one warm-up step first)."""
    import numpy as np
    import torch

    import scenes
    from paper_2408_15583_gb300.learned import UNet

    widths, blocks = (32, 64, 128, 256), (2, 2, 2, 2)
    net = UNet(scenes.unet_init(0, widths, blocks), widths, blocks, "cuda:0")
    g = torch.Generator().manual_seed(3)
    P = batch * W * W
    x = torch.rand(P, generator=g).to("cuda:0", torch.bfloat16)
    m = (torch.rand(P, generator=g) > 0.5).float().cuda()
    d = torch.rand(P, generator=g).cuda() * m
    n = torch.nn.functional.normalize(torch.randn(P, 3, generator=g), dim=1).cuda()
    net.train_step(x, d, n, m, batch, W, W, 1e-4)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        loss = net.train_step(x, d, n, m, batch, W, W, 1e-4)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / reps
    print(f"unet: {dt * 1e3:.2f} ms per training step (batch {batch}, {W}^2); "
          f"loss {np.round(loss.cpu().numpy(), 5).tolist()}")


if __name__ == "__main__":
    main(sys.argv[1:])
