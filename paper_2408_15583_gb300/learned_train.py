"""Data, training and evaluation of the learned GFB completion (a8).

Pairs: for a random target (``scenes.random_primitives``) sampled sparsely
(5-50 points per lambda^2) and densely (>= 200 per lambda^2), each view gives
a coarse tube-mode depth map (Alg. 1, tube radius 1-3 pixels) of the sparse
cloud as input, and the dense cloud's surfel GFB (depth, normal in the uvw
frame, hit mask) as target -- both produced by the surfel tracer kernels
(``pe_build_gfb``), whose output is bit-identical to the CPU oracle's FP32
mode.  The ray pitch is lambda/10 (Sec. IV-A).

Evaluation (what the network gains): for held-out targets, the monostatic PO
RCS (single bounce, Eq. 14) of (a) the dense surfel GFB -- the reference --,
(b) the coarse tube-mode GFB with normals from its depth by Eq. 16 -- the
method without the network --, and (c) the network's GFB; RMSE in dB over the
views of each target with the floor of c23 (max(sigma_ref) - 60 dB).
"""
from __future__ import annotations

import ctypes as C
import json
import math
import time
from dataclasses import dataclass
from typing import List

import numpy as np
import torch

from . import _lib, api, pipeline
from ._lib import check
from .learned import GraphedUNet, UNet, lr_schedule

C0 = 299_792_458.0


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@dataclass
class ViewSet:
    views: list
    t_near: np.ndarray
    t_scale: np.ndarray
    lam: float
    W: int


def view_set(scene, n_views: int, W: int, seed: int) -> ViewSet:
    rng = np.random.Generator(np.random.PCG64(seed))
    p = scene.pos.astype(np.float64)
    c = 0.5 * (p.min(0) + p.max(0))
    r = float(np.sqrt(((p - c) ** 2).sum(1).max()))
    ext = 1.02 * r
    th = rng.uniform(30.0, 150.0, n_views)
    ph = rng.uniform(0.0, 360.0, n_views)
    views = [api.view_from_angles(t, f, c, ext, W, W) for t, f in zip(th, ph)]
    L = views[0].pitch
    D = ext + L
    return ViewSet(views, np.full(n_views, D - r, np.float32), np.full(n_views, 2 * r, np.float32),
                   10.0 * L, W)


def make_pairs(sparse, dense, vs: ViewSet, delta_px: float, device="cuda:0"):
    """GPU tensors x (BF16 [n*P]), d_gt, m_gt ([n*P]), n_gt ([n*P, 3])."""
    lib = _lib.load()
    n = len(vs.views)
    P = vs.W * vs.W
    ps = torch.from_numpy(np.ascontiguousarray(sparse.pos, dtype=np.float32)).to(device)
    pd = torch.from_numpy(np.ascontiguousarray(dense.pos, dtype=np.float32)).to(device)
    nd_ = torch.from_numpy(np.ascontiguousarray(dense.nrm, dtype=np.float32)).to(device)
    if dense.rad is None:   # surfel radii on the device (8 nearest, pe_point_attributes)
        rd, _ = api.point_attributes(pd, 8, 16, None, radius=True, normal=False)
    else:
        rd = torch.from_numpy(np.ascontiguousarray(dense.rad, dtype=np.float32)).to(device)
    delta = float(delta_px * vs.views[0].pitch)
    keys = api.build_gfb(vs.views, ps, None, None, 1, delta, outputs=("keys",))["keys"]
    nd = api.build_gfb(vs.views, pd, nd_, rd, 0, outputs=("nd",))["nd"]
    x = torch.empty(n * P, dtype=torch.bfloat16, device=device)
    d_gt = torch.empty(n * P, dtype=torch.float32, device=device)
    m_gt = torch.empty(n * P, dtype=torch.float32, device=device)
    n_gt = torch.empty(n * P, 3, dtype=torch.float32, device=device)
    arr = api.views_to_array(vs.views)
    check(lib.pe_learned_pairs(arr, n, vs.t_near.ctypes.data_as(C.c_void_p),
                               vs.t_scale.ctypes.data_as(C.c_void_p), _p(keys), _p(nd), _p(x),
                               _p(d_gt), _p(n_gt), _p(m_gt),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream)),
          "pe_learned_pairs")
    return {"x": x, "d_gt": d_gt, "n_gt": n_gt, "m_gt": m_gt, "vs": vs}


def dataset(n_scenes: int, views_per_scene: int, W: int, seed: int, device="cuda:0",
            dense_density=200.0, keep_scenes=False):
    """Pairs of n_scenes random targets x views_per_scene views.  The tube
    mode needs no radii; the dense cloud's surfel radii are computed on the
    device unless the scenes are kept (for the paths that splat them
    again)."""
    import scenes
    out = []
    for k in range(n_scenes):
        sd = seed * 100_003 + k
        rng = np.random.Generator(np.random.PCG64(sd))
        sparse = scenes.random_primitives(sd, 1.0, bbox_lambdas=W / 10.0, radius=keep_scenes)
        dense = scenes.random_primitives(sd, 1.0, bbox_lambdas=W / 10.0, density=dense_density,
                                         radius=keep_scenes)
        vs = view_set(sparse, views_per_scene, W, sd + 1)
        item = make_pairs(sparse, dense, vs, float(rng.uniform(1.0, 3.0)), device)
        if keep_scenes:
            item["sparse"], item["dense"] = sparse, dense
        out.append(item)
    return out


def forward_flops(widths, blocks, H, W):
    """FP ops of one forward pass on an H x W image (multiply-add = 2)."""
    f = 0.0
    c = widths
    L = len(widths)
    px = [H * W / 4 ** l for l in range(L)]
    f += 2 * px[0] * 9 * 1 * c[0]                              # stem
    blk = lambda p, ch: 2 * p * (49 * ch + 8 * ch * ch)        # dw 7x7 + two 1x1
    for l in range(L):
        if l > 0:
            f += 2 * px[l] * c[l - 1] * c[l]
        f += blocks[l] * blk(px[l], c[l])
    for nout in (1, 3, 1):
        for l in range(L - 2, -1, -1):
            f += 2 * px[l + 1] * 9 * c[l + 1] * 4 * c[l]          # up 3x3
            f += 2 * px[l] * 2 * c[l] * c[l] + blk(px[l], c[l])  # fuse + block
        f += 2 * px[0] * c[0] * nout
    return f


def forward_bytes(widths, blocks, H, W, elem=2):
    """Layer-wise algorithmic bytes of one forward pass on an H x W image:
    every layer reads its inputs and writes its outputs once (activations of
    `elem` bytes; weights and im2col columns not counted).  A ConvNeXt block
    moves 16 C values per pixel: depthwise 7x7 (C in, C out), LayerNorm (C,
    C), 1x1 expansion (C, 4C), 1x1 projection with the residual (4C + C, C)."""
    c = widths
    L = len(widths)
    px = [H * W / 4 ** l for l in range(L)]
    v = px[0] * (1 + c[0])                                     # stem
    blk = lambda p, ch: 16 * p * ch
    for l in range(L):
        if l > 0:
            v += px[l - 1] * c[l - 1] + px[l] * c[l - 1]       # max-pool
            v += px[l] * (c[l - 1] + c[l])                     # 1x1 down
        v += blocks[l] * blk(px[l], c[l])
    for nout in (1, 3, 1):
        for l in range(L - 2, -1, -1):
            v += px[l + 1] * (c[l + 1] + 4 * c[l])             # up 3x3
            v += 2 * px[l] * c[l]                              # sub-pixel shuffle
            v += 2 * px[l] * c[l]                              # skip copy
            v += px[l] * 3 * c[l] + blk(px[l], c[l])           # fuse 1x1 + block
        v += px[0] * (c[0] + nout + 1)                         # head (+ residual)
    return v * elem


def _cat(items, key):
    return torch.cat([it[key] for it in items])


def train(model: UNet, data: List[dict], steps: int, batch: int, lr0=1e-3, seed=0,
          log_every=0, step0=0):
    """Mini-batches of `batch` views drawn from the whole set; the paper's
    halving schedule (Sec. IV-A) with `steps_per_epoch` = views / batch."""
    W = data[0]["vs"].W
    P = W * W
    x = _cat(data, "x").view(-1, P)
    d = _cat(data, "d_gt").view(-1, P)
    n = _cat(data, "n_gt").view(-1, P, 3)
    m = _cat(data, "m_gt").view(-1, P)
    nv = x.shape[0]
    spe = max(1, nv // batch)
    rng = np.random.Generator(np.random.PCG64(seed))
    hist = []
    for step in range(steps):
        idx = torch.from_numpy(rng.choice(nv, size=batch, replace=False)).to(x.device)
        lr = lr_schedule(step0 + step, spe, lr0=lr0, floor=1e-6)
        loss = model.train_step(x[idx].reshape(-1).contiguous(), d[idx].reshape(-1).contiguous(),
                                n[idx].reshape(-1, 3).contiguous(), m[idx].reshape(-1).contiguous(),
                                batch, W, W, lr)
        if log_every and (step % log_every == 0 or step == steps - 1):
            hist.append((step, loss.cpu().numpy().tolist()))
    return hist


def _sigma_from_hits(hits, vs: ViewSet):
    """Monostatic sigma (VV, m^2) of each view at f = c / lambda."""
    n = len(vs.views)
    ks = np.array([[-c for c in v.d] for v in vs.views], np.float32)
    E = api.po_field(hits, n, vs.W * vs.W, ks, np.array([C0 / vs.lam]))
    E = E.cpu().numpy()
    E = E[..., 0] + 1j * E[..., 1]                   # [n][1][pol][3]
    k = 2 * math.pi / vs.lam
    out = np.empty(n)
    for a, v in enumerate(vs.views):
        e = np.array(v.u[:], np.float64)
        out[a] = k * k / math.pi * abs(E[a, 0, 0] @ e) ** 2
    return out


def gfb_sigma(vs: ViewSet, depth, mask, threshold, normal_uvw):
    lib = _lib.load()
    n = len(vs.views)
    h = api.alloc_hits(n * vs.W * vs.W, 1, depth.device, ids=False)
    arr = api.views_to_array(vs.views)
    check(lib.pe_gfb_hits(arr, n, vs.t_near.ctypes.data_as(C.c_void_p),
                          vs.t_scale.ctypes.data_as(C.c_void_p), _p(depth), _p(mask),
                          float(threshold), _p(normal_uvw), C.byref(h.c),
                          C.c_void_p(torch.cuda.current_stream().cuda_stream)), "pe_gfb_hits")
    return _sigma_from_hits(h, vs)


def rmse_db(s, ref, floor_db=60.0):
    sd = 10 * np.log10(np.maximum(s, 1e-30))
    rd = 10 * np.log10(np.maximum(ref, 1e-30))
    lo = rd.max() - floor_db
    return float(np.sqrt(np.mean((np.maximum(sd, lo) - np.maximum(rd, lo)) ** 2)))


def evaluate(model: UNet, data: List[dict]):
    """Per held-out target: RMSE (dB) of the coarse GFB + Eq. 16 normals and
    of the network's GFB against the dense surfel GFB."""
    res = []
    for it in data:
        vs = it["vs"]
        n = len(vs.views)
        W = vs.W
        ref = gfb_sigma(vs, it["d_gt"], it["m_gt"], 0.5, it["n_gt"])
        xf = it["x"].float()
        coarse = gfb_sigma(vs, xf, xf, 0.0, None)
        outs, _ = model.forward(it["x"], n, W, W)
        learned = gfb_sigma(vs, outs["depth"], outs["mask"], 0.0, outs["normal"])
        res.append({"coarse": rmse_db(coarse, ref), "learned": rmse_db(learned, ref)})
    return res


def time_paths(model: UNet, sparse, dense, vs: ViewSet, reps=5):
    """Per-view time of the learned path (tube splat of the sparse cloud +
    network inference; the network eager, and replayed as a captured CUDA
    graph) and of plain surfel splatting of the dense cloud."""
    dev = model.dev
    ps, _, _ = pipeline.scene_to_device(sparse, dev)
    pd, nd_, rd = pipeline.scene_to_device(dense, dev)
    n = len(vs.views)
    delta = 2.0 * vs.views[0].pitch
    lib = _lib.load()
    x = torch.empty(n * vs.W * vs.W, dtype=torch.bfloat16, device=dev)
    arr = api.views_to_array(vs.views)

    graphed = GraphedUNet(model, n, vs.W, vs.W)

    def coarse():
        keys = api.build_gfb(vs.views, ps, None, None, 1, delta, outputs=("keys",))["keys"]
        check(lib.pe_learned_pairs(arr, n, vs.t_near.ctypes.data_as(C.c_void_p),
                                   vs.t_scale.ctypes.data_as(C.c_void_p), _p(keys), None, _p(x),
                                   None, None, None,
                                   C.c_void_p(torch.cuda.current_stream().cuda_stream)),
              "pe_learned_pairs")

    def learned():
        coarse()
        model.forward(x, n, vs.W, vs.W)

    def learned_graphed():
        coarse()
        graphed.forward(x)

    def plain():
        api.build_gfb(vs.views, pd, nd_, rd, 0, outputs=("nd", "mask"))

    out = {}
    for name, fn in (("learned", learned), ("learned_graphed", learned_graphed),
                     ("plain_splatting", plain)):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t) / reps / n
    return out


def finite_k_study(items: List[dict], Ks=(4, 8, 16), delta_px=2.0, device="cuda:0"):
    """How far the unbounded heap (K = all candidates, the default tube mode)
    is from Alg. 1 with a finite K on the coarse-depth inputs: over the
    targets' views, the fraction of covered pixels whose chosen point
    differs and the RMS depth difference (in units of the ray pitch)."""
    out = {}
    for K in Ks:
        diff, n_hit, sq = 0, 0, 0.0
        for it in items:
            vs = it["vs"]
            pos, _, _ = pipeline.scene_to_device(it["sparse"], device)
            delta = float(delta_px * vs.views[0].pitch)
            kinf = api.build_gfb(vs.views, pos, None, None, 1, delta, outputs=("keys",))["keys"]
            kk = api.build_gfb_topk(vs.views, pos, delta, K)
            hit = kinf != -1
            di = (kinf[hit] & 0xFFFFFFFF) != (kk[hit] & 0xFFFFFFFF)
            dinf = ((kinf[hit] >> 32) & 0xFFFFFFFF).to(torch.int32).view(torch.float32)
            dk = ((kk[hit] >> 32) & 0xFFFFFFFF).to(torch.int32).view(torch.float32)
            diff += int(di.sum())
            n_hit += int(hit.sum())
            sq += float(((dk - dinf).double() / vs.views[0].pitch).pow(2).sum())
        out[f"K={K}"] = {"changed_point_fraction": diff / max(n_hit, 1),
                         "rms_depth_change_pitches": math.sqrt(sq / max(n_hit, 1))}
    return out


def study(n_train=160, n_held=16, views_train=16, views_held=12, W=256, steps=(500, 1500, 3000),
          batch=32, lr0=1e-3, seed=5):
    """Train on pairs from n_train random targets and report, at each step
    count in `steps`, the held-out RCS RMSE (dB) of the network's GFB and of
    the coarse GFB, both against the dense surfel GFB."""
    import scenes
    widths, blocks = (32, 64, 128, 256), (2, 2, 2, 2)
    net = UNet(scenes.unet_init(seed, widths, blocks), widths, blocks, "cuda:0")
    t0 = time.perf_counter()
    train_set = dataset(n_train, views_train, W, seed=seed * 7 + 1)
    held = dataset(n_held, views_held, W, seed=seed * 7 + 2)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    rows, done = [], 0
    for target in steps:
        t1 = time.perf_counter()
        train(net, train_set, target - done, batch, lr0=lr0, seed=seed + done, step0=done)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
        done = target
        res = evaluate(net, held)
        rows.append({"steps": target, "train_s": dt,
                     "rmse_db_learned": float(np.mean([r["learned"] for r in res])),
                     "rmse_db_coarse": float(np.mean([r["coarse"] for r in res]))})
        print(json.dumps(rows[-1]), flush=True)
    return {"pairs": len(train_set) * views_train, "held_out_views": n_held * views_held,
            "W": W, "batch": batch, "data_s": t_data, "checkpoints": rows}


if __name__ == "__main__":
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "study":
        kw = {}
        for a in sys.argv[2:]:
            k, v = a.split("=")
            kw[k] = tuple(int(x) for x in v.split(",")) if k == "steps" else int(v)
        print(json.dumps(study(**kw)))
