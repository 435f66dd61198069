"""Thin torch-facing wrappers over the C ABI (argument marshalling only).

Every step of the path runs in the library's CUDA kernels; torch provides the
device buffers (inputs, outputs and the caller-owned workspaces) and the
stream.  Names follow ``include/pointemray.h``.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from ._lib import PeGeom, PeHits, PeParams, PeSweep, PeView, check

__all__ = ["view_from_angles", "make_params", "build_gfb", "aggregate_views", "alloc_hits",
           "trace_bounces", "po_field", "rcs_sweep", "stream_check", "Geom", "Hits",
           "point_attributes", "build_gfb_topk", "po_field_bistatic", "po_field_every_bounce",
           "views_to_array", "workspace"]


def _lib():
    return L.load()


def _p(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _s(stream):
    st = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(st.cuda_stream)


def _check_out(t: Optional[torch.Tensor], dtype, numel: int, device, what: str):
    """An output the library writes through a raw pointer: refused unless it
    is a contiguous tensor of the right type, size and device."""
    if t is not None and not (t.dtype == dtype and t.is_contiguous() and t.numel() == numel
                              and t.device == torch.device(device)):
        raise ValueError(f"{what}: a contiguous {dtype} tensor of {numel} elements on {device}")


def workspace(nbytes: int, device) -> torch.Tensor:
    """A caller-owned scratch buffer, 256-byte aligned."""
    t = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t[off:off + int(nbytes)]


def view_from_angles(theta_deg: float, phi_deg: float, centre, extent: float, W: int,
                     H: int) -> PeView:
    v = PeView()
    c = (C.c_double * 3)(*[float(x) for x in centre])
    check(_lib().pe_view_from_angles(float(theta_deg), float(phi_deg), c, float(extent),
                                     int(W), int(H), C.byref(v)), "pe_view_from_angles")
    return v


def views_to_array(views: Sequence[PeView]):
    arr = (PeView * len(views))()
    for i, v in enumerate(views):
        arr[i] = v
    return arr


def view_from_struct(o, u, v, d, pitch, W, H) -> PeView:
    """A pe_view for a screen given by its frame (any orthographic screen,
    not only one from angles): centre o, unit pixel axes u and v, ray
    direction d, pixel pitch (m) and size W x H; values rounded to FP32."""
    pv = PeView()
    for k in range(3):
        pv.o[k], pv.u[k], pv.v[k], pv.d[k] = float(o[k]), float(u[k]), float(v[k]), float(d[k])
    pv.pitch, pv.W, pv.H = float(pitch), int(W), int(H)
    return pv


def make_params(pos: np.ndarray, eps: float, overlap_r: float, G: int = 256, tau: float = 3.0,
                delta: float = 0.0, first_bounce_from_geom: bool = False,
                edge_mode: int = 0) -> PeParams:
    """pe_params for a point set: voxel grid over its bounding box with cubic
    voxels of (longest edge)/G, origin and inverse voxel size rounded to FP32."""
    p = np.asarray(pos, dtype=np.float64)
    lo, hi = p.min(axis=0), p.max(axis=0)
    ext = float((hi - lo).max())
    if not (ext > 0.0 and math.isfinite(ext)):
        raise ValueError("the fusion grid spans the points' bounding box: it needs points "
                         "of positive, finite extent")
    prm = PeParams()
    prm.delta = float(delta)
    prm.eps = float(eps)
    prm.overlap_r = float(overlap_r)
    prm.edge_tau = float(tau)
    prm.fuse_grid = int(G)
    for k in range(3):
        prm.bbox_min[k] = float(np.float32(lo[k]))
    prm.inv_voxel = float(np.float32(G / ext))
    prm.first_bounce_from_geom = 1 if first_bounce_from_geom else 0
    prm.edge_mode = int(edge_mode)
    return prm


def stream_check(stream=None):
    check(_lib().pe_stream_check(_s(stream)), "pe_stream_check")


# ----------------------------------------------------------------------------
# a2/a3
# ----------------------------------------------------------------------------

def build_gfb(views: Sequence[PeView], pos: torch.Tensor, nrm: Optional[torch.Tensor],
              rad: Optional[torch.Tensor], mode: int = 0, delta: float = 0.0, stream=None,
              outputs=("nd", "hit", "mask", "keys")) -> dict:
    n = len(views)
    W, H = views[0].W, views[0].H
    dev = pos.device
    arr = views_to_array(views)
    ws_bytes = _lib().pe_build_gfb_workspace(n, arr)
    ws = workspace(ws_bytes, dev)
    out = {}
    npix = n * W * H
    nd = torch.empty((npix, 4), dtype=torch.float32, device=dev) if "nd" in outputs else None
    hit = torch.empty(npix, dtype=torch.int32, device=dev) if "hit" in outputs else None
    mask = torch.empty(npix, dtype=torch.uint8, device=dev) if "mask" in outputs else None
    keys = torch.empty(npix, dtype=torch.int64, device=dev) if "keys" in outputs else None
    check(_lib().pe_build_gfb(arr, n, _p(pos), _p(nrm), _p(rad), pos.shape[0], int(mode),
                              float(delta), _p(ws), ws_bytes, _p(nd), _p(hit), _p(mask),
                              _p(keys), _s(stream)), "pe_build_gfb")
    for k, t in (("nd", nd), ("hit", hit), ("mask", mask), ("keys", keys)):
        if t is not None:
            out[k] = t
    return out


def build_gfb_topk(views: Sequence[PeView], pos: torch.Tensor, delta: float, K: int,
                   stream=None) -> torch.Tensor:
    """Alg. 1 with a finite heap of K points per ray tube
    (``pe_build_gfb_topk``): depth keys [n_views * W * H] (int64 holding the
    uint64 (float bits of depth << 32 | point index), all ones = empty)."""
    n = len(views)
    arr = views_to_array(views)
    ws_bytes = _lib().pe_build_gfb_topk_workspace(n, arr, pos.shape[0], float(delta))
    if ws_bytes == 0:
        raise RuntimeError("pe_build_gfb_topk: unsupported size")
    ws = workspace(ws_bytes, pos.device)
    keys = torch.empty(n * views[0].W * views[0].H, dtype=torch.int64, device=pos.device)
    check(_lib().pe_build_gfb_topk(arr, n, _p(pos), pos.shape[0], float(delta), int(K), _p(ws),
                                   ws_bytes, _p(keys), _s(stream)), "pe_build_gfb_topk")
    return keys


# ----------------------------------------------------------------------------
# a4
# ----------------------------------------------------------------------------

@dataclass
class Geom:
    views: List[PeView]
    blob: torch.Tensor
    c: PeGeom

    def planes(self):
        """(splat_cr, splat_nf) as float32 [total_pix, 4] views of the blob."""
        tot = sum(v.W * v.H for v in self.views)
        f = self.blob.view(torch.float32)
        nf_off = ((tot * 16 + 255) // 256) * 256 // 4
        return f[:tot * 4].view(tot, 4), f[nf_off:nf_off + tot * 4].view(tot, 4)


def point_attributes(pos: torch.Tensor, k_r: int = 8, k_n: int = 16,
                     ref: Optional[torch.Tensor] = None, radius: bool = True, normal: bool = True,
                     stream=None):
    """Surfel radius (mean distance to the k_r nearest other points) and PCA
    normal (k_n nearest points) of every point, on the GPU
    (``pe_point_attributes``).  Returns (radius [n] or None, normal [n,3] or
    None), FP32 on pos's device."""
    lib = _lib()
    n = int(pos.shape[0])
    dev = pos.device
    ws = workspace(lib.pe_point_attributes_workspace(n), dev)
    r = torch.empty(n, dtype=torch.float32, device=dev) if radius else None
    nr = torch.empty(n, 3, dtype=torch.float32, device=dev) if normal else None
    check(lib.pe_point_attributes(_p(pos), n, k_r, k_n, _p(ref), _p(ws), ws.numel(), _p(r), _p(nr),
                                  _s(stream)), "pe_point_attributes")
    return r, nr


def order_points(pos: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """A spatially coherent processing order of the points
    (``pe_order_points``): int32 [n] permutation grouping them by cell of a
    32^3 grid, for SweepArgs.set_point_order."""
    lib = _lib()
    n = int(pos.shape[0])
    if out is not None and not (out.dtype == torch.int32 and out.dim() == 1 and out.is_contiguous()
                                and out.numel() == n and out.device == pos.device):
        raise ValueError("order_points: out must be a contiguous int32 tensor with one entry "
                         "per point, on the points' device")
    ws = workspace(lib.pe_order_points_workspace(n), pos.device)
    order = out if out is not None else torch.empty(n, dtype=torch.int32, device=pos.device)
    check(lib.pe_order_points(_p(pos), n, _p(ws), ws.numel(), _p(order), _s(stream)),
          "pe_order_points")
    return order


def alloc_geom(views: Sequence[PeView], device) -> Geom:
    n = len(views)
    arr = views_to_array(views)
    nbytes = _lib().pe_geom_bytes(n, arr)
    if nbytes == 0:
        raise ValueError("invalid views for a geometry")
    blob = workspace(nbytes, device)
    g = PeGeom()
    g.n_views = n
    for i, v in enumerate(views):
        g.views[i] = v
    g.blob_dev = blob.data_ptr()
    g.blob_bytes = nbytes
    return Geom(list(views), blob, g)


def aggregate_views(views: Sequence[PeView], gfb_nd: torch.Tensor, gfb_mask: torch.Tensor,
                    params: PeParams, stream=None, geom: Optional[Geom] = None) -> Geom:
    n = len(views)
    arr = views_to_array(views)
    geom = geom or alloc_geom(views, gfb_nd.device)
    ws_bytes = _lib().pe_aggregate_workspace(n, arr, params.fuse_grid)
    ws = workspace(ws_bytes, gfb_nd.device)
    check(_lib().pe_aggregate_views(arr, n, _p(gfb_nd), _p(gfb_mask), C.byref(params), _p(ws),
                                    ws_bytes, C.byref(geom.c), _s(stream)), "pe_aggregate_views")
    return geom


# ----------------------------------------------------------------------------
# a5
# ----------------------------------------------------------------------------

@dataclass
class Hits:
    p: torch.Tensor
    n: torch.Tensor
    k: torch.Tensor
    u: torch.Tensor
    v: torch.Tensor
    path: torch.Tensor
    M: torch.Tensor
    psi: torch.Tensor
    ids: Optional[torch.Tensor]
    c: PeHits = field(default=None)


def alloc_hits(n_rays: int, mb: int, device, ids: bool = True) -> Hits:
    f3 = lambda: torch.zeros((n_rays, 3), dtype=torch.float32, device=device)
    h = Hits(f3(), f3(), f3(), f3(), f3(), torch.zeros(n_rays, dtype=torch.float64, device=device),
             torch.zeros(n_rays, dtype=torch.int32, device=device),
             torch.zeros(n_rays, dtype=torch.uint8, device=device),
             torch.zeros((mb, n_rays), dtype=torch.int32, device=device) if ids else None)
    c = PeHits()
    for name in ("p", "n", "k", "u", "v", "path", "M", "psi", "ids"):
        t = getattr(h, name)
        setattr(c, name, None if t is None else t.data_ptr())
    c.n_rays = n_rays
    c.max_bounces = mb
    h.c = c
    return h


def trace_bounces(views: Sequence[PeView], keys: Optional[torch.Tensor],
                  nrm: Optional[torch.Tensor], geom: Optional[Geom], max_bounces: int,
                  params: PeParams, hits: Optional[Hits] = None,
                  stats: Optional[torch.Tensor] = None, stream=None, ids: bool = True) -> Hits:
    n = len(views)
    arr = views_to_array(views)
    n_rays = n * views[0].W * views[0].H
    dev = (keys if keys is not None else geom.blob).device
    hits = hits or alloc_hits(n_rays, max_bounces, dev, ids)
    ws_bytes = _lib().pe_trace_workspace(n, arr)
    ws = workspace(ws_bytes, dev)
    check(_lib().pe_trace_bounces(arr, n, _p(keys), _p(nrm),
                                  C.byref(geom.c) if geom is not None else None,
                                  int(max_bounces), C.byref(params), _p(ws), ws_bytes,
                                  C.byref(hits.c), _p(stats), _s(stream)), "pe_trace_bounces")
    return hits


# ----------------------------------------------------------------------------
# a6
# ----------------------------------------------------------------------------

def po_field(hits: Hits, n_groups: int, rays_per_group: int, ks: np.ndarray,
             freqs_hz: np.ndarray, stream=None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    ks = np.ascontiguousarray(ks, dtype=np.float32).reshape(n_groups, 3)
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64).ravel()
    dev = hits.M.device
    _check_out(out, torch.float64, n_groups * fr.shape[0] * 12, dev, "po_field: out")
    E = out if out is not None else torch.empty((n_groups, fr.shape[0], 2, 3, 2),
                                                dtype=torch.float64, device=dev)
    ws_bytes = _lib().pe_po_workspace(n_groups, rays_per_group, fr.shape[0])
    ws = workspace(ws_bytes, dev)
    check(_lib().pe_po_field(C.byref(hits.c), n_groups, rays_per_group,
                             ks.ctypes.data_as(C.c_void_p), fr.ctypes.data_as(C.c_void_p),
                             fr.shape[0], _p(ws), ws_bytes, _p(E), _s(stream)), "pe_po_field")
    return E


def po_field_every_bounce(views: Sequence[PeView], keys: Optional[torch.Tensor],
                          nrm: Optional[torch.Tensor], geom: "Geom", params: PeParams,
                          max_bounces: int, freqs_hz: np.ndarray, stream=None) -> torch.Tensor:
    """PO at every bounce (``pe_po_field_every_bounce``): float64
    [n_views, F, 2 pol, 3, re/im]."""
    n = len(views)
    arr = views_to_array(views)
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64).ravel()
    dev = geom.blob.device
    ws_bytes = _lib().pe_po_field_every_bounce_workspace(n, arr, fr.shape[0])
    if ws_bytes == 0:
        raise ValueError("pe_po_field_every_bounce: invalid views or frequencies")
    ws = workspace(ws_bytes, dev)
    E = torch.empty((n, fr.shape[0], 2, 3, 2), dtype=torch.float64, device=dev)
    check(_lib().pe_po_field_every_bounce(arr, n, _p(keys), _p(nrm), C.byref(geom.c),
                                          int(max_bounces), C.byref(params),
                                          fr.ctypes.data_as(C.c_void_p), fr.shape[0], _p(ws),
                                          ws_bytes, _p(E), _s(stream)),
          "pe_po_field_every_bounce")
    return E


def po_field_bistatic(hits: Hits, n_groups: int, rays_per_group: int, obs_dirs: np.ndarray,
                      geom: "Geom", eps: float, freqs_hz: np.ndarray, only_bounce: int = 0,
                      stream=None) -> torch.Tensor:
    """Eq. 14 toward n_obs receivers per group, Psi tested toward each
    (``pe_po_field_bistatic``).  obs_dirs: [n_groups, n_obs, 3].  Returns
    float64 [n_groups, n_obs, F, 2 pol, 3, re/im]."""
    obs = np.ascontiguousarray(obs_dirs, dtype=np.float32)
    n_obs = obs.shape[1]
    fr = np.ascontiguousarray(freqs_hz, dtype=np.float64).ravel()
    dev = hits.M.device
    E = torch.empty((n_groups, n_obs, fr.shape[0], 2, 3, 2), dtype=torch.float64, device=dev)
    ws_bytes = _lib().pe_po_field_bistatic_workspace(n_groups, rays_per_group, fr.shape[0])
    ws = workspace(ws_bytes, dev)
    check(_lib().pe_po_field_bistatic(C.byref(hits.c), n_groups, rays_per_group,
                                      obs.ctypes.data_as(C.c_void_p), n_obs, C.byref(geom.c),
                                      float(eps), int(only_bounce), fr.ctypes.data_as(C.c_void_p),
                                      fr.shape[0],
                                      _p(ws), ws_bytes, _p(E), _s(stream)), "pe_po_field_bistatic")
    return E


# ----------------------------------------------------------------------------
# a1/a7
# ----------------------------------------------------------------------------

class SweepArgs:
    """Keeps the host arrays a PeSweep points to alive."""

    def __init__(self, theta_deg, phi_deg, W, H, centre, extent, freqs_hz, max_bounces,
                 angle_batch=0):
        self.theta = np.ascontiguousarray(theta_deg, dtype=np.float64)
        self.phi = np.ascontiguousarray(phi_deg, dtype=np.float64)
        self.freqs = np.ascontiguousarray(freqs_hz, dtype=np.float64)
        s = PeSweep()
        s.n_angles = self.theta.shape[0]
        s.theta_deg = self.theta.ctypes.data
        s.phi_deg = self.phi.ctypes.data
        s.W, s.H = int(W), int(H)
        for k in range(3):
            s.centre[k] = float(centre[k])
        s.extent = float(extent)
        s.n_freq = self.freqs.shape[0]
        s.freqs_hz = self.freqs.ctypes.data
        s.max_bounces = int(max_bounces)
        s.angle_batch = int(angle_batch)
        s.point_order = None
        self.order = None
        self.c = s

    def set_point_order(self, order: Optional[torch.Tensor]):
        """The incidence splat's processing order of the points (device
        int32 permutation from order_points, or None); it does not change
        the results.  The tensor must stay alive while the sweep runs."""
        self.order = order
        self.c.point_order = None if order is None else order.data_ptr()

    @classmethod
    def from_sweep(cls, sw, angle_batch=0):
        return cls(sw.theta_deg, sw.phi_deg, sw.W, sw.H, sw.centre, sw.extent, sw.freqs_hz,
                   sw.max_bounces, angle_batch)

    def workspace_bytes(self) -> int:
        return _lib().pe_rcs_sweep_workspace(C.byref(self.c))


def rcs_sweep(args: SweepArgs, pos: torch.Tensor, nrm: torch.Tensor, rad: torch.Tensor,
              geom: Optional[Geom], params: PeParams, stream=None, ws: Optional[torch.Tensor] = None,
              E: Optional[torch.Tensor] = None, sigma: Optional[torch.Tensor] = None,
              stats: Optional[torch.Tensor] = None):
    """Returns (E [A][F][2][3][2] f64, sigma [A][F][2][2] f64) on the device."""
    s = args.c
    dev = pos.device
    o = getattr(args, "order", None)
    if o is not None and not (o.dtype == torch.int32 and o.dim() == 1 and o.is_contiguous()
                              and o.numel() == pos.shape[0] and o.device == dev):
        # the library reads n_points entries through the raw pointer
        raise ValueError("point order: a contiguous int32 tensor with one entry per point, "
                         "on the points' device")
    _check_out(E, torch.float64, s.n_angles * s.n_freq * 12, dev, "rcs_sweep: E")
    _check_out(sigma, torch.float64, s.n_angles * s.n_freq * 4, dev, "rcs_sweep: sigma")
    nbytes = args.workspace_bytes()
    if nbytes == 0:
        raise ValueError("invalid sweep")
    if ws is None or ws.numel() < nbytes:
        ws = workspace(nbytes, dev)
    if E is None:
        E = torch.empty((s.n_angles, s.n_freq, 2, 3, 2), dtype=torch.float64, device=dev)
    if sigma is None:
        sigma = torch.empty((s.n_angles, s.n_freq, 2, 2), dtype=torch.float64, device=dev)
    check(_lib().pe_rcs_sweep(C.byref(s), _p(pos), _p(nrm), _p(rad), pos.shape[0],
                              C.byref(geom.c) if geom is not None else None, C.byref(params),
                              _p(ws), nbytes, _p(E), _p(sigma), _p(stats), _s(stream)),
          "pe_rcs_sweep")
    return E, sigma
