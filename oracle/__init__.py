"""PointEMRay CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(and its ``--impl reference`` arm) may import this package.  The product path
(``paper_2408_15583_gb300``) never imports it and shares no code with it.

What it computes (PointEMRay, arXiv 2408.15583), step by step and by brute
force (large searches take their candidates from a uniform grid instead, with
the same result bit for bit: ``oracle_grid.h``):
  a1  view / ray screen from (theta, phi)          Sec. III-A (uvwo frame)
  a2  PRI: nearest point per pixel ray (GFB)        Alg. 1, surfel or tube
  a3  GFB resolve (depth, oriented normal, mask)    Alg. 1 output, Eq. 16 frame
  a4  edge filter + 256^3 voxel fusion + Eq. 22     Alg. 3, aggregation steps
  a5  bounce tracing with Eq. 23 overlap + epsilon  Alg. 3, bounce loop, Eq. 2-4
  a6  PO field sum (FP64, Neumaier)                 Eq. 5-14
  a7  monostatic RCS sigma = k^2/pi |e . Sigma|^2   Eq. 14 + far field
Two arithmetic modes: ``fp32`` (geometry in FP32 with a fixed op order: the
bit-exact target for hit ids and bounce counts) and ``fp64`` (physics).
Readings of passages the paper leaves open are listed in the repository's
design notes; the ones that change arithmetic are repeated in the docstrings.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle_core.h"),
        os.path.join(_HERE, "oracle_grid.h")]

C0 = 299_792_458.0


def _compile(src_c: str, out_so: str) -> None:
    """gcc -O2 -ffp-contract=off (no fast-math), OpenMP if present, of
    oracle.c (which includes oracle_core.h from its own directory)."""
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
            "-fPIC", "-shared", src_c, "-o", out_so, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)


def build(force: bool = False) -> str:
    """Compile the C oracle."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(s) <= so_t for s in _SRC):
            return _SO
    _compile(_SRC[0], _SO + ".tmp")
    os.replace(_SO + ".tmp", _SO)
    return _SO


class OrView(C.Structure):
    _fields_ = [("o", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3),
                ("d", C.c_double * 3), ("pitch", C.c_double), ("W", C.c_int32),
                ("H", C.c_int32)]


_lib = None


def _bind(path: str):
    """Load a build of the C oracle and declare its entry points."""
    L = C.CDLL(path)
    P = C.c_void_p
    L.or_gfb.argtypes = [C.c_int, P, P, P, P, C.c_int64, C.c_int, C.c_double,
                         P, C.c_int64, C.c_int, P, P, P]
    L.or_aggregate.argtypes = [C.c_int, C.c_int, P, P, P, P, C.c_double, C.c_int, P,
                               C.c_double, C.c_int, P, P, P, P, P, P]
    L.or_aggregate.restype = C.c_int64
    L.or_trace.argtypes = [C.c_int, P, P, C.c_int64, P, P, P, P, P, P, P,
                           C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                           P, P, P, P, P, P, P, P, P]
    L.or_po_field.argtypes = [C.c_int64, P, P, P, P, P, P, P, C.c_int, P,
                              C.c_int, P, P]
    L.or_knn.argtypes = [P, C.c_int64, P, C.c_int64, C.c_int, P, P]
    L.or_shadow_dirs.argtypes = [C.c_int, P, P, P, P, C.c_int64, P, P, C.c_int64, P,
                                 C.c_int, C.c_double, C.c_int, P]
    L.or_acc_sum.argtypes = [P, C.c_int64, P]
    L.or_set_threads.argtypes = [C.c_int]
    L.or_set_threads.restype = C.c_int
    L.or_gfb_topk.argtypes = [C.c_int, P, P, C.c_int64, C.c_double, C.c_int, P, C.c_int64,
                              P, P]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops (n >= 1; 0 only queries)."""
    return int(lib().or_set_threads(int(n)))


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ----------------------------------------------------------------------------
# a1: view frame (Sec. III-A): w from the target toward the transmitter,
# u = theta_hat, v = phi_hat (u x v = w), rays travel along d = -w from a
# screen plane outside the target's bounding sphere.
# ----------------------------------------------------------------------------

@dataclass
class View:
    o: np.ndarray
    u: np.ndarray
    v: np.ndarray
    d: np.ndarray
    pitch: float
    W: int
    H: int

    def c(self) -> OrView:
        s = OrView()
        for k in range(3):
            s.o[k], s.u[k], s.v[k], s.d[k] = self.o[k], self.u[k], self.v[k], self.d[k]
        s.pitch, s.W, s.H = self.pitch, self.W, self.H
        return s


def view_from_angles(theta_deg: float, phi_deg: float, centre, extent: float,
                     W: int, H: int, mode: str = "fp32") -> View:
    th = float(theta_deg) * (math.pi / 180.0)
    ph = float(phi_deg) * (math.pi / 180.0)
    st, ct, sp, cp = math.sin(th), math.cos(th), math.sin(ph), math.cos(ph)
    w = [st * cp, st * sp, ct]
    u = [ct * cp, ct * sp, -st]
    v = [-sp, cp, 0.0]
    L = (2.0 * float(extent)) / float(W)
    D = float(extent) + L
    o = [float(centre[k]) + D * w[k] for k in range(3)]
    d = [-w[k] for k in range(3)]
    if mode == "fp32":
        r = lambda a: np.array(a, dtype=np.float32).astype(np.float64)
        return View(r(o), r(u), r(v), r(d), float(np.float32(L)), W, H)
    return View(np.array(o), np.array(u), np.array(v), np.array(d), L, W, H)


def _fp(mode):
    return 1 if mode == "fp64" else 0


# ----------------------------------------------------------------------------
# a2/a3: GFB (Alg. 1)
# ----------------------------------------------------------------------------

@dataclass
class Gfb:
    depth: np.ndarray   # [npix] float64 (+inf on a miss)
    idx: np.ndarray     # [npix] int64 (-1 on a miss)
    nrm: np.ndarray     # [npix,3] float64, turned to face the view
    view: View
    pix: Optional[np.ndarray]

    @property
    def mask(self):
        return (self.idx >= 0).astype(np.uint8)

    def keys(self) -> np.ndarray:
        """Packed (float bits of depth) << 32 | index, UINT64_MAX on a miss."""
        t32 = self.depth.astype(np.float32)
        bits = t32.view(np.uint32).astype(np.uint64)
        k = (bits << np.uint64(32)) | (self.idx.astype(np.uint64) & np.uint64(0xFFFFFFFF))
        k[self.idx < 0] = np.uint64(0xFFFFFFFFFFFFFFFF)
        return k


# Searches over more element/ray pairs than this take their candidates from a
# uniform grid (oracle_grid.h: the same result as brute force, bit for bit).
GRID_ABOVE = 2_000_000


def _use_grid(accel: str, n_elem: int, n_query: int) -> int:
    """accel: "brute" (every element for every ray), "grid", or "auto"
    (the grid only for large searches)."""
    if accel == "brute":
        return 0
    if accel == "grid":
        return 1
    if accel != "auto":
        raise ValueError(f"accel must be 'auto', 'grid' or 'brute', not {accel!r}")
    return 1 if int(n_elem) * int(n_query) > GRID_ABOVE else 0


def gfb(scene, view: View, mode: str = "fp32", tube: bool = False, delta: float = 0.0,
        pix: Optional[np.ndarray] = None, accel: str = "auto") -> Gfb:
    """Alg. 1 for every pixel of `view` (or the listed ones): the nearest
    point per pixel ray, surfel mode (disks of radius rad with normal nrm) or
    tube mode (points within delta of the ray, scored by Length(p - o))."""
    pos = np.ascontiguousarray(scene.pos, dtype=np.float32)
    nrm = np.ascontiguousarray(scene.nrm, dtype=np.float32)
    rad = np.ascontiguousarray(scene.rad, dtype=np.float32)
    npix = view.W * view.H if pix is None else len(pix)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    depth = np.empty(npix, np.float64)
    idx = np.empty(npix, np.int64)
    nout = np.empty((npix, 3), np.float64)
    vc = view.c()
    lib().or_gfb(_fp(mode), C.byref(vc), _p(pos), _p(nrm), _p(rad), pos.shape[0],
                 1 if tube else 0, float(delta), _p(pixa), npix,
                 _use_grid(accel, pos.shape[0], npix), _p(depth), _p(idx), _p(nout))
    return Gfb(depth, idx, nout, view, pixa)


def gfb_topk(pos: np.ndarray, view: View, delta: float, K: int, mode: str = "fp32",
             pix: Optional[np.ndarray] = None) -> Gfb:
    """Alg. 1 with a finite heap of K points per ray tube (1 <= K <= 64):
    the K candidates nearest the central ray, then the one nearest the
    tube's origin."""
    assert 1 <= K <= 64
    p = np.ascontiguousarray(pos, dtype=np.float32)
    npix = view.W * view.H if pix is None else len(pix)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    depth = np.empty(npix, np.float64)
    idx = np.empty(npix, np.int64)
    vc = view.c()
    lib().or_gfb_topk(_fp(mode), C.byref(vc), _p(p), p.shape[0], float(delta), int(K), _p(pixa),
                      npix, _p(depth), _p(idx))
    return Gfb(depth, idx, np.zeros((npix, 3)), view, pixa)


# ----------------------------------------------------------------------------
# a4: aggregation (Alg. 3, aggregation steps, Eq. 22)
# ----------------------------------------------------------------------------

@dataclass
class Splats:
    id: np.ndarray      # int64, global owner-pixel index (sorted)
    c: np.ndarray       # [n,3]
    n: np.ndarray       # [n,3]
    r: np.ndarray       # [n]
    count: np.ndarray   # contributors per voxel
    keep: np.ndarray    # per GFB pixel: 1 if it survived the edge filter

    @property
    def ns(self):
        return int(self.id.shape[0])


@dataclass
class FuseParams:
    tau: float
    bmin: np.ndarray    # float32-representable
    inv_vox: float      # float32-representable
    G: int = 256
    edge_mode: int = 0  # 0: the edge rule of c14; 1: Canny on the depth map


def fuse_params(scene, G: int = 256, tau: float = 3.0) -> FuseParams:
    """Voxel grid over the point bounding box: cubic voxels, edge = longest
    bbox edge / G (Sec. III-B); values rounded to FP32."""
    lo, hi = scene.bbox()
    ext = float((hi - lo).max())
    if not (ext > 0.0 and np.isfinite(ext)):
        # the grid over the bounding box (Sec. III-B) is undefined for a box
        # of zero extent
        raise ValueError("fusion grid: the points' bounding box has zero extent")
    return FuseParams(tau=float(np.float32(tau)),
                      bmin=lo.astype(np.float32).astype(np.float64),
                      inv_vox=float(np.float32(G / ext)), G=G)


def aggregate(gfbs, fp: FuseParams, mode: str = "fp32") -> Splats:
    views = (OrView * len(gfbs))(*[g.view.c() for g in gfbs])
    depth = np.ascontiguousarray(np.concatenate([np.where(g.idx >= 0, g.depth, 0.0) for g in gfbs]))
    nrm = np.ascontiguousarray(np.concatenate([g.nrm for g in gfbs]))
    mask = np.ascontiguousarray(np.concatenate([g.mask for g in gfbs]))
    tot = depth.shape[0]
    oid = np.empty(tot, np.int64)
    oc = np.empty((tot, 3), np.float64)
    on = np.empty((tot, 3), np.float64)
    orr = np.empty(tot, np.float64)
    ocnt = np.empty(tot, np.int32)
    keep = np.empty(tot, np.uint8)
    bmin = np.ascontiguousarray(fp.bmin, dtype=np.float64)
    ns = lib().or_aggregate(_fp(mode), len(gfbs), views, _p(depth), _p(nrm), _p(mask),
                            fp.tau, int(fp.edge_mode), _p(bmin), fp.inv_vox, fp.G, _p(oid),
                            _p(oc), _p(on),
                            _p(orr), _p(ocnt), _p(keep))
    return Splats(oid[:ns].copy(), oc[:ns].copy(), on[:ns].copy(), orr[:ns].copy(),
                  ocnt[:ns].copy(), keep)


# ----------------------------------------------------------------------------
# a5: bounce tracing (Alg. 3, Eq. 23)
# ----------------------------------------------------------------------------

@dataclass
class Trace:
    M: np.ndarray       # [nr] bounces (hits)
    ids: np.ndarray     # [nr, mb] hit ids per bounce, -1 after the last
    p: np.ndarray
    n: np.ndarray
    k: np.ndarray
    u: np.ndarray
    v: np.ndarray
    path: np.ndarray
    psi: np.ndarray


def trace(view: View, splats: Optional[Splats], mb: int, eps: float, r_ov: float,
          first: Optional[Gfb] = None, pix: Optional[np.ndarray] = None,
          mode: str = "fp32", shadow: bool = True, accel: str = "auto") -> Trace:
    """Alg. 3's bounce loop for every pixel ray of `view` (or the listed
    ones): bounce 1 from `first` (the view's GFB) or from the splats, then
    up to mb - 1 reflections (Eq. 4) through the splats with the Eq. 23
    overlap rule and minimum travel eps, and Psi toward the transmitter."""
    if pix is None and first is not None:
        pix = first.pix
    nr = view.W * view.H if pix is None else len(pix)
    pixa = None if pix is None else np.ascontiguousarray(pix, dtype=np.int64)
    if splats is None:
        sc = np.zeros((0, 3)); sn = np.zeros((0, 3)); sr = np.zeros(0); sid = np.zeros(0, np.int64)
    else:
        sc, sn, sr, sid = (np.ascontiguousarray(splats.c), np.ascontiguousarray(splats.n),
                           np.ascontiguousarray(splats.r), np.ascontiguousarray(splats.id))
    M = np.empty(nr, np.int32)
    ids = np.empty((nr, mb), np.int64)
    out = [np.empty((nr, 3), np.float64) for _ in range(5)]
    path = np.empty(nr, np.float64)
    psi = np.empty(nr, np.uint8)
    vc = view.c()
    ft = fi = fn = None
    if first is not None:
        ft = np.ascontiguousarray(first.depth)
        fi = np.ascontiguousarray(first.idx)
        fn = np.ascontiguousarray(first.nrm)
    lib().or_trace(_fp(mode), C.byref(vc), _p(pixa), nr, _p(ft), _p(fi), _p(fn),
                   _p(sc), _p(sn), _p(sr), _p(sid), sid.shape[0], mb, float(eps),
                   float(r_ov), 1 if shadow else 0,
                   _use_grid(accel, sid.shape[0], nr * max(1, mb)), _p(M), _p(ids),
                   *[_p(a) for a in out],
                   _p(path), _p(psi))
    return Trace(M, ids, *out, path, psi)


# ----------------------------------------------------------------------------
# a6/a7: PO field (Eq. 14) and RCS
# ----------------------------------------------------------------------------

def po_field(tr: Trace, freqs_hz, ks_dirs) -> np.ndarray:
    """Sigma of Eq. 14 (without -j eta0 k0 / 2pi) as complex [obs][F][pol][3],
    pol 0 = V (E along theta_hat), 1 = H (E along phi_hat)."""
    freqs = np.ascontiguousarray(np.atleast_1d(freqs_hz), dtype=np.float64)
    ks = np.ascontiguousarray(np.atleast_2d(ks_dirs), dtype=np.float64)
    use = np.ascontiguousarray(((tr.M > 0) & (tr.psi > 0)).astype(np.uint8))
    nr = tr.M.shape[0]
    E = np.empty((ks.shape[0], freqs.shape[0], 2, 3, 2), np.float64)
    arr = [np.ascontiguousarray(a) for a in (tr.p, tr.n, tr.k, tr.u, tr.v, tr.path)]
    lib().or_po_field(nr, *[_p(a) for a in arr], _p(use), freqs.shape[0], _p(freqs),
                      ks.shape[0], _p(ks), _p(E))
    return E[..., 0] + 1j * E[..., 1]


def shadow_dirs(tr: Trace, splats: Splats, dirs, eps: float, mode: str = "fp32",
                accel: str = "auto") -> np.ndarray:
    """Psi toward other receivers (bistatic): [nobs][nr] uint8, 1 unless a
    splat is hit from the ray's last hit point along dirs[o] (t > eps); 0 for
    rays without a hit."""
    d = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    nr = tr.M.shape[0]
    psi = np.empty((d.shape[0], nr), np.uint8)
    arr = [np.ascontiguousarray(a) for a in (splats.c, splats.n, splats.r, splats.id)]
    lib().or_shadow_dirs(_fp(mode), *[_p(a) for a in arr], arr[3].shape[0],
                         _p(np.ascontiguousarray(tr.p)), _p(np.ascontiguousarray(tr.M)), nr,
                         _p(d), d.shape[0], float(eps),
                         _use_grid(accel, arr[3].shape[0], nr * d.shape[0]), _p(psi))
    return psi


def po_field_bistatic(tr: Trace, splats: Splats, freqs_hz, obs_dirs, eps: float,
                      mode: str = "fp32", only_bounce: int = 0) -> np.ndarray:
    """Eq. 14 toward each receiver direction of obs_dirs, with Psi tested
    toward that receiver (only rays with M == only_bounce if > 0):
    complex [obs][F][pol][3]."""
    obs = np.atleast_2d(np.asarray(obs_dirs, np.float64))
    psi = shadow_dirs(tr, splats, obs, eps, mode)
    if only_bounce > 0:
        psi = psi * (tr.M == only_bounce).astype(np.uint8)[None]
    out = []
    for o in range(obs.shape[0]):
        t = Trace(tr.M, tr.ids, tr.p, tr.n, tr.k, tr.u, tr.v, tr.path, psi[o])
        out.append(po_field(t, freqs_hz, obs[o])[0])
    return np.array(out)


def po_field_every_bounce(view: View, splats: Splats, first: Gfb, mb: int, eps: float,
                          r_ov: float, freqs_hz, mode: str = "fp32") -> np.ndarray:
    """PO at every bounce instead of Eq. 14's last hit: for b = 1..mb, the
    rays traced to b bounces whose b-th hit is their last contribute Eq. 14
    at that hit, with Psi toward the (monostatic) receiver; the fields are
    summed.  complex [F][pol][3]."""
    w = -np.asarray(view.d, np.float64)
    E = 0.0
    for b in range(1, mb + 1):
        tr = trace(view, splats, b, eps, r_ov, first=first, mode=mode)
        psi = shadow_dirs(tr, splats, [w], eps, mode)[0] * (tr.M == b).astype(np.uint8)
        t = Trace(tr.M, tr.ids, tr.p, tr.n, tr.k, tr.u, tr.v, tr.path, psi)
        E = E + po_field(t, freqs_hz, w)[0]
    return E


def sigma_from_field(E: np.ndarray, freqs_hz, u_hat, v_hat) -> np.ndarray:
    """sigma[f][tx][rx] = k^2/pi |e_rx . Sigma_tx|^2 (m^2); e_V = u_hat
    (theta_hat), e_H = v_hat (phi_hat).  E is [F][pol][3] complex."""
    k = 2.0 * math.pi * np.asarray(freqs_hz, dtype=np.float64) / C0
    e = np.stack([np.asarray(u_hat, np.float64), np.asarray(v_hat, np.float64)])
    proj = np.einsum("ftc,rc->ftr", E, e)
    return (k[:, None, None] ** 2 / math.pi) * np.abs(proj) ** 2


def db(x):
    return 10.0 * np.log10(np.maximum(np.asarray(x, dtype=np.float64), 1e-30))


@dataclass
class SweepResult:
    E: np.ndarray       # [A][F][pol][3] complex
    sigma: np.ndarray   # [A][F][tx][rx] m^2
    traces: list
    views: list


def sweep_views(sweep, mode="fp32"):
    return [view_from_angles(sweep.theta_deg[a], sweep.phi_deg[a], sweep.centre, sweep.extent,
                             sweep.W, sweep.H, mode) for a in range(sweep.n_angles)]


def gfb_views(views_desc, mode="fp32"):
    return [view_from_angles(views_desc.theta_deg[a], views_desc.phi_deg[a], views_desc.centre,
                             views_desc.extent, views_desc.W, views_desc.H, mode)
            for a in range(len(views_desc.theta_deg))]


def default_eps(gviews) -> float:
    """epsilon = r = the smallest aggregation-view pitch (the paper leaves
    both unset)."""
    return float(min(v.pitch for v in gviews))


def build_geometry(scene, views_desc, mode="fp32", G=256, tau=3.0):
    gv = gfb_views(views_desc, mode)
    gf = [gfb(scene, v, mode) for v in gv]
    fp = fuse_params(scene, G, tau)
    return aggregate(gf, fp, mode), gv, gf, fp


def rcs_sweep(scene, sweep, splats: Optional[Splats], eps: float, r_ov: float,
              mode: str = "fp32", angles=None, pix=None, first_from_geom=False) -> SweepResult:
    """Monostatic sweep: per angle, GFB at the ray screen (bounce 1), bounces
    2..mb through the splats, Psi, PO sum, sigma."""
    angles = range(sweep.n_angles) if angles is None else angles
    Es, sig, trs, vs = [], [], [], []
    for a in angles:
        v = view_from_angles(sweep.theta_deg[a], sweep.phi_deg[a], sweep.centre,
                             sweep.extent, sweep.W, sweep.H, mode)
        first = None if first_from_geom else gfb(scene, v, mode, pix=pix)
        tr = trace(v, splats if sweep.max_bounces > 1 or first_from_geom else None,
                   sweep.max_bounces, eps, r_ov, first=first, pix=pix, mode=mode)
        ks = -np.asarray(v.d, dtype=np.float64)
        E = po_field(tr, sweep.freqs_hz, ks)[0]
        Es.append(E)
        sig.append(sigma_from_field(E, sweep.freqs_hz, v.u, v.v))
        trs.append(tr)
        vs.append(v)
    return SweepResult(np.array(Es), np.array(sig), trs, vs)


# ----------------------------------------------------------------------------
# Surfel attributes: radius from the k nearest other points (mean distance)
# and the PCA normal of the k nearest points (the smallest principal axis),
# the per-point inputs of Alg. 1 in surfel mode.
# ----------------------------------------------------------------------------

def knn(pos: np.ndarray, K: int, queries=None):
    """Brute-force K nearest points (itself included) of every point, or of
    the points listed in `queries`: indices [nq][K] and FP32 squared
    distances, ordered by (d2, index)."""
    p = np.ascontiguousarray(pos, dtype=np.float32)
    n = p.shape[0]
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = n if q is None else q.shape[0]
    idx = np.empty((nq, K), np.int64)
    d2 = np.empty((nq, K), np.float32)
    lib().or_knn(_p(p), n, _p(q), nq, K, _p(idx), _p(d2))
    return idx, d2


def knn_radius(idx: np.ndarray, d2: np.ndarray, self_idx: np.ndarray, k_r: int) -> np.ndarray:
    """Mean distance to the first k_r neighbours other than the point itself
    (square roots and sum in FP64 in list order, rounded once to FP32)."""
    out = np.empty(idx.shape[0], np.float32)
    for r in range(idx.shape[0]):
        s, used = 0.0, 0
        for e in range(idx.shape[1]):
            if used == k_r:
                break
            if idx[r, e] == self_idx[r]:
                continue
            s += math.sqrt(float(d2[r, e]))
            used += 1
        out[r] = np.float32(s / k_r)
    return out


def point_attributes(pos: np.ndarray, k_r: int = 8, k_n: int = 16, ref=None):
    """radius[i] = mean distance to the k_r nearest other points (square
    roots and sum in FP64, in neighbour order, rounded once to FP32);
    normal[i] = unit eigenvector of the smallest eigenvalue of the FP64
    covariance of the k_n nearest points (itself included), turned to agree
    with ref[i] if given, else to point away from the bounding-box centre.
    Also returns the three eigenvalues (ascending) per point."""
    p = np.ascontiguousarray(pos, dtype=np.float32)
    K = max(k_r + 1, k_n)
    idx, d2 = knn(p, K)
    n = p.shape[0]
    rad = knn_radius(idx, d2, np.arange(n), k_r)
    nb = p.astype(np.float64)[idx[:, :k_n]]                 # [n, k_n, 3]
    m = nb.sum(axis=1) / k_n
    c = nb - m[:, None, :]
    cov = np.einsum("nki,nkj->nij", c, c)
    w, vec = np.linalg.eigh(cov)
    nrm = vec[:, :, 0]
    if ref is not None:
        flip = (nrm * np.asarray(ref, np.float64)).sum(axis=1) < 0
    else:
        lo, hi = p.astype(np.float64).min(axis=0), p.astype(np.float64).max(axis=0)
        flip = (nrm * (p.astype(np.float64) - 0.5 * (lo + hi))).sum(axis=1) < 0
    nrm[flip] *= -1.0
    return rad, nrm, w, idx
