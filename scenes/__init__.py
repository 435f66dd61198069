"""Seeded synthetic scenes and sweeps shaped like PointEMRay's workloads.

This module only *produces inputs*: point positions, normals, surfel radii and
the (theta, phi, screen, frequency) descriptions of monostatic sweeps.  It holds
none of the method's arithmetic (no view frames, no ray/splat intersection, no
field sums), so both the CUDA path and the CPU oracle can consume it.

Shapes follow the paper's experiments (Sec. IV): targets scaled to metre/10 m
class boxes, 10k-1M points sampled on the surface, ray pitch about lambda/10,
8 aggregation views at theta in {60, 120} x phi in {45, 135, 225, 315} deg
(Sec. IV-B, the OctAR set-up).  The paper's Free3D meshes are not available, so
analytic primitives (plates, dihedral, trihedral, sphere, cylinder) stand in for
them.

Surfel radii (mean distance to the 8 nearest neighbours) and PCA normals
(16 neighbours) are *inputs* to both sides; they are computed here in FP64 with
scipy's k-d tree and rounded once to FP32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

C0 = 299_792_458.0  # speed of light, m/s

__all__ = [
    "C0", "Scene", "Sweep", "GfbViews", "Workload",
    "knn_radius", "pca_normals", "bounding_sphere",
    "plate", "dihedral", "trihedral", "sphere", "cylinder", "composite", "octar",
    "random_primitives", "aggregation_views", "freq_grid", "c5_target",
    "workload_dihedral", "workload_sphere", "workload_composite", "workload_octar",
    "workload_small",
]


@dataclass
class Scene:
    """A point-sampled PEC target.  pos/nrm are float32 [N,3], rad float32 [N]."""
    pos: np.ndarray
    nrm: np.ndarray
    rad: np.ndarray
    name: str = "scene"
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def bbox(self):
        lo = self.pos.astype(np.float64).min(axis=0)
        hi = self.pos.astype(np.float64).max(axis=0)
        return lo, hi


@dataclass
class Sweep:
    """A monostatic sweep: incidence angles, ray screen, frequencies, bounces.

    The ray screen is square, centred on ``centre`` and ``2*extent`` wide, with
    ``W x H`` rays; ``extent`` must be at least the scene's bounding radius.
    """
    theta_deg: np.ndarray
    phi_deg: np.ndarray
    W: int
    H: int
    centre: np.ndarray
    extent: float
    freqs_hz: np.ndarray
    max_bounces: int = 1

    @property
    def n_angles(self) -> int:
        return int(len(self.theta_deg))

    @property
    def n_freq(self) -> int:
        return int(len(self.freqs_hz))


@dataclass
class GfbViews:
    """Views used to build and aggregate GFBs (Alg. 3 input)."""
    theta_deg: np.ndarray
    phi_deg: np.ndarray
    W: int
    H: int
    centre: np.ndarray
    extent: float


@dataclass
class Workload:
    scene: Scene
    sweep: Sweep
    views: Optional[GfbViews]
    name: str
    params: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# Input preparation: surfel radius and PCA normals (FP64 on the host)
# ----------------------------------------------------------------------------

def knn_radius(pos: np.ndarray, k: int = 8) -> np.ndarray:
    """Mean distance from each point to its k nearest neighbours (FP64 -> FP32)."""
    from scipy.spatial import cKDTree
    p = pos.astype(np.float64)
    tree = cKDTree(p)
    d, _ = tree.query(p, k=k + 1, workers=-1)
    return d[:, 1:].mean(axis=1).astype(np.float32)


def pca_normals(pos: np.ndarray, ref: np.ndarray, k: int = 16) -> np.ndarray:
    """Normals from the smallest principal axis of the k nearest neighbours,
    oriented to agree with the generator's side ``ref``."""
    from scipy.spatial import cKDTree
    p = pos.astype(np.float64)
    tree = cKDTree(p)
    _, idx = tree.query(p, k=k, workers=-1)
    out = np.empty_like(p)
    chunk = 200_000
    for s in range(0, p.shape[0], chunk):
        nb = p[idx[s:s + chunk]]                      # [c,k,3]
        nb = nb - nb.mean(axis=1, keepdims=True)
        cov = np.einsum("cki,ckj->cij", nb, nb)
        _, vec = np.linalg.eigh(cov)
        out[s:s + chunk] = vec[:, :, 0]
    flip = (out * ref.astype(np.float64)).sum(axis=1) < 0
    out[flip] *= -1.0
    out /= np.linalg.norm(out, axis=1, keepdims=True)
    return out.astype(np.float32)


def bounding_sphere(pos: np.ndarray):
    """Centre of the bounding box and the radius of the sphere around it (FP64)."""
    p = pos.astype(np.float64)
    c = 0.5 * (p.min(axis=0) + p.max(axis=0))
    r = float(np.sqrt(((p - c) ** 2).sum(axis=1).max()))
    return c, r


def freq_grid(f0: float, f1: float, n: int) -> np.ndarray:
    """f_i = f0 + i (f1 - f0)/(n-1), inclusive (n = 1 gives f0)."""
    if n == 1:
        return np.array([f0], dtype=np.float64)
    return f0 + np.arange(n, dtype=np.float64) * ((f1 - f0) / (n - 1))


# ----------------------------------------------------------------------------
# Primitive samplers
# ----------------------------------------------------------------------------

def _stratified_rect(rng, n_u, n_v, lu, lv):
    """One uniform point per cell of an n_u x n_v grid over [0,lu] x [0,lv]."""
    iu, iv = np.meshgrid(np.arange(n_u), np.arange(n_v), indexing="ij")
    su = (iu.ravel() + rng.random(iu.size)) * (lu / n_u)
    sv = (iv.ravel() + rng.random(iv.size)) * (lv / n_v)
    return su, sv


def _finish(pos, nrm, name, seed, noise=0.0, rng=None, pca_k=0, radius=True):
    pos = np.asarray(pos, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    nrm = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    if noise > 0.0:
        pos = pos + rng.normal(0.0, noise, size=pos.shape)
    pos32 = pos.astype(np.float32)
    if pca_k > 0:
        nrm32 = pca_normals(pos32, nrm, k=pca_k)
    else:
        nrm32 = nrm.astype(np.float32)
    rad = knn_radius(pos32, 8) if radius else None
    return Scene(pos=pos32, nrm=nrm32, rad=rad, name=name, seed=seed)


def plate(a: float = 1.0, b: float = 1.0, n_u: int = 100, n_v: int = 100, seed: int = 3,
          centre=(0.0, 0.0, 0.0), jitter: bool = True) -> Scene:
    """Flat a x b plate in the xy-plane (normal +z), stratified samples."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if jitter:
        su, sv = _stratified_rect(rng, n_u, n_v, a, b)
    else:
        iu, iv = np.meshgrid(np.arange(n_u), np.arange(n_v), indexing="ij")
        su = (iu.ravel() + 0.5) * (a / n_u)
        sv = (iv.ravel() + 0.5) * (b / n_v)
    pos = np.stack([su - a / 2, sv - b / 2, np.zeros_like(su)], axis=1) + np.asarray(centre)
    nrm = np.tile([0.0, 0.0, 1.0], (pos.shape[0], 1))
    return _finish(pos, nrm, "plate", seed)


def dihedral(n_points: int = 10_000, a: float = 0.5, seed: int = 1, jitter: bool = True) -> Scene:
    """Two a x a PEC plates at 90 deg: y=0 (x in [0,a]) and x=0 (y in [0,a]),
    z in [-a/2, a/2]; fold along z.  Each plate has n/2 points, one uniform
    point per cell of a 100 x 50 grid (for 10k points; scaled otherwise).
    Normals are the exact inward normals (+y and +x).  With jitter=False the
    points sit at the cell centres, so the target is mirror-symmetric about
    the plane x = y."""
    rng = np.random.Generator(np.random.PCG64(seed))
    per = n_points // 2
    n_u = int(round(math.sqrt(per * 2)))
    n_v = max(1, per // n_u)

    def cells():
        if jitter:
            return _stratified_rect(rng, n_u, n_v, a, a)
        iu, iv = np.meshgrid(np.arange(n_u), np.arange(n_v), indexing="ij")
        return (iu.ravel() + 0.5) * (a / n_u), (iv.ravel() + 0.5) * (a / n_v)

    su, sv = cells()
    p1 = np.stack([su, np.zeros_like(su), sv - a / 2], axis=1)
    n1 = np.tile([0.0, 1.0, 0.0], (p1.shape[0], 1))
    su, sv = cells()
    p2 = np.stack([np.zeros_like(su), su, sv - a / 2], axis=1)
    n2 = np.tile([1.0, 0.0, 0.0], (p2.shape[0], 1))
    return _finish(np.concatenate([p1, p2]), np.concatenate([n1, n2]), "dihedral", seed)


def octar(n_points: int = 50_000, size: float = 20.0, seed: int = 8) -> Scene:
    """The paper's OctAR target (Sec. IV-B, Fig. 11): eight trihedral corner
    reflectors formed by three mutually orthogonal square plates of side
    `size` crossing at the origin (the planes x=0, y=0, z=0).  n/3 points per
    plate, one uniform point per cell of a square grid; exact normals along
    each plate's axis (the plates are two-sided)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    per = n_points // 3
    n_u = max(1, int(round(math.sqrt(per))))
    n_v = max(1, per // n_u)
    ps, ns = [], []
    for axis in range(3):
        su, sv = _stratified_rect(rng, n_u, n_v, size, size)
        p = np.zeros((su.size, 3))
        p[:, (axis + 1) % 3] = su - size / 2
        p[:, (axis + 2) % 3] = sv - size / 2
        n = np.zeros_like(p)
        n[:, axis] = 1.0
        ps.append(p)
        ns.append(n)
    return _finish(np.concatenate(ps), np.concatenate(ns), "octar", seed)


def trihedral(n_points: int = 30_000, a: float = 0.6, seed: int = 4,
              origin=(0.0, 0.0, 0.0)) -> Scene:
    """Square trihedral corner: faces x=0, y=0, z=0, each [0,a]^2, opening
    toward +x+y+z.  Normals point into the opening."""
    rng = np.random.Generator(np.random.PCG64(seed))
    per = n_points // 3
    n_u = max(1, int(round(math.sqrt(per))))
    ps, ns = [], []
    for ax in range(3):
        su, sv = _stratified_rect(rng, n_u, n_u, a, a)
        p = np.zeros((su.size, 3))
        o1, o2 = [i for i in range(3) if i != ax]
        p[:, o1] = su
        p[:, o2] = sv
        n = np.zeros_like(p)
        n[:, ax] = 1.0
        ps.append(p + np.asarray(origin))
        ns.append(n)
    return _finish(np.concatenate(ps), np.concatenate(ns), "trihedral", seed)


def sphere(n_points: int = 200_000, a: float = 1.0, seed: int = 2) -> Scene:
    """Fibonacci (golden-angle spiral) lattice on a sphere of radius a with
    exact radial normals."""
    i = np.arange(n_points, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n_points
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = math.pi * (3.0 - math.sqrt(5.0))
    ph = i * ga
    nrm = np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)
    return _finish(a * nrm, nrm, "sphere", seed)


def _cylinder_samples(rng, n, r, h, centre):
    side = 2 * math.pi * r * h
    cap = math.pi * r * r
    tot = side + 2 * cap
    ns = int(round(n * side / tot))
    nc = (n - ns) // 2
    ph = rng.random(ns) * 2 * math.pi
    z = (rng.random(ns) - 0.5) * h
    ps = np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)
    nside = np.stack([np.cos(ph), np.sin(ph), np.zeros_like(ph)], axis=1)
    out_p, out_n = [ps], [nside]
    for sgn in (1.0, -1.0):
        rr = r * np.sqrt(rng.random(nc))
        pp = rng.random(nc) * 2 * math.pi
        pc = np.stack([rr * np.cos(pp), rr * np.sin(pp), np.full(nc, sgn * h / 2)], axis=1)
        out_p.append(pc)
        out_n.append(np.tile([0.0, 0.0, sgn], (nc, 1)))
    return np.concatenate(out_p) + np.asarray(centre), np.concatenate(out_n)


def cylinder(n_points: int = 20_000, r: float = 0.3, h: float = 1.0, seed: int = 6,
             centre=(0.0, 0.0, 0.0)) -> Scene:
    rng = np.random.Generator(np.random.PCG64(seed))
    p, n = _cylinder_samples(rng, n_points, r, h, centre)
    return _finish(p, n, "cylinder", seed)


def composite(n_points: int = 1_000_000, seed: int = 7, freq_hz: float = 10e9,
              pca: bool = True) -> Scene:
    """Trihedral corner (0.6 m faces, corner at the origin) + 1 m x 1 m plate
    centred at (-1.5, 0, 0) with normal +x + cylinder r=0.3 m, h=1 m at
    (0, -1.5, 0).  Points are distributed in proportion to area, with Gaussian
    position noise sigma = lambda/50 and (optionally) 16-NN PCA normals."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lam = C0 / freq_hz
    a_tri = 3 * 0.36
    a_pl = 1.0
    a_cy = 2 * math.pi * 0.3 * 1.0 + 2 * math.pi * 0.09
    tot = a_tri + a_pl + a_cy
    n_tri = int(n_points * a_tri / tot)
    n_pl = int(n_points * a_pl / tot)
    n_cy = n_points - n_tri - n_pl
    # trihedral faces: uniform samples
    ps, ns = [], []
    per = n_tri // 3
    for ax in range(3):
        uv = rng.random((per, 2)) * 0.6
        p = np.zeros((per, 3))
        o1, o2 = [i for i in range(3) if i != ax]
        p[:, o1], p[:, o2] = uv[:, 0], uv[:, 1]
        n = np.zeros_like(p)
        n[:, ax] = 1.0
        ps.append(p)
        ns.append(n)
    uv = rng.random((n_pl, 2)) - 0.5
    ps.append(np.stack([np.full(n_pl, -1.5), uv[:, 0], uv[:, 1]], axis=1))
    ns.append(np.tile([1.0, 0.0, 0.0], (n_pl, 1)))
    pc, nc = _cylinder_samples(rng, n_cy, 0.3, 1.0, (0.0, -1.5, 0.0))
    ps.append(pc)
    ns.append(nc)
    return _finish(np.concatenate(ps), np.concatenate(ns), "composite", seed,
                   noise=lam / 50.0, rng=rng, pca_k=16 if pca else 0)


def random_primitives(seed: int, lam: float, bbox_lambdas: float = 25.6,
                      n_min: int = 3, n_max: int = 12, density: Optional[float] = None,
                      sample_seed: Optional[int] = None, radius: bool = True) -> Scene:
    """3-12 random boxes / cylinders / spheres of 0.2-2 m (then rescaled so the
    scene's longest bbox edge is ``bbox_lambdas`` wavelengths), sampled at a
    uniform density of 5-50 points per lambda^2 (or ``density`` points per
    lambda^2).  The shapes depend on ``seed`` only, so the same target can be
    sampled sparsely and densely."""
    srng = np.random.Generator(np.random.PCG64(seed))
    k = int(srng.integers(n_min, n_max + 1))
    shapes = []
    for _ in range(k):
        kind = int(srng.integers(0, 3))
        size = srng.uniform(0.2, 2.0, size=3)
        ctr = srng.uniform(-2.0, 2.0, size=3)
        shapes.append((kind, size, ctr))
    dens = float(srng.uniform(5.0, 50.0)) if density is None else float(density)
    rng = np.random.Generator(np.random.PCG64(seed * 7919 + 1 if sample_seed is None else sample_seed))
    sp = np.array([c - s for _, s, c in shapes] + [c + s for _, s, c in shapes])
    ext = float((sp.max(axis=0) - sp.min(axis=0)).max())
    s = bbox_lambdas * lam / ext
    density = dens / (lam * lam)
    parts_p, parts_n = [], []
    for kind, size, ctr in shapes:
        size = size * s
        ctr = ctr * s
        if kind == 0:  # box
            a, b, c = size
            faces = [(0, a, b, c), (1, b, a, c), (2, c, a, b)]
            for ax, d, u, v in faces:
                for sgn in (-1.0, 1.0):
                    n = max(4, int(density * u * v))
                    uv = (rng.random((n, 2)) - 0.5) * np.array([u, v])
                    p = np.zeros((n, 3))
                    o1, o2 = [i for i in range(3) if i != ax]
                    p[:, o1], p[:, o2] = uv[:, 0], uv[:, 1]
                    p[:, ax] = sgn * d / 2
                    nn = np.zeros_like(p)
                    nn[:, ax] = sgn
                    parts_p.append(p + ctr)
                    parts_n.append(nn)
        elif kind == 1:  # cylinder along z
            r, h = size[0] / 2, size[2]
            area = 2 * math.pi * r * h + 2 * math.pi * r * r
            n = max(8, int(density * area))
            p, nn = _cylinder_samples(rng, n, r, h, ctr)
            parts_p.append(p)
            parts_n.append(nn)
        else:  # sphere
            r = size[0] / 2
            n = max(8, int(density * 4 * math.pi * r * r))
            v = rng.normal(size=(n, 3))
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            parts_p.append(ctr + r * v)
            parts_n.append(v)
    # radius=False: positions and normals only (rad None; a caller with a
    # GPU computes the radii there)
    return _finish(np.concatenate(parts_p), np.concatenate(parts_n), "primitives", seed,
                   radius=radius)


def c5_target(seed: int, n_points: int):
    """A serving request's target: positions and exact normals (no radii:
    the server computes them on the device), n_points on one of the shapes
    of the standard workloads at a random size: a dihedral or trihedral of
    0.3-1.5 m faces, a sphere of radius 0.3-1.5 m, the composite layout
    (trihedral, plate, cylinder; position noise 0.6 mm), or the OctAR plates
    of 2-20 m.  Returns (pos float32 [n,3], nrm float32 [n,3], kind)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = ("dihedral", "sphere", "trihedral", "composite", "octar")
    kind = kinds[int(rng.integers(0, len(kinds)))]
    n = int(n_points)

    def plates(axes, size, offset=0.0, centred=False):
        per = [n // len(axes)] * len(axes)
        per[0] += n - sum(per)
        ps, ns = [], []
        for ax, m in zip(axes, per):
            uv = rng.random((m, 2)) * size - (size / 2 if centred else 0.0)
            p = np.zeros((m, 3))
            o1, o2 = [i for i in range(3) if i != ax]
            p[:, o1], p[:, o2] = uv[:, 0], uv[:, 1]
            q = np.zeros_like(p)
            q[:, ax] = 1.0
            ps.append(p)
            ns.append(q)
        return np.concatenate(ps), np.concatenate(ns)

    if kind == "dihedral":
        pos, nrm = plates((1, 0), float(rng.uniform(0.3, 1.5)))
    elif kind == "trihedral":
        pos, nrm = plates((0, 1, 2), float(rng.uniform(0.3, 1.5)))
    elif kind == "octar":
        pos, nrm = plates((0, 1, 2), float(rng.uniform(2.0, 20.0)), centred=True)
    elif kind == "sphere":
        a = float(rng.uniform(0.3, 1.5))
        i = np.arange(n, dtype=np.float64)
        z = 1.0 - (2.0 * i + 1.0) / n
        r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        t = i * (math.pi * (3.0 - math.sqrt(5.0)))
        nrm = np.stack([r * np.cos(t), r * np.sin(t), z], axis=1)
        pos = a * nrm
    else:
        a_tri, a_pl, a_cy = 3 * 0.36, 1.0, 2 * math.pi * 0.3 + 2 * math.pi * 0.09
        tot = a_tri + a_pl + a_cy
        n_tri, n_pl = int(n * a_tri / tot), int(n * a_pl / tot)
        n_cy = n - n_tri - n_pl
        per = [n_tri // 3] * 3
        per[0] += n_tri - sum(per)
        ps, ns = [], []
        for ax, m in zip(range(3), per):
            uv = rng.random((m, 2)) * 0.6
            p = np.zeros((m, 3))
            o1, o2 = [i for i in range(3) if i != ax]
            p[:, o1], p[:, o2] = uv[:, 0], uv[:, 1]
            q = np.zeros_like(p)
            q[:, ax] = 1.0
            ps.append(p)
            ns.append(q)
        uv = rng.random((n_pl, 2)) - 0.5
        ps.append(np.stack([np.full(n_pl, -1.5), uv[:, 0], uv[:, 1]], axis=1))
        ns.append(np.tile([1.0, 0.0, 0.0], (n_pl, 1)))
        pc, nc = _cylinder_samples(rng, n_cy, 0.3, 1.0, (0.0, -1.5, 0.0))
        ps.append(pc)
        ns.append(nc)
        pos = np.concatenate(ps)
        pos = pos + rng.normal(0.0, 0.6e-3, size=pos.shape)
        nrm = np.concatenate(ns)
    return pos.astype(np.float32), nrm.astype(np.float32), kind


# ----------------------------------------------------------------------------
# Sweeps / views for the standard workloads
# ----------------------------------------------------------------------------

def aggregation_views(scene: Scene, W: int = 512, H: int = 512, margin: float = 1.02) -> GfbViews:
    """The 8 views of the paper's OctAR experiment: theta in {60,120} deg x
    phi in {45,135,225,315} deg, each covering the scene's bounding sphere."""
    c, r = bounding_sphere(scene.pos)
    th = np.array([60.0] * 4 + [120.0] * 4)
    ph = np.array([45.0, 135.0, 225.0, 315.0] * 2)
    return GfbViews(theta_deg=th, phi_deg=ph, W=W, H=H, centre=c, extent=r * margin)


def _sweep_over(scene, theta, phi, W, freqs, mb, margin=1.02):
    c, r = bounding_sphere(scene.pos)
    return Sweep(theta_deg=np.asarray(theta, dtype=np.float64),
                 phi_deg=np.asarray(phi, dtype=np.float64), W=W, H=W,
                 centre=c, extent=r * margin, freqs_hz=np.asarray(freqs, dtype=np.float64),
                 max_bounces=mb)


def workload_dihedral(n_points=10_000, W=128, view_W=512, n_angles=91) -> Workload:
    """PEC dihedral, 3 GHz, W x W ray screen, mb=2, monostatic phi 0..90 deg."""
    sc = dihedral(n_points)
    phi = np.linspace(0.0, 90.0, n_angles)
    sw = _sweep_over(sc, np.full(n_angles, 90.0), phi, W, [3e9], 2)
    return Workload(sc, sw, aggregation_views(sc, view_W, view_W), "dihedral")


def workload_sphere(n_points=200_000, W=1024, view_W=512, n_angles=360, n_freq=64) -> Workload:
    """PEC sphere a=1 m, 8-12 GHz (n_freq points), mb=2, phi 0..359 deg."""
    sc = sphere(n_points)
    phi = np.arange(n_angles, dtype=np.float64) * (360.0 / n_angles)
    sw = _sweep_over(sc, np.full(n_angles, 90.0), phi, W, freq_grid(8e9, 12e9, n_freq), 2)
    return Workload(sc, sw, aggregation_views(sc, view_W, view_W), "sphere")


def workload_composite(n_points=1_000_000, W=2048, view_W=512, n_angles=72, pca=True) -> Workload:
    """Composite scene, 10 GHz, mb=5, theta=60 deg, phi 0..355 step 5 deg."""
    sc = composite(n_points, pca=pca)
    phi = np.arange(n_angles, dtype=np.float64) * (360.0 / n_angles)
    sw = _sweep_over(sc, np.full(n_angles, 60.0), phi, W, [10e9], 5)
    return Workload(sc, sw, aggregation_views(sc, view_W, view_W), "composite")


def workload_octar(n_points=50_000, size=20.0, view_W=512, n_angles=360, freq_hz=500e6,
                   W=None) -> Workload:
    """OctAR at the paper's settings (Sec. IV-B): 50k points, longest bbox edge
    20 m, 500 MHz, monostatic theta = 60 deg over phi 0..359, three bounces,
    ray pitch lambda/10 (W x W rays over the bounding sphere)."""
    sc = octar(n_points, size)
    phi = np.arange(n_angles, dtype=np.float64) * (360.0 / n_angles)
    if W is None:
        _, r = bounding_sphere(sc.pos)
        pitch = C0 / freq_hz / 10.0
        W = int(math.ceil(2.0 * r * 1.02 / pitch / 8.0)) * 8
    sw = _sweep_over(sc, np.full(n_angles, 60.0), phi, W, [freq_hz], 3)
    return Workload(sc, sw, aggregation_views(sc, view_W, view_W), "octar")


def workload_small(seed: int = 11) -> Workload:
    """A small dihedral case the oracle finishes in seconds (parity tests)."""
    sc = dihedral(2_000, seed=seed)
    phi = np.array([0.0, 17.0, 45.0, 71.0])
    sw = _sweep_over(sc, np.full(4, 90.0), phi, 48, [3e9, 3.5e9, 4e9], 2)
    return Workload(sc, sw, aggregation_views(sc, 96, 96), "dihedral-small")


# ----------------------------------------------------------------------------
# Network parameters for the learned GFB completion (seeded random init)
# ----------------------------------------------------------------------------

UNET_HEADS = (("depth", 1), ("normal", 3), ("mask", 1))


def unet_param_shapes(widths=(32, 64, 128, 256), blocks=(2, 2, 2, 2)):
    """Names and shapes of the U-Net parameters (layout used by both sides):
    3x3 convs [Cout, 3, 3, Cin]; 1x1 convs [Cout, Cin]; depthwise 7x7 [7, 7, C];
    vectors [C].  ConvNeXt block p: dw 7x7 -> LayerNorm -> 1x1 C->4C -> GELU ->
    1x1 4C->C, residual."""
    shp = {}

    def block(p, c):
        shp[p + ".dw.w"] = (7, 7, c)
        shp[p + ".dw.b"] = (c,)
        shp[p + ".ln.g"] = (c,)
        shp[p + ".ln.b"] = (c,)
        shp[p + ".pw1.w"] = (4 * c, c)
        shp[p + ".pw1.b"] = (4 * c,)
        shp[p + ".pw2.w"] = (c, 4 * c)
        shp[p + ".pw2.b"] = (c,)

    c = widths
    shp["stem.w"] = (c[0], 3, 3, 1)
    shp["stem.b"] = (c[0],)
    for lvl in range(len(c)):
        if lvl > 0:
            shp[f"down{lvl}.w"] = (c[lvl], c[lvl - 1])
            shp[f"down{lvl}.b"] = (c[lvl],)
        for k in range(blocks[lvl]):
            block(f"enc{lvl}.{k}", c[lvl])
    for head, nout in UNET_HEADS:
        for lvl in range(len(c) - 2, -1, -1):
            p = f"{head}.up{lvl}"
            shp[p + ".w"] = (4 * c[lvl], 3, 3, c[lvl + 1])
            shp[p + ".b"] = (4 * c[lvl],)
            shp[f"{head}.fuse{lvl}.w"] = (c[lvl], 2 * c[lvl])
            shp[f"{head}.fuse{lvl}.b"] = (c[lvl],)
            block(f"{head}.blk{lvl}", c[lvl])
        shp[f"{head}.head.w"] = (nout, c[0])
        shp[f"{head}.head.b"] = (nout,)
    return shp


def unet_init(seed: int = 0, widths=(32, 64, 128, 256), blocks=(2, 2, 2, 2)):
    """Seeded float32 initial parameters: weights ~ N(0, 1/fan_in) (scaled
    down on the residual branch's last 1x1), biases 0, LayerNorm gain 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, shp in unet_param_shapes(widths, blocks).items():
        if name.endswith(".b"):
            a = np.zeros(shp)
        elif name.endswith(".ln.g"):
            a = np.ones(shp)
        else:
            if name.endswith(".dw.w"):
                fan_in = 49
            elif len(shp) == 4:
                fan_in = shp[1] * shp[2] * shp[3]
            else:
                fan_in = shp[-1]
            a = rng.normal(0.0, 1.0 / math.sqrt(fan_in), size=shp)
            if name.endswith(".pw2.w"):
                a *= 0.1
        out[name] = a.astype(np.float32)
    return out
