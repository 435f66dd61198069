"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, never against the oracle's own formulas retyped.

Pins used: hand-worked intersection cases (counts and depths read off the
geometry), Eq. 22 values at chosen angles, the edge rule on a hand-drawn mask,
the Eq. 23 selection/blend on a two-splat case worked by hand, the epsilon
rule, the mirror paths of a dihedral and a trihedral, the textbook PO
plate pattern (4 pi A^2/lambda^2) cos^2(theta) sinc^2(k a sin(theta)), the
parallelogram PO integral, the exact PO backscatter of a sphere, the phase
convention under translation, f^2 scaling, and the realised-aperture forms of
the dihedral and trihedral RCS.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenes

C0 = scenes.C0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def down_view(W, H, pitch, z=5.0):
    """Screen at height z looking down -z; u = x, v = y."""
    return oracle.View(o=np.array([0.0, 0.0, z]), u=np.array([1.0, 0.0, 0.0]),
                       v=np.array([0.0, 1.0, 0.0]), d=np.array([0.0, 0.0, -1.0]),
                       pitch=pitch, W=W, H=H)


def mk_scene(pos, nrm, rad):
    return scenes.Scene(pos=np.asarray(pos, np.float32), nrm=np.asarray(nrm, np.float32),
                        rad=np.asarray(rad, np.float32))


# ----------------------------------------------------------------------------
# a1: view frame
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_view_frame_is_the_spherical_basis(mode):
    # w = r_hat(theta, phi) toward the transmitter, u = theta_hat, v = phi_hat
    # (u x v = w), rays along d = -w; pitch 2 extent / W; the screen centre
    # one extent plus one pitch from the target's centre along w
    tol = 1e-7 if mode == "fp32" else 1e-15
    for th, ph, w, u, v in ((90.0, 0.0, [1, 0, 0], [0, 0, -1], [0, 1, 0]),
                            (0.0, 0.0, [0, 0, 1], [1, 0, 0], [0, 1, 0]),
                            (90.0, 90.0, [0, 1, 0], [0, 0, -1], [-1, 0, 0])):
        V = oracle.view_from_angles(th, ph, [0.5, -1.0, 2.0], 1.5, 60, 40, mode)
        assert np.allclose(-V.d, w, atol=tol) and np.allclose(V.u, u, atol=tol)
        assert np.allclose(V.v, v, atol=tol)
        assert abs(V.pitch - 2 * 1.5 / 60) < tol
        assert np.allclose(V.o, np.array([0.5, -1.0, 2.0]) + (1.5 + V.pitch) * np.asarray(w, float),
                           atol=1e-6)
    rng = np.random.default_rng(4)
    for th, ph in zip(rng.uniform(0, 180, 20), rng.uniform(0, 360, 20)):
        V = oracle.view_from_angles(th, ph, [0, 0, 0], 1.0, 8, 8, mode)
        assert np.allclose(np.cross(V.u, V.v), -V.d, atol=4 * tol)


# ----------------------------------------------------------------------------
# a2/a3: GFB (Alg. 1)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_gfb_single_disk_handmade(mode):
    # unit disk at the origin; 8x8 pixels of pitch 0.5 => centres at
    # +-0.25, +-0.75, ...; exactly 12 centres lie within radius 1.
    sc = mk_scene([[0, 0, 0]], [[0, 0, -1]], [1.0])
    g = oracle.gfb(sc, down_view(8, 8, 0.5), mode)
    hit = g.idx >= 0
    assert hit.sum() == 12
    # which 12: centres (i + 0.5 - 4) * 0.5 = +-0.25, +-0.75 on both axes,
    # i, j in 2..5, except the four corners (0.75^2 + 0.75^2 > 1)
    expect = {(i, j) for i in range(2, 6) for j in range(2, 6)} - {(2, 2), (2, 5), (5, 2), (5, 5)}
    assert {(int(p % 8), int(p // 8)) for p in np.flatnonzero(hit)} == expect
    assert np.all(g.depth[hit] == 5.0)
    assert np.all(np.isinf(g.depth[~hit]))
    # the stored normal is turned to face the view (n . d < 0)
    assert np.all(g.nrm[hit] == np.array([0.0, 0.0, 1.0]))


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_gfb_nearest_and_tie_break(mode):
    # A at z=0 (idx 0), B and its duplicate C at z=1 (idx 1, 2): B wins
    # (nearest; equal depth -> smaller index), depth 4.
    sc = mk_scene([[0, 0, 0], [0, 0, 1], [0, 0, 1]], [[0, 0, 1]] * 3, [10.0] * 3)
    g = oracle.gfb(sc, down_view(4, 4, 0.5), mode)
    assert np.all(g.idx == 1)
    assert np.all(g.depth == 4.0)
    k = g.keys()
    assert np.all(k == ((np.uint64(np.float32(4.0).view(np.uint32)) << np.uint64(32)) | np.uint64(1)))


@pytest.mark.parametrize("mode,tol", [("fp32", 3e-6), ("fp64", 2e-7)])
def test_gfb_tilted_plate_depth_is_ray_plane(mode, tol):
    # every surfel lies in the plane z = 0.3 x + 0.1 y with the plane's
    # normal, so any hit's depth is the ray-plane distance (up to the FP32
    # rounding of the stored positions).
    rng = np.random.default_rng(5)
    xy = rng.uniform(-0.5, 0.5, size=(3000, 2))
    z = 0.3 * xy[:, 0] + 0.1 * xy[:, 1]
    n = np.array([-0.3, -0.1, 1.0]) / math.sqrt(1.1)
    sc = mk_scene(np.c_[xy, z], np.tile(n, (3000, 1)), np.full(3000, 0.03))
    v = oracle.view_from_angles(30.0, 20.0, [0, 0, 0], 0.8, 40, 40, mode)
    g = oracle.gfb(sc, v, mode)
    hit = g.idx >= 0
    assert hit.sum() > 300
    j, i = np.divmod(np.arange(40 * 40), 40)
    a = ((i + 0.5) - 20) * v.pitch
    b = ((j + 0.5) - 20) * v.pitch
    o = v.o[None] + a[:, None] * v.u[None] + b[:, None] * v.v[None]
    # ray-plane: n.(o + t d) = 0
    t = -(o @ n) / (v.d @ n)
    assert np.max(np.abs(g.depth[hit] - t[hit]) / t[hit]) < tol


def test_gfb_sphere_normals_are_radial():
    sc = scenes.sphere(5000, 1.0)
    v = oracle.view_from_angles(70.0, 10.0, [0, 0, 0], 1.05, 48, 48, "fp64")
    g = oracle.gfb(sc, v, "fp64")
    hit = g.idx >= 0
    j, i = np.divmod(np.arange(48 * 48), 48)
    a = ((i + 0.5) - 24) * v.pitch
    b = ((j + 0.5) - 24) * v.pitch
    o = v.o[None] + a[:, None] * v.u[None] + b[:, None] * v.v[None]
    x = o[hit] + g.depth[hit][:, None] * v.d[None]
    radial = x / np.linalg.norm(x, axis=1, keepdims=True)
    ang = np.arccos(np.clip((radial * g.nrm[hit]).sum(1), -1, 1))
    # the hit lies on a tangent disk within R of its centre: angle <~ R/a
    assert np.max(ang) < 1.2 * float(sc.rad.max())
    # and the normal faces the view
    assert np.all(g.nrm[hit] @ v.d < 0)


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_gfb_tube_mode_handmade(mode):
    # 4x4 pixels, pitch 0.5; P0 on the axis of pixel (0.25, 0.25) at depth 5,
    # P1 0.05 off that axis but 1 m closer: both inside delta = 0.1, P1 is
    # nearer the tube origin => depth = |P1 - o| = sqrt(0.05^2 + 4^2).  P2 on
    # the same axis 1 m behind the screen (z = 6) is no candidate.
    sc = mk_scene([[0.25, 0.25, 0.0], [0.25, 0.30, 1.0], [0.25, 0.25, 6.0]], [[0, 0, 1]] * 3,
                  [0.0, 0.0, 0.0])
    g = oracle.gfb(sc, down_view(4, 4, 0.5), mode, tube=True, delta=0.1)
    hit = np.flatnonzero(g.idx >= 0)
    assert list(hit) == [2 * 4 + 2]
    assert g.idx[hit[0]] == 1
    assert abs(g.depth[hit[0]] - math.sqrt(0.05 ** 2 + 16.0)) < 1e-6


def test_gfb_fp32_and_fp64_agree():
    sc = scenes.sphere(4000, 1.0)
    v32 = oracle.view_from_angles(50.0, 30.0, [0, 0, 0], 1.05, 64, 64, "fp32")
    g32 = oracle.gfb(sc, v32, "fp32")
    g64 = oracle.gfb(sc, v32, "fp64")
    same = g32.idx == g64.idx
    assert same.mean() > 0.995
    both = same & (g32.idx >= 0)
    # FP32 cancellation in (c - o) . n / (d . n) grows as d . n -> 0
    assert np.max(np.abs(g32.depth[both] - g64.depth[both]) / g64.depth[both]) < 2e-5


# ----------------------------------------------------------------------------
# a4: edge filter, fusion, Eq. 22
# ----------------------------------------------------------------------------

def _handmade_gfb(view, depth, nrm, mask):
    W, H = view.W, view.H
    return oracle.Gfb(depth=np.asarray(depth, np.float64).ravel(),
                      idx=np.where(np.asarray(mask).ravel() > 0, 0, -1).astype(np.int64),
                      nrm=np.asarray(nrm, np.float64).reshape(W * H, 3), view=view, pix=None)


def _exact_fuse(bmin_z=-0.0625):
    # voxel = 0.125 m, grid origin at -0.3125 so pixel centres (multiples of
    # 0.125) fall in the middle of distinct voxels.
    return oracle.FuseParams(tau=3.0, bmin=np.array([-0.3125, -0.3125, bmin_z]),
                             inv_vox=8.0, G=256)


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_eq22_radius_values(mode):
    L = 0.125
    v = down_view(5, 5, L)
    cases = {0.0: math.sqrt(2) * L,                      # s = 1
             60.0: 2.0 * L,                              # s = sqrt(2)
             85.0: 3.535 * L,                            # s = 3.39 >= 2.5
             math.degrees(math.acos(0.165)): math.sqrt(2) * L * math.sqrt(1 / 0.165)}
    for alpha, R_expect in cases.items():
        n = np.array([math.sin(math.radians(alpha)), 0.0, math.cos(math.radians(alpha))])
        n = n.astype(np.float32).astype(np.float64)
        g = _handmade_gfb(v, np.full(25, 5.0), np.tile(n, (25, 1)), np.ones(25))
        s = oracle.aggregate([g], _exact_fuse(), mode)
        # only the 3x3 interior survives the edge rule; one splat per pixel
        assert list(s.id) == [6, 7, 8, 11, 12, 13, 16, 17, 18]
        assert np.all(s.count == 1)
        assert np.allclose(s.r, R_expect, rtol=2e-7), (alpha, s.r[0], R_expect)
        # centres are the pixels' surface points (z = 0)
        assert np.all(s.c[:, 2] == 0.0)
        assert np.allclose(s.c[:, 0], np.tile([-0.125, 0.0, 0.125], 3))


def test_eq22_continuity_at_2_5():
    # sqrt(2) * 2.5 = 3.5355...; the paper caps with 3.535 L (Eq. 22)
    L = 0.125
    v = down_view(5, 5, L)
    for cosv, R_expect in ((1 / 2.5 ** 2 * 1.0001, math.sqrt(2) * L * math.sqrt(1 / (1 / 2.5 ** 2 * 1.0001))),
                           (1 / 2.5 ** 2 * 0.9999, 3.535 * L)):
        n = np.array([math.sqrt(1 - cosv ** 2), 0.0, cosv]).astype(np.float32).astype(np.float64)
        g = _handmade_gfb(v, np.full(25, 5.0), np.tile(n, (25, 1)), np.ones(25))
        s = oracle.aggregate([g], _exact_fuse(), "fp64")
        assert abs(s.r[0] - R_expect) < 2e-4 * L


def test_edge_filter_handmade():
    # 6x6, a hole at (i=2, j=2), depth 5 for i<=3 and 6 for i>=4
    # (jump 1 > 3 L = 0.375).  Border pixels, the hole's 4-neighbours and both
    # sides of the jump are edges; the survivors were worked out by hand.
    L = 0.125
    v = down_view(6, 6, L)
    mask = np.ones((6, 6))
    mask[2, 2] = 0
    depth = np.where(np.arange(6)[None, :] >= 4, 6.0, 5.0) * np.ones((6, 1))
    g = _handmade_gfb(v, depth, np.tile([0, 0, 1.0], (36, 1)), mask)
    s = oracle.aggregate([g], _exact_fuse(-2.0), "fp64")
    assert sorted(np.flatnonzero(s.keep)) == [7, 19, 25, 26]


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_fusion_average_over_views(mode):
    # two views with the same frame; view 1 sees the surface 1/32 m lower and
    # with flipped normals.  Every voxel gets one contributor per view: count 2,
    # centre z = the mean (-1/64), normal = the owner's (flips undone), owner =
    # the view-0 pixel.
    L = 0.125
    v0 = down_view(5, 5, L)
    v1 = down_view(5, 5, L)
    n = np.array([0.0, 0.6, 0.8])
    g0 = _handmade_gfb(v0, np.full(25, 5.0), np.tile(n, (25, 1)), np.ones(25))
    g1 = _handmade_gfb(v1, np.full(25, 5.03125), np.tile(-n, (25, 1)), np.ones(25))
    s = oracle.aggregate([g0, g1], _exact_fuse(), mode)
    assert list(s.id) == [6, 7, 8, 11, 12, 13, 16, 17, 18]
    assert np.all(s.count == 2)
    assert np.all(s.c[:, 2] == -0.015625)
    assert np.allclose(s.n, n[None], atol=1e-7)


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_fusion_owner_is_the_most_frontal_view(mode):
    # view 0 looks down -z; view 1 looks along (0.6, 0, -0.8) from a screen
    # placed so its pixels land on the same surface points (x_i, y_j, 0).
    # With both normals (-0.6, 0, 0.8): |n.d0| = 0.8 < |n.d1| = 1, so view 1
    # owns every splat (ids 25 + pixel); with (0.6, 0, 0.8): 0.8 > 0.28 and
    # view 0 owns them.
    L = 0.125
    v0 = down_view(5, 5, L)
    v1 = oracle.View(o=np.array([-3.0, 0.0, 4.0]), u=np.array([1.0, 0.0, 0.0]),
                     v=np.array([0.0, 1.0, 0.0]), d=np.array([0.6, 0.0, -0.8]), pitch=L, W=5, H=5)
    # The radius is the larger Eq. 22 value of the two contributors,
    # sqrt(2) L / sqrt(|n.d|) here (|n| = |d| = 1, s < 2.5): 1/sqrt(0.8) from
    # view 0 in the first case, 1/sqrt(0.28) from view 1 in the second.  A
    # third normal, (-1, 0, 3)/sqrt(10), bisects the two view directions:
    # |n.d0| = |n.d1| = 3/sqrt(10), a tie that goes to the lower view.
    inner = [6, 7, 8, 11, 12, 13, 16, 17, 18]
    t = 1.0 / math.sqrt(10.0)
    cases = (([-0.6, 0.0, 0.8], 25, 1.0 / math.sqrt(0.8)),
             ([0.6, 0.0, 0.8], 0, 1.0 / math.sqrt(0.28)),
             ([-t, 0.0, 3.0 * t], 0, 1.0 / math.sqrt(3.0 * t)))
    for n, owner_off, s_max in cases:
        n = np.array(n)
        g0 = _handmade_gfb(v0, np.full(25, 5.0), np.tile(n, (25, 1)), np.ones(25))
        g1 = _handmade_gfb(v1, np.full(25, 5.0), np.tile(n, (25, 1)), np.ones(25))
        s = oracle.aggregate([g0, g1], _exact_fuse(), mode)
        assert list(s.id) == [owner_off + i for i in inner]
        assert np.all(s.count == 2)
        assert np.allclose(s.n, n[None], atol=1e-7)
        assert np.allclose(s.r, math.sqrt(2.0) * L * s_max, rtol=1e-6)


# ----------------------------------------------------------------------------
# a5: Eq. 23 overlap selection / blend, epsilon, mirror paths
# ----------------------------------------------------------------------------

def _splats(rows):
    ids, c, n, r = zip(*rows)
    order = np.argsort(ids)
    a = lambda x: np.asarray(x, np.float64)[order]
    return oracle.Splats(id=np.asarray(ids, np.int64)[order], c=a(c), n=a(n), r=a(r),
                         count=np.ones(len(ids), np.int32), keep=np.zeros(0, np.uint8))


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_eq23_overlap_select_and_blend(mode):
    # Ray straight down the z axis.  Splat A (id 10): centre (0.5,0,0), normal
    # +z, R 1 -> hit at z=0 (t=5), rho = 0.5.  Splat B (id 20): normal
    # (0.6,0,0.8), centre (0.9,0,-0.625), R 1.5 -> its plane meets the axis at
    # z=0.05 (t=4.95), |e| = 1.125, rho = 0.75.  Splat C (id 30) far below.
    rows = [(20, [0.9, 0, -0.625], [0.6, 0, 0.8], 1.5),
            (10, [0.5, 0, 0], [0, 0, 1], 1.0),
            (30, [0, 0, -3.0], [0, 0, 1], 1.0)]
    S = _splats(rows)
    v = down_view(1, 1, 1.0)
    # r = 0.1: A is within r of the nearest hit (B) and is closer to its centre
    tr = oracle.trace(v, S, 1, 1e-3, 0.1, mode=mode)
    assert tr.M[0] == 1 and tr.ids[0, 0] == 10
    assert np.allclose(tr.p[0], [0, 0, 0], atol=1e-6)
    m = 0.5 * np.array([0, 0, 1.0]) + 0.25 * np.array([0.6, 0, 0.8])
    assert np.allclose(tr.n[0], m / np.linalg.norm(m), atol=2e-7)
    # r = 0.01: only the nearest (B) is a candidate
    tr = oracle.trace(v, S, 1, 1e-3, 0.01, mode=mode)
    assert tr.ids[0, 0] == 20
    assert np.allclose(tr.p[0], [0, 0, 0.05], atol=1e-6)
    assert np.allclose(tr.n[0], [0.6, 0, 0.8], atol=2e-7)


def test_eq23_tie_break_smaller_id():
    rows = [(7, [0.2, 0, 0], [0, 0, 1], 1.0), (5, [0.2, 0, 0], [0, 0, 1], 1.0)]
    tr = oracle.trace(down_view(1, 1, 1.0), _splats(rows), 1, 1e-3, 0.1)
    assert tr.ids[0, 0] == 5


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_epsilon_minimum_travel(mode):
    # Bounce 1 from a GFB on the plane z=0; the reflected ray goes straight up.
    # A splat at z=0 (the surface itself) is never re-hit; a splat at height h
    # is hit iff h > eps (Fig. 4b).
    v = down_view(1, 1, 1.0)
    first = oracle.Gfb(depth=np.array([5.0]), idx=np.array([0]), nrm=np.array([[0, 0, 1.0]]),
                       view=v, pix=None)
    eps = 0.01
    for h, M_expect in ((2 * eps, 2), (0.5 * eps, 1)):
        S = _splats([(1, [0, 0, 0], [0, 0, 1], 1.0), (2, [0, 0, h], [0, 0, 1], 1.0)])
        tr = oracle.trace(v, S, 2, eps, 1e-4, first=first, mode=mode)
        assert tr.M[0] == M_expect
        if M_expect == 2:
            assert tr.ids[0, 1] == 2
            assert abs(tr.path[0] - (-0.0 + h)) < 1e-7


@pytest.fixture(scope="module")
def dihedral_geom():
    sc = scenes.dihedral(6000, seed=21)
    vd = scenes.aggregation_views(sc, 128, 128)
    S, gv, gf, fp = oracle.build_geometry(sc, vd, "fp32")
    return sc, S, gv


def test_dihedral_interior_rays_bounce_twice(dihedral_geom):
    # At phi = 45 deg broadside, a ray hitting plate y=0 at (x1, 0, z) is
    # mirrored to (0, x1, z) on plate x=0 and leaves: exactly 2 bounces.
    sc, S, gv = dihedral_geom
    eps = oracle.default_eps(gv)
    sw = scenes._sweep_over(sc, [90.0], [45.0], 64, [3e9], 3)
    v = oracle.sweep_views(sw)[0]
    first = oracle.gfb(sc, v)
    tr = oracle.trace(v, S, 3, eps, eps, first=first)
    hit = first.idx >= 0
    j, i = np.divmod(np.arange(64 * 64), 64)
    o = v.o[None] + (((i + 0.5) - 32) * v.pitch)[:, None] * v.u[None] + \
        (((j + 0.5) - 32) * v.pitch)[:, None] * v.v[None]
    p1 = o + np.where(hit, first.depth, 0)[:, None] * v.d[None]
    m = 4 * float(S.r.max())
    inner = hit & (np.abs(p1[:, 2]) < 0.25 - m) & (np.abs(p1[:, 0] - p1[:, 1]) > m) & \
        (np.maximum(p1[:, 0], p1[:, 1]) < 0.5 - m)
    assert inner.sum() > 500
    assert np.all(tr.M[inner] == 2)
    assert np.all(tr.psi[inner] == 1)
    mirror = np.stack([p1[:, 1], p1[:, 0], p1[:, 2]], 1)
    assert np.max(np.abs(tr.p[inner] - mirror[inner])) < 1e-5


def test_trihedral_axis_triple_bounce_aperture():
    # Along the trihedral's symmetry axis every ray in the triple-bounce
    # aperture (area sqrt(3) a^2) returns after exactly 3 reflections, and
    # sigma = 4 pi A_eff^2 / lambda^2 with A_eff the realised aperture
    # (12 pi a^4 / lambda^2 for the ideal corner).
    a = 0.3
    sc = scenes.trihedral(9000, a=a, seed=8)
    vd = scenes.aggregation_views(sc, 128, 128)
    S, gv, gf, fp = oracle.build_geometry(sc, vd, "fp32")
    eps = oracle.default_eps(gv)
    th = math.degrees(math.acos(1 / math.sqrt(3)))
    sw = scenes._sweep_over(sc, [th], [45.0], 96, [10e9], 3)
    res = oracle.rcs_sweep(sc, sw, S, eps, eps)
    tr, v = res.traces[0], res.views[0]
    n3 = int(((tr.M == 3) & (tr.psi == 1)).sum())
    a_eff = n3 * v.pitch ** 2
    assert abs(a_eff / (math.sqrt(3) * a * a) - 1) < 0.12
    lam = C0 / 10e9
    sig = res.sigma[0, 0, 0, 0]
    assert abs(oracle.db(sig) - oracle.db(4 * math.pi * a_eff ** 2 / lam ** 2)) < 0.5
    assert abs(oracle.db(sig) - oracle.db(12 * math.pi * a ** 4 / lam ** 2)) < 1.5


# ----------------------------------------------------------------------------
# a6/a7: PO field (Eq. 5-14)
# ----------------------------------------------------------------------------

def _plate_cells(theta_deg, a, b, nu, nv, shift=(0.0, 0.0, 0.0), skew=0.0):
    """Synthetic last-hit records of an a x b plate in the plane z=0 tiled by
    the projections of nu x nv screen cells (incidence in the xz-plane)."""
    th = math.radians(theta_deg)
    w = np.array([math.sin(th), 0, math.cos(th)])
    u = np.array([math.cos(th), 0, -math.sin(th)])
    v = np.array([0, 1.0, 0])
    d = -w
    Lu = a / nu * math.cos(th)
    us = Lu * u
    vs = (b / nv) * v + skew * us      # a skewed cell (non-orthogonal u', v')
    # projected cell vectors on the plate (Eq. 12-13 with n = z)
    up = us - d * (us[2] / d[2])
    vp = vs - d * (vs[2] / d[2])
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    ps = (ii.ravel()[:, None] - (nu - 1) / 2) * up[None] + (jj.ravel()[:, None] - (nv - 1) / 2) * vp[None]
    ps = ps + np.asarray(shift)[None]
    nr = ps.shape[0]
    tr = oracle.Trace(M=np.ones(nr, np.int32), ids=np.zeros((nr, 1), np.int64), p=ps,
                      n=np.tile([0, 0, 1.0], (nr, 1)), k=np.tile(d, (nr, 1)),
                      u=np.tile(us, (nr, 1)), v=np.tile(vs, (nr, 1)), path=ps @ d,
                      psi=np.ones(nr, np.uint8))
    return tr, w, u, v, up * nu, vp * nv


@pytest.mark.parametrize("theta", [0.0, 10.0, 25.0, 40.0, 60.0])
def test_po_plate_pattern_textbook(theta):
    f = 3e9
    lam = C0 / f
    k = 2 * math.pi / lam
    a, b = 0.5, 0.3
    tr, w, u, v, _, _ = _plate_cells(theta, a, b, 40, 30)
    E = oracle.po_field(tr, [f], w)[0]
    s = oracle.sigma_from_field(E, [f], u, v)[0]
    x = k * a * math.sin(math.radians(theta))
    ref = 4 * math.pi * (a * b) ** 2 / lam ** 2 * math.cos(math.radians(theta)) ** 2 * \
        (math.sin(x) / x if x else 1.0) ** 2
    assert abs(s[0, 0] / ref - 1) < 1e-9
    assert abs(s[1, 1] / ref - 1) < 1e-9
    # single-bounce PO has no cross-polarised backscatter
    assert s[0, 1] < 1e-20 * ref and s[1, 0] < 1e-20 * ref


def test_po_parallelogram_cells_use_cross_product_area():
    # With skewed (non-orthogonal) cells the exact integral over the tiled
    # parallelogram is |U x V| sinc(q.U/2) sinc(q.V/2); the sum of per-cell
    # Eq. 11 terms equals it only with the area |u' x v'|.
    f = 5e9
    lam = C0 / f
    k = 2 * math.pi / lam
    tr, w, u, v, U, V = _plate_cells(35.0, 0.4, 0.25, 32, 20, skew=0.7)
    E = oracle.po_field(tr, [f], w)[0]
    q = k * (-w - w)
    sinc = lambda x: math.sin(x) / x if x else 1.0
    I = np.linalg.norm(np.cross(U, V)) * sinc(q @ U / 2) * sinc(q @ V / 2)
    # vector factor for pol H (h = u_hat) with n = z
    n = np.array([0, 0, 1.0])
    vec = np.cross(np.cross(np.cross(n, u), w), w)
    assert np.allclose(E[0, 1].real, I * vec, rtol=1e-9, atol=1e-12 * abs(I))
    assert np.allclose(E[0, 1].imag, 0.0, atol=1e-9 * abs(I))


def test_po_translation_phase_convention():
    # exp(+j w t) convention with exp(-j k.r) propagation: moving the target by
    # t multiplies the field by exp(-j q.t), q = k (k_in - k_s).
    f = 3e9
    k = 2 * math.pi * f / C0
    t = np.array([0.013, -0.02, 0.031])
    tr0, w, u, v, _, _ = _plate_cells(20.0, 0.3, 0.3, 16, 16)
    tr1, *_ = _plate_cells(20.0, 0.3, 0.3, 16, 16, shift=t)
    E0 = oracle.po_field(tr0, [f], w)[0]
    E1 = oracle.po_field(tr1, [f], w)[0]
    q = k * (-w - w)
    assert np.allclose(E1, E0 * np.exp(-1j * (q @ t)), rtol=1e-9, atol=1e-12)


def test_po_broadside_f_squared_and_polarisation_free():
    tr, w, u, v, _, _ = _plate_cells(0.0, 0.4, 0.4, 20, 20)
    fs = [2e9, 4e9]
    E = oracle.po_field(tr, fs, w)[0]
    s = oracle.sigma_from_field(E, fs, u, v)
    assert abs(s[1, 0, 0] / s[0, 0, 0] - 4.0) < 1e-12
    # a flat plate at normal incidence has no preferred polarisation: the
    # backscattered field is the same multiple c of the incident e for e = V
    # (theta_hat = u) and e = H (phi_hat = v).
    cV = E[0, 0] @ u
    cH = E[0, 1] @ v
    assert abs(cV - cH) < 1e-12 * abs(cV)
    assert np.allclose(E[0, 0], cV * u, atol=1e-12 * abs(cV))
    assert np.allclose(E[0, 1], cH * v, atol=1e-12 * abs(cH))


def test_po_sphere_exact_backscatter():
    # exact PO backscatter of a sphere: sigma = 4 pi k^2 a^4 |e^{jb}/(jb) +
    # (e^{jb} - 1)/b^2|^2 with b = 2ka (-> pi a^2).  Synthetic hits on the exact
    # sphere; the discrete cell sum misses part of the shadow-boundary term,
    # which is O(1/b) of the field.
    f = 3e9
    k = 2 * math.pi * f / C0
    a, W = 1.0, 300
    ext = a * 1.02
    L = 2 * ext / W
    c = (np.arange(W) + 0.5 - W / 2) * L
    X, Y = np.meshgrid(c, c)
    X, Y = X.ravel(), Y.ravel()
    hit = X * X + Y * Y < a * a
    Z = np.sqrt(np.maximum(a * a - X * X - Y * Y, 0))
    p = np.stack([X, Y, Z], 1)[hit]
    nr = p.shape[0]
    d = np.array([0, 0, -1.0])
    tr = oracle.Trace(M=np.ones(nr, np.int32), ids=np.zeros((nr, 1), np.int64), p=p, n=p / a,
                      k=np.tile(d, (nr, 1)), u=np.tile([L, 0, 0], (nr, 1)),
                      v=np.tile([0, L, 0], (nr, 1)), path=p @ d, psi=np.ones(nr, np.uint8))
    E = oracle.po_field(tr, [f], [0, 0, 1.0])[0]
    s = oracle.sigma_from_field(E, [f], [1, 0, 0], [0, 1, 0])[0]
    b = 2 * k * a
    ref = 4 * math.pi * k ** 2 * a ** 4 * abs(np.exp(1j * b) / (1j * b) + (np.exp(1j * b) - 1) / b ** 2) ** 2
    bound_db = 20 * math.log10(1 + 2.0 / b)
    for pol in (0, 1):
        assert abs(oracle.db(s[pol, pol]) - oracle.db(ref)) < bound_db


# ----------------------------------------------------------------------------
# a7: end-to-end RCS through the oracle
# ----------------------------------------------------------------------------

def test_rcs_dihedral_realised_aperture(dihedral_geom):
    # broadside to one face (phi = 0): single bounce, sigma = 4 pi (N L^2)^2 /
    # lambda^2; at phi = 45: every hit is a double bounce, same form with the
    # double-bounce aperture, which tends to sqrt(2) a b (8 pi a^2 b^2/lambda^2).
    sc, S, gv = dihedral_geom
    eps = oracle.default_eps(gv)
    f = 3e9
    lam = C0 / f
    sw = scenes._sweep_over(sc, [90.0, 90.0], [0.0, 45.0], 96, [f], 2)
    res = oracle.rcs_sweep(sc, sw, S, eps, eps)
    L = res.views[0].pitch
    n1 = int((res.traces[0].M == 1).sum())
    assert res.traces[0].M.max() == 1
    s0 = res.sigma[0, 0]
    assert abs(oracle.db(s0[0, 0]) - oracle.db(4 * math.pi * (n1 * L * L) ** 2 / lam ** 2)) < 1e-3
    assert abs(oracle.db(s0[1, 1]) - oracle.db(4 * math.pi * (n1 * L * L) ** 2 / lam ** 2)) < 1e-3
    tr = res.traces[1]
    n2 = int(((tr.M == 2) & (tr.psi == 1)).sum())
    s45 = res.sigma[1, 0]
    ap = n2 * L * L
    assert abs(oracle.db(s45[0, 0]) - oracle.db(4 * math.pi * ap ** 2 / lam ** 2)) < 0.05
    assert abs(oracle.db(s45[1, 1]) - oracle.db(4 * math.pi * ap ** 2 / lam ** 2)) < 0.05
    assert abs(ap / (math.sqrt(2) * 0.25) - 1) < 0.15


def test_rcs_dihedral_mirror_symmetry():
    # the regular-grid dihedral is symmetric about x = y, so
    # sigma(phi) = sigma(90 deg - phi)
    sc = scenes.dihedral(4000, seed=3, jitter=False)
    vd = scenes.aggregation_views(sc, 96, 96)
    S, gv, gf, fp = oracle.build_geometry(sc, vd, "fp64")
    eps = oracle.default_eps(gv)
    sw = scenes._sweep_over(sc, [90.0] * 4, [12.0, 78.0, 30.0, 60.0], 64, [3e9], 2)
    res = oracle.rcs_sweep(sc, sw, S, eps, eps, mode="fp64")
    sd = oracle.db(res.sigma[:, 0, 0, 0])
    assert abs(sd[0] - sd[1]) < 0.05
    assert abs(sd[2] - sd[3]) < 0.05


def test_rcs_sphere_surfels_vs_exact_po():
    sc = scenes.sphere(20000, 1.0)
    f = 3e9
    k = 2 * math.pi * f / C0
    sw = scenes._sweep_over(sc, [90.0, 30.0], [0.0, 200.0], 128, [f], 1)
    res = oracle.rcs_sweep(sc, sw, None, 0.01, 0.01)
    b = 2 * k
    ref = 4 * math.pi * k ** 2 * abs(np.exp(1j * b) / (1j * b) + (np.exp(1j * b) - 1) / b ** 2) ** 2
    assert np.max(np.abs(oracle.db(res.sigma[:, 0, 0, 0]) - oracle.db(ref))) < 0.15
    assert np.max(np.abs(oracle.db(res.sigma[:, 0, 1, 1]) - oracle.db(ref))) < 0.15


def _roll(scene, axis, deg):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    R = np.eye(3) + math.sin(math.radians(deg)) * K + (1 - math.cos(math.radians(deg))) * K @ K
    return scenes.Scene(pos=(scene.pos.astype(np.float64) @ R.T).astype(np.float32),
                        nrm=(scene.nrm.astype(np.float64) @ R.T).astype(np.float32), rad=scene.rad)


def test_rolled_dihedral_twist_and_reciprocity():
    # Seen into its corner, a dihedral's double bounce acts on the (V, H)
    # amplitudes as diag(1, -1) in the dihedral's own frame; rolled by psi
    # about the line of sight it becomes [[cos 2psi, sin 2psi], [sin 2psi,
    # -cos 2psi]]: co- to cross-polarised power cot^2(2 psi) (equal at 22.5
    # deg, -4.77 dB at 30, all cross-polarised at 45) and sigma_VH = sigma_HV
    # (monostatic reciprocity).
    base = scenes.dihedral(6000, seed=21)
    w = [math.cos(math.pi / 4), math.sin(math.pi / 4), 0.0]
    for psi in (22.5, 30.0, 45.0):
        sc = _roll(base, w, psi)
        S, gv, _, _ = oracle.build_geometry(sc, scenes.aggregation_views(sc, 128, 128), "fp32")
        eps = oracle.default_eps(gv)
        sw = scenes._sweep_over(sc, [90.0], [45.0], 96, [3e9, 3.4e9], 2)
        s = oracle.rcs_sweep(sc, sw, S, eps, eps).sigma[0]       # [F][tx][rx]
        assert np.all(np.abs(s[:, 0, 1] - s[:, 1, 0]) < 1e-5 * s[:, 0, 1])
        ratio = oracle.db(s[:, 0, 0]) - oracle.db(s[:, 0, 1])
        if psi == 45.0:
            assert np.all(ratio < -30.0), ratio
        else:
            expect = 20 * math.log10(1 / math.tan(math.radians(2 * psi)))
            assert np.all(np.abs(ratio - expect) < 0.3), (psi, ratio, expect)


def test_rcs_sphere_converges_with_sampling():
    # the surfel sphere's monostatic sigma approaches the exact PO value as
    # the points and the ray screen are refined together (1500 points on
    # 40^2 rays, 5000 on 64^2, 20000 on 128^2): the mean dB error over four
    # aspects and both polarisations at least halves at each step
    f = 3e9
    k = 2 * math.pi * f / C0
    b = 2 * k
    ref = 4 * math.pi * k ** 2 * abs(np.exp(1j * b) / (1j * b) + (np.exp(1j * b) - 1) / b ** 2) ** 2
    th, ph = [90.0, 30.0, 120.0, 75.0], [0.0, 200.0, 45.0, 310.0]
    errs = []
    for n, W in ((1500, 40), (5000, 64), (20000, 128)):
        sc = scenes.sphere(n, 1.0)
        res = oracle.rcs_sweep(sc, scenes._sweep_over(sc, th, ph, W, [f], 1), None, 0.01, 0.01)
        errs.append(np.abs(oracle.db(res.sigma[:, 0, [0, 1], [0, 1]]) - oracle.db(ref)).mean())
    assert errs[1] < 0.5 * errs[0] and errs[2] < 0.5 * errs[1], errs
    assert errs[2] < 0.15


def test_point_order_changes_only_the_hit_labels():
    # GFB keys order candidates by depth, then index, and fusion sorts by
    # (voxel, view, pixel) and stores each splat at a pixel slot: with no two
    # points at exactly the same depth on a pixel, permuting the points
    # relabels the GFB hit ids and changes nothing else -- depth, normals,
    # splats, traces and the field are bit-identical.
    sc = scenes.sphere(3000, 1.0)
    perm = np.random.default_rng(17).permutation(3000)
    sp = scenes.Scene(pos=sc.pos[perm], nrm=sc.nrm[perm], rad=sc.rad[perm])
    v = oracle.view_from_angles(70.0, 30.0, [0, 0, 0], 1.05, 48, 48, "fp32")
    g0, g1 = oracle.gfb(sc, v, "fp32"), oracle.gfb(sp, v, "fp32")
    hit = g0.idx >= 0
    assert hit.sum() > 1000
    assert np.array_equal(g0.depth, g1.depth) and np.array_equal(g0.nrm, g1.nrm)
    assert np.array_equal(perm[g1.idx[hit]], g0.idx[hit])
    vd = scenes.aggregation_views(sc, 48, 48)
    S0, gv, _, _ = oracle.build_geometry(sc, vd, "fp32")
    S1, _, _, _ = oracle.build_geometry(sp, vd, "fp32")
    for name in ("id", "c", "n", "r", "count"):
        assert np.array_equal(getattr(S0, name), getattr(S1, name)), name
    eps = oracle.default_eps(gv)
    sw = scenes._sweep_over(sc, [90.0, 60.0], [0.0, 100.0], 40, [3e9, 3.3e9], 2)
    r0 = oracle.rcs_sweep(sc, sw, S0, eps, eps)
    r1 = oracle.rcs_sweep(sp, sw, S1, eps, eps)
    assert np.array_equal(r0.E, r1.E)


def _golden_sigma(kind, freq_hz):
    """The oracle's monostatic co-polarised sigma (V and H) of a golden row's
    target: the workloads' own generators, surfel splats fused from 8 views
    for the multi-bounce targets, ray pitch well below lambda/10."""
    trih_th = math.degrees(math.acos(1 / math.sqrt(3)))
    if kind in ("dihedral45", "dihedral_face"):
        sc = scenes.workload_dihedral().scene            # a = b = 0.5 m, 10k points
        ph = 45.0 if kind == "dihedral45" else 0.0
        th, W, mb, views = 90.0, 128, 2, 256
    elif kind == "sphere":
        sc = scenes.sphere(50_000, 1.0)
        th, ph, W, mb, views = 90.0, 0.0, 512, 1, 0
    elif kind == "plate":
        sc = scenes.plate(1.0, 1.0, 200, 200)
        th, ph, W, mb, views = 0.0, 0.0, 512, 1, 0
    else:
        sc = scenes.trihedral(60_000, a=0.6)
        th, ph, W, mb, views = trih_th, 45.0, 384, 3, 256
    S, eps = None, 0.01
    if mb > 1:
        S, gv, _, _ = oracle.build_geometry(sc, scenes.aggregation_views(sc, views, views), "fp32")
        eps = oracle.default_eps(gv)
    res = oracle.rcs_sweep(sc, scenes._sweep_over(sc, [th], [ph], W, [freq_hz], mb), S, eps, eps)
    s = res.sigma[0, 0]
    return oracle.db(s[0, 0]), oracle.db(s[1, 1]), sc


def test_golden_closed_forms():
    """The oracle's sigma of the standard workloads' targets against their
    textbook PO values (stored with their sources in tests/golden).  A
    surfel target realises its aperture up to its disks' overhang at the
    edges: a square plate of side a whose edge disks reach R beyond it has
    at most (a + 2R)^2 of area, and sigma ~ A^2, so its excess is at most
    40 log10(1 + 2R/a) dB; the sphere has no edge and the textbook value
    pi a^2 is its optical limit (the exact PO value differs by 0.02 dB at
    ka = 209); the trihedral's triple-bounce aperture loses the rays that
    miss an edge disk at the corners' seams (measured within 0.25 dB)."""
    g = json.load(open(os.path.join(GOLDEN, "closed_forms.json")))
    which = {("dihedral", 0): "dihedral45", ("plate", 3e9): "dihedral_face",
             ("sphere", 0): "sphere", ("plate", 1e10): "plate", ("trihedral", 0): "trihedral"}
    for row in g["rows"]:
        kind = which.get((row["kind"], 0)) or which[(row["kind"], row["freq_hz"])]
        v, h, sc = _golden_sigma(kind, row["freq_hz"])
        if kind in ("dihedral45", "dihedral_face", "plate"):
            a = row["a"]
            over = 40 * math.log10(1 + 2 * float(sc.rad.max()) / a)
            lo, hi = -0.15, over + 0.15
        elif kind == "sphere":
            lo, hi = -0.1, 0.1
        else:
            lo, hi = -0.5, 0.5
        for pol, val in (("V", v), ("H", h)):
            dv = val - row["dbsm"]
            assert lo <= dv <= hi, (row["note"], pol, val, row["dbsm"], (lo, hi))


# ----------------------------------------------------------------------------
# the field's compensated sum (Neumaier)
# ----------------------------------------------------------------------------

def _acc_sum(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty(2, np.float64)
    oracle.lib().or_acc_sum(oracle._p(x), x.shape[0], oracle._p(out))
    return out[0], out[1]            # compensated, plain left-to-right


def test_neumaier_sum_against_exact_rational_sums():
    """The field's accumulator (Neumaier's compensated summation) against
    the exact sum of its FP64 terms, computed in rational arithmetic.  Its
    error bound is |S - S_hat| <= eps |S| + O(n eps^2) sum |x_i|; the plain
    sum's is (n - 1) eps sum |x_i|, so on ill-conditioned lists the plain
    sum loses every digit that the compensated one keeps."""
    from fractions import Fraction
    # hand cases: a term below the running sum's ulp between two that
    # cancel (1e16 + 1 rounds to 1e16), and one where a term larger than
    # the running sum arrives (Kahan's form without Neumaier's branch
    # returns 0 here, the exact sum is 2)
    for xs, exact in (([1e16, 1.0, -1e16], 1.0), ([1.0, 1e100, 1.0, -1e100], 2.0),
                      ([0.1] * 10, float(sum(Fraction(0.1) for _ in range(10))))):
        comp, plain = _acc_sum(xs)
        assert comp == exact, (xs, comp)
    assert _acc_sum([1e16, 1.0, -1e16])[1] == 0.0
    assert _acc_sum([1.0, 1e100, 1.0, -1e100])[1] == 0.0
    # random ill-conditioned lists: terms up to 1e15 that cancel in pairs,
    # shuffled among small ones (the exact sum is the small terms' sum)
    rng = np.random.default_rng(11)
    eps = 2.0 ** -53
    worse = 0
    for trial in range(40):
        n = int(rng.integers(3, 200))
        big = rng.standard_normal(n) * 10.0 ** rng.uniform(0, 15, n)
        small = rng.standard_normal(int(rng.integers(1, 50))) * 10.0 ** rng.uniform(-3, 0)
        x = np.concatenate([big, -big, small])
        rng.shuffle(x)
        exact = sum(Fraction(float(t)) for t in x)
        comp, plain = _acc_sum(x)
        err_c = abs(Fraction(comp) - exact)
        err_p = abs(Fraction(plain) - exact)
        bound = eps * abs(exact) + 4 * len(x) * eps * eps * sum(Fraction(abs(float(t))) for t in x)
        assert err_c <= bound, (trial, float(err_c), float(bound))
        assert err_c <= err_p
        worse += err_p > 1000 * err_c
    assert worse > 30        # the plain sum is far worse on most of them


def test_po_field_keeps_a_term_below_the_running_sums_ulp():
    """Eq. 14's sum over rays is compensated: a ray whose contribution is
    1e-18 of two others that cancel exactly (the same ray with its normal
    turned over: the vector factor changes sign, nothing else) survives in
    the field, as the field of that ray alone.  A plain FP64 sum returns
    zero."""
    big = 3e8
    n_hat = np.array([0.0, 0.0, 1.0])
    d = np.array([0.3, 0.0, -math.sqrt(1 - 0.09)])
    p = np.array([[0.01, 0.02, 0.0]] * 3)
    u = np.array([[big * 0.9, 0.0, big * 0.3], [0.9e-3, 0.0, 0.3e-3], [big * 0.9, 0.0, big * 0.3]])
    v = np.array([[0.0, big, 0.0], [0.0, 1e-3, 0.0], [0.0, big, 0.0]])
    nn = np.array([n_hat, n_hat, -n_hat])
    tr = oracle.Trace(M=np.ones(3, np.int32), ids=np.zeros((3, 1), np.int64), p=p, n=nn,
                      k=np.tile(d, (3, 1)), u=u, v=v, path=p @ d, psi=np.ones(3, np.uint8))
    ks = -d
    E3 = oracle.po_field(tr, [3e9, 7e9], ks)
    one = oracle.Trace(M=np.ones(1, np.int32), ids=np.zeros((1, 1), np.int64), p=p[1:2],
                       n=nn[1:2], k=d[None], u=u[1:2], v=v[1:2], path=p[1:2] @ d,
                       psi=np.ones(1, np.uint8))
    E1 = oracle.po_field(one, [3e9, 7e9], ks)
    assert np.abs(E1).max() > 0
    assert np.allclose(E3, E1, rtol=1e-12, atol=0.0)


# ----------------------------------------------------------------------------
# surfel attributes (radius from the k nearest points, PCA normals)
# ----------------------------------------------------------------------------

def test_knn_radius_and_normal_on_a_square_lattice():
    # 9 x 9 lattice of pitch 1/8 in z = 0: an interior point's 8 nearest
    # other points are 4 at 1/8 and 4 at sqrt(2)/8, so R = (1 + sqrt 2)/16;
    # the plane's normal is +z (turned to agree with the reference)
    a = 0.125
    g = np.stack(np.meshgrid(np.arange(9), np.arange(9), indexing="ij"), -1).reshape(-1, 2) * a
    pos = np.concatenate([g, np.zeros((81, 1))], axis=1).astype(np.float32)
    ref = np.tile([0.0, 0.0, 1.0], (81, 1))
    r, n, w, _ = oracle.point_attributes(pos, 8, 9, ref=ref)
    inner = [i for i in range(81) if 2 <= i // 9 <= 6 and 2 <= i % 9 <= 6]
    expect = np.float32(a * (1.0 + math.sqrt(2.0)) / 2.0)
    assert np.all(np.abs(r[inner] - expect) <= 1e-7 * expect)
    assert np.allclose(n, ref, atol=1e-12)
    assert np.allclose(w[:, 0], 0.0, atol=1e-12)


def test_knn_distances_match_an_independent_kd_tree():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(4)
    pos = rng.random((2000, 3)).astype(np.float32)
    idx, d2 = oracle.knn(pos, 12)
    dk, _ = cKDTree(pos.astype(np.float64)).query(pos.astype(np.float64), k=12)
    assert np.allclose(np.sqrt(d2.astype(np.float64)), dk, rtol=2e-6, atol=1e-7)
    assert np.all(idx[:, 0] == np.arange(2000))        # itself first (distance 0)


def test_pca_normal_of_a_tilted_plane_and_duplicates():
    rng = np.random.default_rng(5)
    nrm = np.array([1.0, 2.0, 2.0]) / 3.0
    t1 = np.array([2.0, -1.0, 0.0]) / math.sqrt(5.0)
    t2 = np.cross(nrm, t1)
    uv = rng.random((3000, 2)) * 4.0 - 2.0
    pos = (uv[:, :1] * t1 + uv[:, 1:] * t2 + 0.5).astype(np.float32)
    _, n, _, _ = oracle.point_attributes(pos, 8, 16, ref=np.tile(nrm, (3000, 1)))
    assert np.max(np.arccos(np.clip(n @ nrm, -1, 1))) < 2e-5
    # a duplicated point: its twin is a neighbour at distance 0; only the
    # point itself is left out of its radius
    dup = np.concatenate([pos[:50], pos[:1]]).astype(np.float32)
    r, _, _, idx = oracle.point_attributes(dup, 4, 8)
    d = np.sqrt(((dup[:, None, :].astype(np.float64) - dup[None]) ** 2).sum(-1))
    d0 = np.sort(np.delete(d[0], 0))[:4]
    assert d0[0] == 0.0 and abs(r[0] - d0.mean()) < 1e-6 * max(d0.mean(), 1e-9)


# ----------------------------------------------------------------------------
# Alg. 1 with a finite K (the heap of K points nearest the central ray)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_alg1_finite_k_hand_case(mode):
    # one pixel looking down -z from z = 5; delta = 0.1.  A: depth 4 (z = 1),
    # 0.03 off the axis; C: depth 3, 0.05 off; B: depth 2, 0.08 off.
    # K = 1 keeps A (most central): 4; K = 2 keeps A, C: 3; K >= 3: 2.
    v = down_view(1, 1, 1.0)
    pos = np.array([[0.03, 0.0, 1.0], [0.0, 0.08, 3.0], [0.0, -0.05, 2.0]], np.float32)
    for K, i in {1: 0, 2: 2, 3: 1, 8: 1}.items():
        g = oracle.gfb_topk(pos, v, 0.1, K, mode)
        assert g.idx[0] == i
        # the score is Length(p - o), o = (0, 0, 5) the pixel's origin
        expect = np.linalg.norm(pos[i].astype(np.float64) - [0.0, 0.0, 5.0])
        assert abs(g.depth[0] - expect) < 1e-6


def test_alg1_large_k_equals_the_unbounded_heap():
    rng = np.random.default_rng(9)
    sc = mk_scene(rng.random((400, 3)) * [1.0, 1.0, 0.2], np.tile([0, 0, 1.0], (400, 1)),
                  np.full(400, 0.05))
    v = down_view(24, 24, 1.0 / 24, z=3.0)
    v.o = v.o + np.array([0.5, 0.5, 0.0])
    g_inf = oracle.gfb(sc, v, "fp32", tube=True, delta=0.06)
    g_k = oracle.gfb_topk(sc.pos, v, 0.06, 64, "fp32")
    assert np.array_equal(g_inf.idx, g_k.idx) and np.array_equal(g_inf.depth, g_k.depth)
    assert (g_inf.idx >= 0).mean() > 0.5
    g1 = oracle.gfb_topk(sc.pos, v, 0.06, 1, "fp32")
    assert np.array_equal(g1.idx >= 0, g_inf.idx >= 0)      # same hit pixels
    assert (g1.idx != g_inf.idx).mean() > 0.05               # but other points chosen


# ----------------------------------------------------------------------------
# bistatic observation (Eq. 14 toward other receivers, Psi per receiver)
# ----------------------------------------------------------------------------

def _splats_of(rows):
    if not rows:
        z = np.zeros((0, 3))
        return oracle.Splats(id=np.zeros(0, np.int64), c=z, n=z, r=np.zeros(0),
                             count=np.zeros(0, np.int32), keep=np.zeros(0, np.uint8))
    return _splats(rows)


@pytest.mark.parametrize("beta", [0.0, 15.0, 40.0])
def test_bistatic_plate_exact_integral_and_receiver_shadowing(beta):
    # a 0.5 x 0.3 plate lit at normal incidence, received at beta from the
    # normal in the xz-plane: the sum of the cells' Eq. 11 terms is the exact
    # plate integral |U x V| sinc(q.U/2) sinc(q.V/2), q = k (k_in - k_s),
    # times [(n x h) x k_s] x k_s for each transmit polarisation
    f = 3e9
    k = 2 * math.pi * f / C0
    tr, w, u, v, U, V = _plate_cells(0.0, 0.5, 0.3, 40, 30)
    ks = np.array([math.sin(math.radians(beta)), 0.0, math.cos(math.radians(beta))])
    E = oracle.po_field_bistatic(tr, _splats_of([]), [f], [ks], 1e-3)[0, 0]   # [pol][3]
    q = k * (-w - ks)
    sinc = lambda x: math.sin(x) / x if x else 1.0
    I = np.linalg.norm(np.cross(U, V)) * sinc(q @ U / 2) * sinc(q @ V / 2)
    n = np.array([0.0, 0.0, 1.0])
    us, vs = tr.u[0], tr.v[0]
    for pol, h in ((0, -vs / np.linalg.norm(vs)), (1, us / np.linalg.norm(us))):
        vec = np.cross(np.cross(np.cross(n, h), ks), ks)
        assert np.allclose(E[pol].real, I * vec, rtol=1e-9, atol=1e-12 * abs(I))
        assert np.allclose(E[pol].imag, 0.0, atol=1e-9 * abs(I))
    # a large disk above the plate blocks every receiver on that side
    lid = _splats_of([(0, [0.0, 0.0, 0.5], [0.0, 0.0, 1.0], 10.0)])
    assert np.all(oracle.shadow_dirs(tr, lid, [ks], 1e-3) == 0)
    assert np.all(oracle.po_field_bistatic(tr, lid, [f], [ks], 1e-3) == 0)


def test_bistatic_psi_toward_the_transmitter_is_the_monostatic_psi():
    # dihedral rays that bounce twice: the receiver at the transmitter sees
    # the monostatic shadow test exactly; single-bounce rays are unblocked
    sc = scenes.dihedral(2000, seed=5)
    vd = scenes.aggregation_views(sc, 64, 64)
    S, gv, _, _ = oracle.build_geometry(sc, vd, "fp32")
    eps = oracle.default_eps(gv)
    c, r = scenes.bounding_sphere(sc.pos)
    v = oracle.view_from_angles(90.0, 40.0, c, r * 1.02, 32, 32, "fp32")
    tr = oracle.trace(v, S, 2, eps, eps, first=oracle.gfb(sc, v, "fp32"), mode="fp32")
    psi = oracle.shadow_dirs(tr, S, [-np.asarray(v.d)], eps)[0]
    two = tr.M >= 2
    assert two.sum() > 50
    assert np.array_equal(psi[two], tr.psi[two])
    assert psi[tr.M == 1].mean() > 0.95


# ----------------------------------------------------------------------------
# PO at every bounce (the variant of Eq. 14 that sums the field of every hit)
# ----------------------------------------------------------------------------

def test_every_bounce_field_on_the_dihedral(dihedral_geom):
    # phi = 0: broadside to the plate x = 0 and edge-on to y = 0, so no ray
    # hits twice and PO at every bounce is the last-hit field exactly.
    # phi = 45: the last-hit field is the double bounce (pinned above), and the
    # every-bounce field adds each double-bounce ray's first hit: the two
    # a x a plates seen 45 deg off their normals.  Each contributes
    # cos(45) a |integral_0^l exp(j q x) dx|, q = 2 k cos(45), in phase with
    # the other for both polarisations (the PO currents 2 n x H of the two
    # plates project onto e_V and e_H with the same sign).  At q a / 2 =
    # 7.5 pi the integral is at a sidelobe peak, 2 / q; the illuminated
    # length l is a to within one projected screen cell (pitch / cos 45), so
    # |sin(q l / 2)| >= cos(q pitch / (2 cos 45)), and the height is a to
    # within a pitch at each end.
    sc, S, gv = dihedral_geom
    eps = oracle.default_eps(gv)
    a = 0.5
    q = 15 * math.pi / a
    f = q / math.sqrt(2) * C0 / (2 * math.pi)
    for phi in (0.0, 45.0):
        sw = scenes._sweep_over(sc, [90.0], [phi], 96, [f], 2)
        v = oracle.sweep_views(sw)[0]
        Ee = oracle.po_field_every_bounce(v, S, oracle.gfb(sc, v), 2, eps, eps, [f])
        res = oracle.rcs_sweep(sc, sw, S, eps, eps)
        El = res.E[0]
        if phi == 0.0:
            assert res.traces[0].M.max() == 1
            assert np.array_equal(Ee, El)
            continue
        assert int((res.traces[0].M == 2).sum()) > 4000
        e = np.stack([v.u, v.v])                    # e_V, e_H
        d = np.abs(np.einsum("ftc,tc->ft", Ee - El, e)[0])
        peak = 2 * math.cos(math.pi / 4) * a * 2 / q
        lo = math.cos(q * v.pitch / (2 * math.cos(math.pi / 4))) * (1 - 2 * v.pitch / a)
        hi = 1 + 2 * v.pitch / a
        assert np.all(d > lo * peak) and np.all(d < hi * peak), (d / peak, lo, hi)
        # and the first hits are a sidelobe: about 28 dB below the double bounce
        assert np.all(d < 0.06 * np.abs(np.einsum("ftc,tc->ft", El, e)[0]))


# ----------------------------------------------------------------------------
# Canny edge mode of the fusion (edge_mode 1)
# ----------------------------------------------------------------------------

def _canny_keep(depth, mode="fp32", tau=3.0):
    W = H = depth.shape[0]
    v = down_view(W, H, 0.125)
    g = _handmade_gfb(v, depth.ravel(), np.tile([0.0, 0.0, 1.0], (W * H, 1)), np.ones(W * H))
    fp = oracle.FuseParams(tau=tau, bmin=np.array([-2.0, -2.0, -40.0]), inv_vox=8.0, G=256,
                           edge_mode=1)
    return oracle.aggregate([g], fp, mode).keep.reshape(H, W)


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_canny_ramp_threshold_and_flat_map(mode):
    # a linear ramp of slope s metres per pixel: smoothing keeps it, Sobel
    # gives 8 s, so interior pixels are strong iff 8 s >= 8 tau L = 3 (all
    # equal: the suppression keeps them); below low = 1.5 nothing survives.
    # Dyadic slopes keep every step exact in both precisions.
    tau, n = 3.0, 24
    ii = np.arange(n)[None, :] * np.ones((n, 1))
    inner = (slice(3, n - 3), slice(3, n - 3))
    keep_hi = _canny_keep(5.0 + 0.5 * ii, mode, tau)      # 8 s = 4 >= 3
    keep_lo = _canny_keep(5.0 + 0.125 * ii, mode, tau)    # 8 s = 1 < 1.5
    keep_flat = _canny_keep(np.full((n, n), 5.0), mode, tau)
    assert not keep_hi[inner].any()                 # every interior pixel an edge
    assert keep_lo[inner].all() and keep_flat[1:-1, 1:-1].all()
    assert not keep_flat[0].any()                   # the border rule still applies


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_canny_step_gives_the_two_columns_beside_it(mode):
    # a depth step between columns 9 and 10: the smoothed profile is
    # symmetric about 9.5, the two columns beside the step tie in gradient and
    # both survive suppression; everything else keeps (besides the border)
    n = 24
    d = np.full((n, n), 5.0)
    d[:, 10:] = 5.0 + 20 * 0.125
    keep = _canny_keep(d, mode)
    interior = keep[1:-1, 1:-1]
    cols = np.flatnonzero(~interior.any(axis=0)) + 1
    assert list(cols) == [9, 10]
    assert interior[:, [c - 1 for c in range(1, n - 1) if c not in (9, 10)]].all()


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
def test_canny_weak_step_alone_and_joined_to_a_strong_one(mode):
    # After the 5 x 5 binomial smoothing a depth step of height h between
    # columns 9 and 10 reads 1/16, 5/16, 11/16, 15/16 of h on columns 8..11,
    # so the Sobel response on both columns beside it is 4 (11 - 1) h / 16 =
    # 2.5 h.  With tau = 3, L = 0.125: high = 8 tau L = 3, low = 1.5.
    # h = 0.875 gives 2.1875, a weak response: alone, no edge.  Continuing a
    # strong step (h = 2: 5) along the same columns, the hysteresis carries
    # it: away from the junction (rows 9-14), both columns are edges in the
    # strong half and in the weak half.
    n = 24
    weak = np.full((n, n), 5.0)
    weak[:, 10:] = 5.875
    assert _canny_keep(weak, mode)[1:-1, 1:-1].all()
    joined = weak.copy()
    joined[:12, 10:] = 7.0
    edge = _canny_keep(joined, mode) == 0
    for r in list(range(1, 9)) + list(range(15, n - 1)):
        assert edge[r, 9] and edge[r, 10], r
