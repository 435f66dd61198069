"""Parity at the limits the C ABI declares, through the whole path.

* PE_MAX_VIEWS: a geometry fused from 16 views, splats bit-exact.
* Deep bounces: a 30 degree wedge (two plates hinged along the y-axis), where
  rays from above reflect back and forth up to six times; traced with
  max_bounces 8 and 64 (the maximum) on screens that are not a multiple of
  the 8 x 4 ray tiles, hit ids, bounce counts and Psi bit-exact, with
  max_bounces 4 (every deeper ray cut at its fourth hit), with the first
  bounce taken from the geometry, and on one-row, one-column and one-ray
  screens.  The screens look straight down (ray directions with exact zero
  components) or nearly so; bistatic receivers along the coordinate axes.
* Fusion: grids of 1, 7 and 64 voxels per edge, and views of two screen
  sizes in one geometry.
* Frequencies and groups beyond one PO launch: 600 frequencies (launches of
  256, 256 and 88) over 70 receiver groups (launches of 64 and 6), and a
  sweep of 4100 frequencies, more than the library stages at once.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _mods():
    from paper_2408_15583_gb300 import api, pipeline
    return api, pipeline


def _oviews(th, ph, centre, extent, W, H):
    """The oracle's own views for the angles the library's views are made
    from (every oracle input is built on the oracle's side)."""
    return [oracle.view_from_angles(t, p, centre, extent, W, H, "fp32") for t, p in zip(th, ph)]


def _cplx(E):
    E = E.detach().cpu().numpy()
    return E[..., 0] + 1j * E[..., 1]


def field_err(E, Eref):
    d = np.sqrt((np.abs(E - Eref) ** 2).sum(axis=-1))
    r = np.sqrt((np.abs(Eref) ** 2).sum(axis=-1))
    return d / np.maximum(r, 1e-3 * r.max())


def wedge(n_points=3000, L=0.6, half_deg=15.0, seed=17):
    """Two L x L plates hinged along the y-axis, each at half_deg from +z,
    opening upward; inner normals.  One uniform point per grid cell."""
    rng = np.random.Generator(np.random.PCG64(seed))
    per = n_points // 2
    n_u = int(round(math.sqrt(per)))
    n_v = per // n_u
    h = math.radians(half_deg)
    ps, ns = [], []
    for sgn in (1.0, -1.0):
        s, y = scenes._stratified_rect(rng, n_u, n_v, L, L)
        along = np.array([sgn * math.sin(h), 0.0, math.cos(h)])
        ps.append(s[:, None] * along[None] + (y - L / 2)[:, None] * np.array([0.0, 1.0, 0.0]))
        ns.append(np.tile([-sgn * math.cos(h), 0.0, math.sin(h)], (s.size, 1)))
    return scenes._finish(np.concatenate(ps), np.concatenate(ns), "wedge", seed)


@pytest.fixture(scope="module")
def wedge16():
    api, pipe = _mods()
    sc = wedge()
    c, r = scenes.bounding_sphere(sc.pos)
    th = np.repeat([0.0, 10.0, 20.0, 30.0], 4)
    ph = np.tile([0.0, 90.0, 180.0, 270.0], 4)
    pos, nrm, rad = pipe.scene_to_device(sc, DEV)
    gv = pipe.views_from_angles(th, ph, c, r * 1.02, 64, 64)
    assert len(gv) == 16
    prm = pipe.default_params(sc.pos, gv)
    geom, _ = pipe.build_geometry(pos, nrm, rad, gv, prm)
    api.stream_check()
    ogv = _oviews(th, ph, c, r * 1.02, 64, 64)
    ogf = [oracle.gfb(sc, v, "fp32") for v in ogv]
    fp = oracle.fuse_params(sc)
    S = oracle.aggregate(ogf, fp, "fp32")
    return dict(sc=sc, c=c, r=r, pos=pos, nrm=nrm, rad=rad, gv=gv, prm=prm, geom=geom, S=S,
                ogf=ogf, fp=fp, eps=oracle.default_eps(ogv))


def test_sixteen_view_fusion_bitexact(wedge16):
    d = wedge16
    cr, nf = d["geom"].planes()
    cr = cr.cpu().numpy()
    nf = nf.cpu().numpy()
    ids = np.flatnonzero(cr[:, 3] > 0)
    S = d["S"]
    assert S.ns > 2000
    assert np.array_equal(ids, S.id)
    assert np.array_equal(cr[ids, :3].astype(np.float64), S.c)
    assert np.array_equal(cr[ids, 3].astype(np.float64), S.r)
    assert np.array_equal(nf[ids, :3].astype(np.float64), S.n)
    assert np.array_equal(nf[ids, 3].astype(np.int64), S.count)
    # views 9-16 change the fused set (they are not ignored)
    S8 = oracle.aggregate(d["ogf"][:8], d["fp"], "fp32")
    assert S8.ns != S.ns or not np.array_equal(S8.id, S.id)


def _trace_vs_oracle(d, th, ph, centre, extent, W, H, mb, geom_first=False):
    """Trace the screens of angles (th, ph) through the ABI and the oracle;
    every record bit-exact.  Returns the oracle traces."""
    api, pipe = _mods()
    sc = d["sc"]
    views = pipe.views_from_angles(th, ph, centre, extent, W, H)
    prm = pipe.default_params(sc.pos, d["gv"], first_bounce_from_geom=geom_first)
    keys = None
    if not geom_first:
        keys = api.build_gfb(views, d["pos"], d["nrm"], d["rad"], 0, outputs=("keys",))["keys"]
    h = api.trace_bounces(views, keys, d["nrm"], d["geom"], mb, prm)
    api.stream_check()
    per = W * H
    trs = []
    for a, ov in enumerate(_oviews(th, ph, centre, extent, W, H)):
        first = None if geom_first else oracle.gfb(sc, ov, "fp32")
        tr = oracle.trace(ov, d["S"], mb, d["eps"], d["eps"], first=first, mode="fp32")
        sl = slice(a * per, (a + 1) * per)
        assert np.array_equal(h.M[sl].cpu().numpy(), tr.M), f"angle {a}"
        ids = h.ids[:, sl].cpu().numpy().view(np.uint32).astype(np.int64)
        ids[ids == 0xFFFFFFFF] = -1
        assert np.array_equal(ids.T, tr.ids), f"angle {a}"
        assert np.array_equal(h.psi[sl].cpu().numpy(), tr.psi)
        live = tr.M > 0
        for name in ("p", "n", "k", "u", "v"):
            got = getattr(h, name)[sl].cpu().numpy().astype(np.float64)
            assert np.array_equal(got[live], getattr(tr, name)[live]), name
        assert np.allclose(h.path[sl].cpu().numpy()[live], tr.path[live], rtol=1e-13, atol=1e-13)
        trs.append(tr)
    return trs


@pytest.mark.parametrize("mb,geom_first", [(8, False), (4, False), (64, False), (8, True)])
def test_wedge_deep_bounces_bitexact(wedge16, mb, geom_first):
    # screens from straight above (theta = 0: d = (0, 0, -1), whose
    # reflections keep d_y = 0 exactly) and slightly off it; 42 x 38 rays
    api, pipe = _mods()
    d = wedge16
    trs = _trace_vs_oracle(d, [0.0, 5.0, 8.0], [0.0, 90.0, 200.0], d["c"], d["r"] * 1.02,
                           42, 38, mb, geom_first)
    M = np.concatenate([t.M for t in trs])
    deep = int((M >= 5).sum()) if mb >= 5 else int((M == mb).sum())
    assert deep > 300            # the case reaches the deep bounces (or the cut)
    assert M.max() < min(mb, 8) + 1


@pytest.mark.parametrize("W,H", [(1, 9), (13, 1), (1, 1)])
def test_wedge_thin_screens_bitexact(wedge16, W, H):
    # one-row, one-column and one-ray screens (a single partial 8 x 4 tile);
    # the pitch is fixed by W, so the 1-column screen is a column of wide
    # cells down the middle of the wedge
    api, pipe = _mods()
    d = wedge16
    trs = _trace_vs_oracle(d, [0.0, 3.0], [0.0, 45.0], d["c"], d["r"] * 1.02, W, H, 8)
    assert sum(int((t.M > 0).sum()) for t in trs) > 0


def test_wedge_bistatic_axis_receivers(wedge16):
    # receivers along the coordinate axes (shadow rays with two zero
    # components) and the transmitter's own direction; inside the wedge the
    # receivers along x are blocked by the plates
    api, pipe = _mods()
    d = wedge16
    sc = d["sc"]
    views = pipe.views_from_angles([0.0, 5.0], [0.0, 90.0], d["c"], d["r"] * 1.02, 40, 40)
    ovs = _oviews([0.0, 5.0], [0.0, 90.0], d["c"], d["r"] * 1.02, 40, 40)
    mb = 8
    keys = api.build_gfb(views, d["pos"], d["nrm"], d["rad"], 0, outputs=("keys",))["keys"]
    h = api.trace_bounces(views, keys, d["nrm"], d["geom"], mb, d["prm"], ids=False)
    freqs = scenes.freq_grid(2.5e9, 3.5e9, 3)
    axes = [[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]]
    obs = np.asarray([[list(-np.asarray(ov.d, np.float64))] + axes for ov in ovs], np.float32)
    E = _cplx(api.po_field_bistatic(h, 2, 40 * 40, obs, d["geom"], float(d["prm"].eps), freqs))
    api.stream_check()
    eps = d["eps"]
    blocked = 0
    for a, ov in enumerate(ovs):
        tr = oracle.trace(ov, d["S"], mb, eps, eps, first=oracle.gfb(sc, ov, "fp32"), mode="fp32")
        o64 = obs[a].astype(np.float64)
        Eo = oracle.po_field_bistatic(tr, d["S"], freqs, o64, eps)
        blocked += int((oracle.shadow_dirs(tr, d["S"], o64, eps) == 0)[:, tr.M > 0].sum())
        assert field_err(E[a], Eo).max() < 1e-3, f"angle {a}"
    assert blocked > 100


def test_wedge_sweep_beyond_the_staged_frequencies(wedge16):
    # 4100 frequencies: wavenumbers staged in two pieces, PO in 17 launches
    api, pipe = _mods()
    d = wedge16
    sc = d["sc"]
    sw = scenes._sweep_over(sc, [0.0, 6.0], [0.0, 120.0], 32, scenes.freq_grid(2e9, 4e9, 4100), 8)
    E, sig = api.rcs_sweep(api.SweepArgs.from_sweep(sw), d["pos"], d["nrm"], d["rad"],
                           d["geom"], d["prm"])
    api.stream_check()
    ref = oracle.rcs_sweep(sc, sw, d["S"], d["eps"], d["eps"], mode="fp32")
    assert int(max((t.M >= 5).sum() for t in ref.traces)) > 100
    assert field_err(_cplx(E), ref.E).max() < 1e-3
    s = sig.cpu().numpy()
    for p in (0, 1):
        sd, so = oracle.db(s[..., p, p]), oracle.db(ref.sigma[..., p, p])
        keep = so >= so.max() - 40.0
        assert np.abs(sd - so)[keep].max() < 0.1


def test_po_field_beyond_one_launch():
    # a plate tiled by 20 x 15 projected screen cells, replicated for 70
    # receiver groups with their own directions; 600 frequencies 2-18 GHz
    api, _ = _mods()
    th = math.radians(20.0)
    w = np.array([math.sin(th), 0, math.cos(th)])
    u = np.array([math.cos(th), 0, -math.sin(th)])
    v = np.array([0, 1.0, 0])
    dd = -w
    nu, nv = 20, 15
    us = (0.1 / nu * math.cos(th)) * u
    vs = (0.075 / nv) * v
    up = us - dd * (us[2] / dd[2])
    vp = vs - dd * (vs[2] / dd[2])
    ii, jj = np.meshgrid(np.arange(nu), np.arange(nv), indexing="ij")
    ps = (ii.ravel()[:, None] - (nu - 1) / 2) * up[None] + \
        (jj.ravel()[:, None] - (nv - 1) / 2) * vp[None]
    f32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    ps = f32(ps + np.array([0.02, -0.01, 0.03]))
    n = ps.shape[0]
    tr = oracle.Trace(M=np.ones(n, np.int32), ids=np.zeros((n, 1), np.int64), p=ps,
                      n=np.tile([0, 0, 1.0], (n, 1)), k=np.tile(f32(dd), (n, 1)),
                      u=np.tile(f32(us), (n, 1)), v=np.tile(f32(vs), (n, 1)),
                      path=ps @ f32(dd), psi=np.ones(n, np.uint8))
    G = 70
    rng = np.random.default_rng(5)
    t = np.radians(rng.uniform(0.0, 60.0, G))
    p = np.radians(rng.uniform(0.0, 360.0, G))
    ks = f32(np.stack([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)], 1))
    freqs = scenes.freq_grid(2e9, 18e9, 600)
    Eo = oracle.po_field(tr, freqs, ks)                          # [G][F][pol][3]
    h = api.alloc_hits(n * G, 1, DEV, ids=False)
    for name in ("p", "n", "k", "u", "v"):
        getattr(h, name).copy_(torch.from_numpy(np.tile(getattr(tr, name), (G, 1)).astype(np.float32)))
    h.path.copy_(torch.from_numpy(np.tile(tr.path, G)))
    h.M.copy_(torch.from_numpy(np.tile(tr.M, G)))
    h.psi.copy_(torch.from_numpy(np.tile(tr.psi, G)))
    E = _cplx(api.po_field(h, G, n, ks, freqs))
    api.stream_check()
    assert E.shape == Eo.shape == (G, 600, 2, 3)
    assert field_err(E, Eo).max() < 1e-3


@pytest.mark.parametrize("G", [1, 7, 64])
def test_small_fusion_grids_bitexact(G):
    # fuse_grid from 1 (every kept pixel in one voxel: a single splat at the
    # target's centroid) to a coarse 64^3; splats and a 2-bounce trace
    # through them bit-exact
    api, pipe = _mods()
    sc = scenes.dihedral(2000, seed=41)
    vd = scenes.aggregation_views(sc, 48, 48)
    pos, nrm, rad = pipe.scene_to_device(sc, DEV)
    gv = pipe.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, vd.W, vd.H)
    prm = pipe.default_params(sc.pos, gv, G=G)
    geom, _ = pipe.build_geometry(pos, nrm, rad, gv, prm)
    api.stream_check()
    ogv = oracle.gfb_views(vd, "fp32")
    ogf = [oracle.gfb(sc, v, "fp32") for v in ogv]
    S = oracle.aggregate(ogf, oracle.fuse_params(sc, G), "fp32")
    cr, nf = geom.planes()
    cr = cr.cpu().numpy()
    nf = nf.cpu().numpy()
    ids = np.flatnonzero(cr[:, 3] > 0)
    assert S.ns >= 1 and (G > 1 or S.ns == 1)
    assert np.array_equal(ids, S.id)
    assert np.array_equal(cr[ids, :3].astype(np.float64), S.c)
    assert np.array_equal(cr[ids, 3].astype(np.float64), S.r)
    assert np.array_equal(nf[ids, :3].astype(np.float64), S.n)
    assert np.array_equal(nf[ids, 3].astype(np.int64), S.count)
    c, r = scenes.bounding_sphere(sc.pos)
    d = dict(sc=sc, pos=pos, nrm=nrm, rad=rad, gv=gv, geom=geom, S=S,
             eps=oracle.default_eps(ogv))
    trs = _trace_vs_oracle(d, [90.0, 70.0], [45.0, 20.0], c, r * 1.02, 32, 32, 2)
    assert sum(int((t.M > 0).sum()) for t in trs) > 100


def test_fusion_of_views_of_different_sizes():
    # the GFBs of a call share one screen size, but a geometry may fuse views
    # of several sizes (per-view pixel offsets and pyramids): four 48 x 48
    # views and four 64 x 40 views, built in two calls and fused in one;
    # splats and a 3-bounce trace through them bit-exact
    api, pipe = _mods()
    sc = scenes.dihedral(2500, seed=43)
    c, r = scenes.bounding_sphere(sc.pos)
    pos, nrm, rad = pipe.scene_to_device(sc, DEV)
    ga = pipe.views_from_angles([60.0] * 4, [45.0, 135.0, 225.0, 315.0], c, r * 1.02, 48, 48)
    gb = pipe.views_from_angles([120.0] * 4, [45.0, 135.0, 225.0, 315.0], c, r * 1.02, 64, 40)
    gv = ga + gb
    prm = pipe.default_params(sc.pos, gv)
    fa = api.build_gfb(ga, pos, nrm, rad, 0, outputs=("nd", "mask"))
    fb = api.build_gfb(gb, pos, nrm, rad, 0, outputs=("nd", "mask"))
    nd = torch.cat([fa["nd"], fb["nd"]])
    mask = torch.cat([fa["mask"], fb["mask"]])
    geom = api.aggregate_views(gv, nd, mask, prm)
    api.stream_check()
    ogv = (_oviews([60.0] * 4, [45.0, 135.0, 225.0, 315.0], c, r * 1.02, 48, 48) +
           _oviews([120.0] * 4, [45.0, 135.0, 225.0, 315.0], c, r * 1.02, 64, 40))
    ogf = [oracle.gfb(sc, v, "fp32") for v in ogv]
    S = oracle.aggregate(ogf, oracle.fuse_params(sc), "fp32")
    cr, nf = geom.planes()
    cr = cr.cpu().numpy()
    nf = nf.cpu().numpy()
    assert cr.shape[0] == 4 * 48 * 48 + 4 * 64 * 40
    ids = np.flatnonzero(cr[:, 3] > 0)
    assert S.ns > 1000 and (S.id >= 4 * 48 * 48).any()       # splats owned by both sizes
    assert np.array_equal(ids, S.id)
    assert np.array_equal(cr[ids, :3].astype(np.float64), S.c)
    assert np.array_equal(cr[ids, 3].astype(np.float64), S.r)
    assert np.array_equal(nf[ids, :3].astype(np.float64), S.n)
    assert np.array_equal(nf[ids, 3].astype(np.int64), S.count)
    d = dict(sc=sc, pos=pos, nrm=nrm, rad=rad, gv=gv, geom=geom, S=S,
             eps=oracle.default_eps(ogv))
    trs = _trace_vs_oracle(d, [90.0, 75.0], [45.0, 58.0], c, r * 1.02, 36, 36, 3)
    assert sum(int((t.M >= 2).sum()) for t in trs) > 100
