"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (the same entry points, angle batches and screens).

The oracle computes every expected value from the seeded inputs alone: its
own views, fusion grid, epsilon and overlap radius, its own 8 GFBs of the
whole point set, its own fusion and its own traces of every ray.  At these
sizes its searches take their candidates from a uniform grid (the same result
as brute force, bit for bit, pinned on the CPU).

* Dihedral workload (10k points, 8 fused views at 512^2, 91 angles at 128^2,
  3 GHz, 2 bounces): every splat bit-exact; for angles spread over both angle
  batches of the sweep (64 + 27), every ray's hit ids, bounce counts and Psi
  bit-exact, the field within 1e-3 and sigma within 0.1 dB of the oracle.
* Sphere workload, the bench's default (200k points, 8 fused views at 512^2,
  360 angles at 1024^2, 64 frequencies 8-12 GHz, 2 bounces): every GFB key
  of the 8 views, every splat, and for 8 angles spread over the sweep every
  ray's records bit-exact; the field of those angles from the 360-angle sweep
  (as bench.py runs it) within 1e-3 of the oracle's field over all rays and
  frequencies, sigma within 0.1 dB, reported per angle; the whole 360 x 64
  sweep within 0.2 dB of the sphere's exact physical-optics backscatter.
* Composite workload (1M noisy points with PCA normals, 8 fused views at
  512^2, 2048^2 rays, 10 GHz, 5 bounces): every splat bit-exact; two angles,
  every ray's records bit-exact, field and sigma, reported per angle.

Run with `-s` to see the per-angle table.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
C0 = 299792458.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _mods():
    from paper_2408_15583_gb300 import api, pipeline
    return api, pipeline


def _pool():
    import os
    return ThreadPoolExecutor(max(2, min(16, os.cpu_count() or 2)))


def _cplx(E):
    E = E.detach().cpu().numpy()
    return E[..., 0] + 1j * E[..., 1]


def _field_err(E, Eref):
    d = np.sqrt((np.abs(E - Eref) ** 2).sum(axis=-1))
    r = np.sqrt((np.abs(Eref) ** 2).sum(axis=-1))
    return d / np.maximum(r, 1e-3 * r.max())


def _sigma_err_db(sig, ref, peak_db=40.0):
    """|delta sigma| in dB over the co-polarised samples within peak_db of
    the reference's peak (c24)."""
    worst = 0.0
    for p in (0, 1):
        sd, so = oracle.db(sig[..., p, p]), oracle.db(ref[..., p, p])
        keep = so >= so.max() - peak_db
        worst = max(worst, float(np.abs(sd - so)[keep].max()))
    return worst


def _gpu_geometry(wl):
    api, pipe = _mods()
    sc, vd = wl.scene, wl.views
    pos, nrm, rad = pipe.scene_to_device(sc, DEV)
    gv = pipe.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, vd.W, vd.H)
    prm = pipe.default_params(sc.pos, gv)
    geom, _ = pipe.build_geometry(pos, nrm, rad, gv, prm)
    api.stream_check()
    return pos, nrm, rad, gv, prm, geom


def _oracle_geometry(wl):
    """The oracle's fused splats from its own 8 GFBs (every pixel), its own
    fusion grid, and its epsilon = overlap radius."""
    S, ogv, ogf, fp = oracle.build_geometry(wl.scene, wl.views, "fp32")
    return S, ogv, ogf, oracle.default_eps(ogv)


def _splats_equal(geom, S):
    cr, nf = geom.planes()
    cr = cr.cpu().numpy()
    nf = nf.cpu().numpy()
    ids = np.flatnonzero(cr[:, 3] > 0)
    assert np.array_equal(ids, S.id)
    assert np.array_equal(cr[ids, :3].astype(np.float64), S.c)
    assert np.array_equal(cr[ids, 3].astype(np.float64), S.r)
    assert np.array_equal(nf[ids, :3].astype(np.float64), S.n)
    assert np.array_equal(nf[ids, 3].astype(np.int64), S.count)


def _records_equal(h, sl, tr, tag):
    """Every record of one angle's rays bit-exact (path length to 1e-13)."""
    assert np.array_equal(h.M[sl].cpu().numpy(), tr.M), tag
    ids = h.ids[:, sl].cpu().numpy().view(np.uint32).astype(np.int64)
    ids[ids == 0xFFFFFFFF] = -1
    assert np.array_equal(ids.T, tr.ids), tag
    assert np.array_equal(h.psi[sl].cpu().numpy(), tr.psi), tag
    live = tr.M > 0
    for name in ("p", "n", "k", "u", "v"):
        got = getattr(h, name)[sl].cpu().numpy().astype(np.float64)
        assert np.array_equal(got[live], getattr(tr, name)[live]), f"{tag}: {name}"
    assert np.allclose(h.path[sl].cpu().numpy()[live], tr.path[live], rtol=1e-13, atol=1e-13), tag


def _sweep_parity(wl, d, angles, label):
    """Trace `angles` of the workload's sweep as one batch through the ABI
    and compare every ray with the oracle's trace of that angle; compare the
    sweep's field and sigma at those angles (d["E"], d["sig"]: the whole
    sweep as bench.py runs it) with the oracle's over every ray.  Prints and
    returns the per-angle errors."""
    api, pipe = _mods()
    sc, sw = wl.scene, wl.sweep
    views = [api.view_from_angles(sw.theta_deg[a], sw.phi_deg[a], sw.centre, sw.extent,
                                  sw.W, sw.H) for a in angles]
    keys = api.build_gfb(views, d["pos"], d["nrm"], d["rad"], 0, outputs=("keys",))["keys"]
    h = api.trace_bounces(views, keys, d["nrm"], d["geom"], sw.max_bounces, d["prm"])
    api.stream_check()
    Eg = _cplx(d["E"])
    sg = d["sig"].cpu().numpy()
    per = sw.W * sw.H
    rows = []
    for k, a in enumerate(angles):
        ref = oracle.rcs_sweep(sc, sw, d["S"], d["eps"], d["eps"], mode="fp32", angles=[a])
        tr = ref.traces[0]
        _records_equal(h, slice(k * per, (k + 1) * per), tr, f"{label} angle {a}")
        fe = float(_field_err(Eg[a:a + 1], ref.E).max())
        de = _sigma_err_db(sg[a:a + 1], ref.sigma)
        rows.append(dict(angle=a, theta=float(sw.theta_deg[a]), phi=float(sw.phi_deg[a]),
                         hits=int((tr.M > 0).sum()), multi=int((tr.M >= 2).sum()),
                         field_err=fe, dsigma_db=de))
        del ref, tr
    print(f"\n{label}: per-angle parity against the oracle (every ray, "
          f"{sw.n_freq} frequencies, 2 polarisations)")
    print("  angle  theta    phi     hits  M>=2  max field err (c24)  max |d sigma| dB")
    for r in rows:
        print(f"  {r['angle']:5d} {r['theta']:6.1f} {r['phi']:6.1f} {r['hits']:8d} {r['multi']:5d}"
              f"  {r['field_err']:19.3e}  {r['dsigma_db']:16.3e}")
    for r in rows:
        assert r["field_err"] < 1e-3, r
        assert r["dsigma_db"] < 0.1, r
    return rows


# ----------------------------------------------------------------------------
# dihedral workload, complete
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def dihedral_full():
    api, pipe = _mods()
    wl = scenes.workload_dihedral()
    sc, sw = wl.scene, wl.sweep
    pos, nrm, rad, gv, prm, geom = _gpu_geometry(wl)
    args = api.SweepArgs.from_sweep(sw)
    E, sig = api.rcs_sweep(args, pos, nrm, rad, geom, prm)
    api.stream_check()
    S, ogv, ogf, eps = _oracle_geometry(wl)
    return dict(wl=wl, pos=pos, nrm=nrm, rad=rad, prm=prm, geom=geom, E=E, sig=sig, S=S,
                eps=eps, args=args)


def test_dihedral_full_splats_bitexact(dihedral_full):
    assert dihedral_full["S"].ns > 50_000
    _splats_equal(dihedral_full["geom"], dihedral_full["S"])


def test_dihedral_full_sweep_and_traces(dihedral_full):
    d = dihedral_full
    assert d["args"].c.angle_batch == 0          # the library picks the batch, as in bench.py
    # angles of both angle batches (0..63, 64..90), the batch edges included
    rows = _sweep_parity(d["wl"], d, [0, 1, 22, 45, 63, 64, 65, 90], "dihedral")
    assert sum(r["multi"] for r in rows) > 1000   # the dihedral's double bounces


# ----------------------------------------------------------------------------
# sphere workload (the default bench workload)
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def sphere_full():
    api, pipe = _mods()
    wl = scenes.workload_sphere()
    pos, nrm, rad, gv, prm, geom = _gpu_geometry(wl)
    E, sig = api.rcs_sweep(api.SweepArgs.from_sweep(wl.sweep), pos, nrm, rad, geom, prm)
    api.stream_check()
    S, ogv, ogf, eps = _oracle_geometry(wl)
    return dict(wl=wl, pos=pos, nrm=nrm, rad=rad, gv=gv, prm=prm, geom=geom, E=E, sig=sig,
                S=S, ogv=ogv, ogf=ogf, eps=eps)


def test_sphere_full_gfb_keys_and_splats_bitexact(sphere_full):
    # the 8 fused views at 512^2, all in one launch as the bench builds
    # them: every pixel's key, then every splat of the fusion
    api, pipe = _mods()
    d = sphere_full
    kg = api.build_gfb(d["gv"], d["pos"], d["nrm"], d["rad"], 0, outputs=("keys",))["keys"]
    api.stream_check()
    kk = kg.cpu().numpy().view(np.uint64).reshape(len(d["ogf"]), -1)
    for v, g in enumerate(d["ogf"]):
        assert np.array_equal(kk[v], g.keys()), f"view {v}"
    assert d["S"].ns > 200_000
    _splats_equal(d["geom"], d["S"])


def test_sphere_full_sweep_parity_per_angle(sphere_full):
    # 8 angles spread over the 360-angle sweep (several of the library's
    # angle batches): every one of the 1024^2 rays per angle, 64 frequencies
    rows = _sweep_parity(sphere_full["wl"], sphere_full, [0, 7, 45, 90, 133, 180, 271, 359],
                         "sphere")
    assert all(r["hits"] > 600_000 for r in rows)


def test_sphere_full_sweep_vs_exact_po(sphere_full):
    # exact PO backscatter of a PEC sphere of radius a:
    # sigma = 4 pi k^2 a^4 |e^{jb}/(jb) + (e^{jb} - 1)/b^2|^2, b = 2 k a
    d = sphere_full
    sw = d["wl"].sweep
    s = d["sig"].cpu().numpy()
    assert s.shape[:2] == (360, 64)
    a = 1.0
    k = 2 * math.pi * np.asarray(sw.freqs_hz) / C0
    b = 2 * k * a
    ref = 4 * math.pi * k ** 2 * a ** 4 * np.abs(np.exp(1j * b) / (1j * b) +
                                                 (np.exp(1j * b) - 1) / b ** 2) ** 2
    for p in (0, 1):
        err = np.abs(oracle.db(s[:, :, p, p]) - oracle.db(ref)[None, :])
        assert err.max() < 0.2, f"pol {p}: {err.max():.3f} dB"
    # the cross-polarised return of a sphere vanishes (up to the surfel
    # sampling): 20 dB below the co-polarised one
    assert np.all(s[:, :, 0, 1] < 1e-2 * s[:, :, 0, 0])


# ----------------------------------------------------------------------------
# composite workload: noisy points, PCA normals, 5 bounces
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def composite_full():
    api, pipe = _mods()
    wl = scenes.workload_composite()
    pos, nrm, rad, gv, prm, geom = _gpu_geometry(wl)
    E, sig = api.rcs_sweep(api.SweepArgs.from_sweep(wl.sweep), pos, nrm, rad, geom, prm)
    api.stream_check()
    S, ogv, ogf, eps = _oracle_geometry(wl)
    return dict(wl=wl, pos=pos, nrm=nrm, rad=rad, gv=gv, prm=prm, geom=geom, E=E, sig=sig,
                S=S, eps=eps)


def test_composite_full_splats_bitexact(composite_full):
    assert composite_full["S"].ns > 40_000
    _splats_equal(composite_full["geom"], composite_full["S"])


def test_composite_full_traces_mb5_per_angle(composite_full):
    # two angles of the 72-angle sweep, every one of the 2048^2 rays, up to
    # five bounces through splats fused from PCA normals of noisy points
    rows = _sweep_parity(composite_full["wl"], composite_full, [0, 9], "composite")
    assert sum(r["multi"] for r in rows) > 100_000
