"""The oracle's uniform-grid searches return the brute-force result bit for
bit.

At the workloads' full sizes the oracle draws the candidates of its searches
(Alg. 1's nearest surfel per pixel ray, the nearest splat and Eq. 23's
candidate set per bounce ray, any splat along a shadow ray) from a uniform
grid instead of testing every element; the per-element tests and the rules
that pick among hits are the brute-force ones.  These cases compare the two
on every output the searches feed (GFB depth, index and normal; trace hit
ids, bounce counts, last-hit records, path length, Psi; bistatic Psi), in
both arithmetic modes, on the small scenes of the GPU parity tests (a
dihedral, a sphere, noisy points with PCA normals, the OctAR shape), in tube
mode, with the first bounce from the splats, and on degenerate inputs.  CPU
only.
"""
import numpy as np
import pytest

import oracle
import scenes

SCENES = {
    "dihedral": lambda: scenes.dihedral(3000, seed=12),
    "sphere": lambda: scenes.sphere(3000, 1.0),
    "composite": lambda: scenes.composite(6000, seed=9, pca=True),
    "octar": lambda: scenes.octar(3000, size=2.0, seed=13),
}
ANGLES = [(90.0, 45.0), (60.0, 30.0), (54.7356, 45.0), (75.0, 200.0)]


def _same(a, b, names, tag):
    for n in names:
        assert np.array_equal(getattr(a, n), getattr(b, n)), f"{tag}: {n}"


def grid_equals_brute(name, mode="fp32"):
    """Every search of one small scene, grid against brute force."""
    sc = SCENES[name]()
    vd = scenes.aggregation_views(sc, 64, 64)
    gv = oracle.gfb_views(vd, mode)
    gb = [oracle.gfb(sc, v, mode, accel="brute") for v in gv]
    for k, v in enumerate(gv):
        _same(gb[k], oracle.gfb(sc, v, mode, accel="grid"), ("depth", "idx", "nrm"),
              f"{name} view {k}")
    S = oracle.aggregate(gb, oracle.fuse_params(sc), mode)
    eps = oracle.default_eps(gv)
    c, r = scenes.bounding_sphere(sc.pos)
    multi = 0
    for th, ph in ANGLES:
        v = oracle.view_from_angles(th, ph, c, r * 1.02, 48, 48, mode)
        first = oracle.gfb(sc, v, mode, accel="brute")
        _same(first, oracle.gfb(sc, v, mode, accel="grid"), ("depth", "idx", "nrm"),
              f"{name} screen {th},{ph}")
        for ff in (first, None):
            t1 = oracle.trace(v, S, 4, eps, eps, first=ff, mode=mode, accel="brute")
            t2 = oracle.trace(v, S, 4, eps, eps, first=ff, mode=mode, accel="grid")
            _same(t1, t2, ("M", "ids", "p", "n", "k", "u", "v", "path", "psi"),
                  f"{name} trace {th},{ph} first={'gfb' if ff is not None else 'splats'}")
            multi += int((t1.M >= 2).sum())
        dirs = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.3, 0.4, np.sqrt(0.75)],
                         -np.asarray(v.d)])
        assert np.array_equal(oracle.shadow_dirs(t1, S, dirs, eps, mode, accel="brute"),
                              oracle.shadow_dirs(t1, S, dirs, eps, mode, accel="grid"))
    delta = 2.0 * gv[0].pitch
    _same(oracle.gfb(sc, gv[0], mode, tube=True, delta=delta, accel="brute"),
          oracle.gfb(sc, gv[0], mode, tube=True, delta=delta, accel="grid"), ("depth", "idx"),
          f"{name} tube")
    return multi


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(SCENES))
def test_grid_search_equals_brute_force(name, mode):
    assert grid_equals_brute(name, mode) > 20      # the cases reach the bounce searches


def test_grid_on_degenerate_inputs():
    # no points; a point behind the screen; a NaN point; coincident points
    # of equal depth (the tie goes to the smaller index on both paths)
    v = oracle.view_from_angles(0.0, 0.0, [0, 0, 0], 1.0, 17, 9)
    empty = scenes.Scene(pos=np.zeros((0, 3), np.float32), nrm=np.zeros((0, 3), np.float32),
                         rad=np.zeros(0, np.float32))
    g = oracle.gfb(empty, v, accel="grid")
    assert np.all(g.idx == -1)
    sc = scenes.Scene(pos=np.array([[0.05, -0.02, 0.0], [0.0, 0.0, 5.0], [np.nan, 0, 0],
                                    [0.05, -0.02, 0.0]], np.float32),
                      nrm=np.array([[0, 0, 1], [0, 0, 1], [0, 0, 1], [0, 0, 1]], np.float32),
                      rad=np.array([0.3, 0.5, 0.3, 0.3], np.float32))
    for mode in ("fp32", "fp64"):
        a = oracle.gfb(sc, v, mode, accel="brute")
        b = oracle.gfb(sc, v, mode, accel="grid")
        _same(a, b, ("depth", "idx", "nrm"), mode)
        assert set(np.unique(a.idx)) == {-1, 0}
    # a trace with no splats at all: bounce 1 only, from the GFB
    tr0 = oracle.trace(v, None, 3, 0.01, 0.01, first=a, accel="grid")
    tr1 = oracle.trace(v, None, 3, 0.01, 0.01, first=a, accel="brute")
    _same(tr0, tr1, ("M", "ids", "psi"), "no splats")


def test_auto_uses_the_grid_only_for_large_searches():
    assert oracle._use_grid("auto", 10, 100) == 0
    assert oracle._use_grid("auto", 200_000, 1 << 20) == 1
    assert oracle._use_grid("brute", 200_000, 1 << 20) == 0
    with pytest.raises(ValueError):
        oracle._use_grid("fast", 1, 1)
