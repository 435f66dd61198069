"""Alg. 1 with a finite heap of K points per ray tube (pe_build_gfb_topk)
against the oracle's brute-force statement of it: keys bit-exact for K from
1 to 64 on sparse clouds shaped like the learned part's inputs, on a
dihedral and at the ragged edge of the screen; a large K equals the default
tube mode (the unbounded heap)."""
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


def _ov(v):
    return oracle.View(o=np.array(v.o[:], np.float64), u=np.array(v.u[:], np.float64),
                       v=np.array(v.v[:], np.float64), d=np.array(v.d[:], np.float64),
                       pitch=float(v.pitch), W=v.W, H=v.H)


def _case(name):
    from paper_2408_15583_gb300 import pipeline
    if name == "sparse_primitives":
        sc = scenes.random_primitives(3, 1.0, bbox_lambdas=6.4)
        W, H = 64, 64
    else:
        sc = scenes.dihedral(1500, seed=4)
        W, H = 45, 37                       # ragged: not a multiple of anything
    c, r = scenes.bounding_sphere(sc.pos)
    views = pipeline.views_from_angles([60.0, 120.0, 90.0], [45.0, 200.0, 10.0], c, r * 1.02, W, H)
    return sc, views


@pytest.mark.parametrize("name", ["sparse_primitives", "dihedral"])
@pytest.mark.parametrize("K", [1, 2, 4, 8, 16, 64])
def test_topk_keys_bitexact(name, K):
    from paper_2408_15583_gb300 import api
    sc, views = _case(name)
    pos = torch.from_numpy(sc.pos).to(DEV)
    delta = float(np.float32(2.0 * views[0].pitch))
    keys = api.build_gfb_topk(views, pos, delta, K).cpu().numpy().view(np.uint64)
    api.stream_check()
    per = views[0].W * views[0].H
    hits = 0
    for a, v in enumerate(views):
        g = oracle.gfb_topk(sc.pos, _ov(v), delta, K, "fp32")
        assert np.array_equal(keys[a * per:(a + 1) * per], g.keys()), f"view {a}"
        hits += int((g.idx >= 0).sum())
    assert hits > 0.2 * per


def test_large_k_is_the_default_tube_mode():
    from paper_2408_15583_gb300 import api
    # a tube of one pixel's radius: every pixel has fewer than 64 candidates
    sc, views = _case("sparse_primitives")
    pos = torch.from_numpy(sc.pos).to(DEV)
    delta = float(np.float32(1.0 * views[0].pitch))
    k64 = api.build_gfb_topk(views, pos, delta, 64)
    kinf = api.build_gfb(views, pos, None, None, 1, delta, outputs=("keys",))["keys"]
    api.stream_check()
    assert torch.equal(k64, kinf)
    k1 = api.build_gfb_topk(views, pos, delta, 1)
    hit = kinf != -1
    assert torch.equal(k1 != -1, hit)           # same pixels have a candidate
    assert bool((k1[hit] != kinf[hit]).any())   # K = 1 picks other points somewhere
