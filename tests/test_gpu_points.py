"""Surfel attributes on the GPU (pe_point_attributes) against the brute-force
oracle: radii bit-exact (same neighbour lists: FP32 squared distances in one
order, ties by index; FP64 sums in list order), PCA normals within 1e-6 rad
wherever the normal is well defined (the two smallest covariance eigenvalues
apart by at least 10 % of the middle one), orientation exact where the
reference is not near perpendicular.  At the composite workload's full size
(1M points) a sample of points is checked one by one."""

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


def _gpu(pos, k_r, k_n, ref=None):
    from paper_2408_15583_gb300 import api
    p = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).to(DEV)
    rf = None if ref is None else torch.from_numpy(np.ascontiguousarray(ref, np.float32)).to(DEV)
    r, n = api.point_attributes(p, k_r, k_n, rf)
    api.stream_check()
    return r.cpu().numpy(), n.cpu().numpy()


def _clouds():
    rng = np.random.default_rng(7)
    line = np.zeros((400, 3), np.float32)
    line[:, 0] = np.sort(rng.random(400)).astype(np.float32)          # collinear
    dup = np.concatenate([rng.random((300, 3)), rng.random((300, 3))[:100]])
    dup = np.concatenate([dup, dup[:60]]).astype(np.float32)           # exact duplicates
    return {
        "sphere": (scenes.sphere(6000, 1.0).pos, scenes.sphere(6000, 1.0).nrm),
        "octar": (scenes.octar(6000, 2.0, seed=3).pos, scenes.octar(6000, 2.0, seed=3).nrm),
        "noisy_composite": (scenes.composite(8000, seed=3, pca=False).pos,
                            scenes.composite(8000, seed=3, pca=False).nrm),
        "uniform": (rng.random((3000, 3)).astype(np.float32), None),
        "line": (line, None),
        "duplicates": (dup, None),
        "minimal": (rng.random((17, 3)).astype(np.float32), None),
    }


@pytest.mark.parametrize("name", list(_clouds().keys()))
def test_radius_bitexact_and_normals_vs_oracle(name):
    pos, ref = _clouds()[name]
    _check(pos, ref, 8, 16, name != "line")


@pytest.mark.parametrize("k_r,k_n", [(31, 32), (1, 3), (31, 3), (1, 32)])
@pytest.mark.parametrize("cloud", ["octar", "uniform", "exactly_k"])
def test_neighbour_count_limits(k_r, k_n, cloud):
    # the smallest and largest neighbour counts the ABI accepts, and a cloud
    # of exactly max(k_r + 1, k_n) points (every list is the whole cloud)
    rng = np.random.default_rng(k_r * 100 + k_n)
    if cloud == "exactly_k":
        pos, ref = rng.random((max(k_r + 1, k_n), 3)).astype(np.float32), None
    else:
        pos, ref = _clouds()[cloud]
    _check(pos, ref, k_r, k_n, cloud != "exactly_k" and k_n > 3)


def _check(pos, ref, k_r, k_n, most_defined):
    r, n = _gpu(pos, k_r, k_n, ref)
    ro, no, w, _ = oracle.point_attributes(pos, k_r, k_n, ref=ref)
    assert np.array_equal(r, ro), f"{np.flatnonzero(r != ro)[:10]}"
    good = (w[:, 1] - w[:, 0]) > 0.1 * np.maximum(w[:, 1], 1e-300)
    if most_defined:
        assert good.mean() > 0.5
    # angle from atan2(|a x b|, |a . b|): acos of a dot product near 1 would
    # turn the FP32 rounding of the output into ~1e-4 rad
    n64 = n.astype(np.float64)
    ang = np.arctan2(np.linalg.norm(np.cross(n64, no), axis=1), np.abs((n64 * no).sum(1)))
    assert ang[good].max(initial=0.0) < 1e-6
    # orientation: the same side wherever the reference direction decides it
    if ref is not None:
        firm = good & (np.abs((no * ref).sum(1)) > 1e-3)
    else:
        lo, hi = pos.astype(np.float64).min(0), pos.astype(np.float64).max(0)
        firm = good & (np.abs((no * (pos - 0.5 * (lo + hi))).sum(1)) > 1e-3)
    assert np.all((n.astype(np.float64) * no).sum(1)[firm] > 0)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)


def test_full_size_sampled():
    # the composite workload's 1M noisy points; 2000 sampled points checked
    # against brute force over the whole cloud
    sc = scenes.composite(1_000_000, pca=False)
    pos = sc.pos
    r, _ = _gpu(pos, 8, 16, sc.nrm)
    q = np.random.default_rng(11).choice(pos.shape[0], 2000, replace=False)
    idx, d2 = oracle.knn(pos, 9, queries=q)
    assert np.array_equal(r[q], oracle.knn_radius(idx, d2, q, 8))


def test_argument_errors():
    from paper_2408_15583_gb300 import api
    p = torch.zeros(10, 3, device=DEV)
    with pytest.raises(RuntimeError):
        api.point_attributes(p, 8, 16)            # fewer points than neighbours
    with pytest.raises(RuntimeError):
        api.point_attributes(torch.zeros(100, 3, device=DEV), 8, 40)   # k_n > 32
