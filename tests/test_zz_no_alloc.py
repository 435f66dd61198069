"""The allocation-free PO entry point (pe_po_field_static).

It exists for callers that cannot give the library a workspace: it must give
the same field as pe_po_field (which uses a caller workspace) on the same
hits, on two calls in a row (the fixed scratch array keeps the previous call's
contents, which must not leak into the next result), and it must refuse
requests larger than its fixed scratch before touching the GPU.  This file is
collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def traced():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2408_15583_gb300 import api, pipeline
    sc = scenes.dihedral(3000, seed=17)
    vd = scenes.aggregation_views(sc, 64, 64)
    pos, nrm, rad = pipeline.scene_to_device(sc, DEV)
    gv = pipeline.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, vd.W, vd.H)
    prm = pipeline.default_params(sc.pos, gv)
    geom, _ = pipeline.build_geometry(pos, nrm, rad, gv, prm)
    c, r = scenes.bounding_sphere(sc.pos)
    views = pipeline.views_from_angles([90.0, 80.0, 60.0], [45.0, 20.0, 70.0], c, r * 1.02, 64, 64)
    keys = api.build_gfb(views, pos, nrm, rad, 0, outputs=("keys",))["keys"]
    h = api.trace_bounces(views, keys, nrm, geom, 2, prm, ids=False)
    ks = np.array([[-x for x in v.d] for v in views], np.float32)
    return api, h, ks


def _field_err(E, Eref):
    d = np.sqrt((np.abs(E - Eref) ** 2).sum(axis=-1))
    r = np.sqrt((np.abs(Eref) ** 2).sum(axis=-1))
    return d / np.maximum(r, 1e-3 * r.max())


def _cplx(E):
    E = E.detach().cpu().numpy()
    return E[..., 0] + 1j * E[..., 1]


def _static(api, h, ks, freqs, out):
    from paper_2408_15583_gb300 import _lib
    fr = np.ascontiguousarray(freqs, dtype=np.float64)
    k = np.ascontiguousarray(ks, dtype=np.float32)
    st = _lib.load().pe_po_field_static(C.byref(h.c), k.shape[0], 64 * 64,
                                        k.ctypes.data_as(C.c_void_p), fr.ctypes.data_as(C.c_void_p),
                                        fr.shape[0], C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st, "pe_po_field_static")
    return out


def test_static_po_matches_workspace_po_twice(traced):
    # pe_po_field_static runs the same kernels in the same fixed order as
    # pe_po_field; only where its partial sums live differs, so its field
    # must equal pe_po_field's bit for bit, and a leftover of an earlier
    # call (the array keeps the last call's contents) would show as a
    # difference in the bits
    api, h, ks = traced
    # two different requests back to back: the second must not see the first's scratch
    for freqs in (scenes.freq_grid(2.5e9, 3.5e9, 7), scenes.freq_grid(3.0e9, 3.2e9, 2)):
        ref = api.po_field(h, 3, 64 * 64, ks, freqs).cpu().numpy()
        out = torch.full((3, len(freqs), 2, 3, 2), float("nan"), dtype=torch.float64, device=DEV)
        got = _static(api, h, ks, freqs, out).cpu().numpy()
        api.stream_check()
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, ref)
        assert _field_err(_cplx(torch.from_numpy(got)), _cplx(torch.from_numpy(ref))).max() < 1e-3
    # and the same request twice in a row gives the same field both times
    freqs = scenes.freq_grid(2.9e9, 3.1e9, 5)
    a = _static(api, h, ks, freqs, torch.empty((3, 5, 2, 3, 2), dtype=torch.float64,
                                               device=DEV)).cpu().numpy()
    b = _static(api, h, ks, freqs, torch.empty((3, 5, 2, 3, 2), dtype=torch.float64,
                                               device=DEV)).cpu().numpy()
    ref = api.po_field(h, 3, 64 * 64, ks, freqs).cpu().numpy()
    assert np.array_equal(a, ref) and np.array_equal(b, ref)


def test_static_po_rejects_requests_beyond_its_scratch(traced):
    api, h, ks = traced
    from paper_2408_15583_gb300 import _lib
    lib = _lib.load()
    # 64 groups x 1M rays x 256 frequencies needs far more than 16 MiB of partials
    big = _lib.PeHits()
    big.p = big.n = big.k = big.u = big.v = big.path = big.M = big.psi = h.c.p
    big.n_rays = 64 * (1 << 20)
    ksb = np.zeros((64, 3), np.float32)
    ksb[:, 2] = 1
    fr = np.linspace(8e9, 12e9, 256)
    st = lib.pe_po_field_static(C.byref(big), 64, 1 << 20, ksb.ctypes.data_as(C.c_void_p),
                                fr.ctypes.data_as(C.c_void_p), 256, C.c_void_p(h.c.p), None)
    assert st == 1
    assert b"scratch" in lib.pe_last_error()
