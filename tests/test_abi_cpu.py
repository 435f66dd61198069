"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every symbol the header declares, computes views exactly as
the oracle does, sizes workspaces, and rejects bad arguments before touching
the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pointemray.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2408_15583_gb300 import _lib
    from paper_2408_15583_gb300.build import build
    build()
    return _lib.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pe_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pe_build_gfb", "pe_aggregate_views", "pe_trace_bounces", "pe_po_field",
                     "pe_rcs_sweep", "pe_stream_check", "pe_last_error", "pe_abi_version"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2408_15583_gb300 import _lib
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks {name}"
    assert lib.pe_abi_version() == 1


def test_view_setup_matches_oracle_bitwise(lib):
    from paper_2408_15583_gb300 import api
    rng = np.random.default_rng(3)
    for _ in range(500):
        th, ph = float(rng.uniform(0, 180)), float(rng.uniform(-360, 360))
        c = rng.normal(size=3) * 3
        ext = float(rng.uniform(0.05, 30))
        W = int(rng.integers(1, 4097))
        v = api.view_from_angles(th, ph, c, ext, W, W)
        o = oracle.view_from_angles(th, ph, c, ext, W, W, "fp32")
        a = np.array(list(v.o) + list(v.u) + list(v.v) + list(v.d) + [v.pitch], np.float32)
        b = np.array(list(o.o) + list(o.u) + list(o.v) + list(o.d) + [o.pitch], np.float32)
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_sweep_workspace_two_lanes(lib):
    # A sweep of several batches with at least 8 frequencies holds two sets
    # of batch buffers (its field sums run beside the next batch's trace);
    # one frequency, or a single batch, holds one.
    from paper_2408_15583_gb300 import api
    import numpy as np

    def ws(n_angles, n_freq):
        args = api.SweepArgs(np.full(n_angles, 90.0), np.linspace(0, 359, n_angles), 1024, 1024,
                             [0.0, 0.0, 0.0], 1.0, np.linspace(8e9, 12e9, n_freq), 2)
        return args.workspace_bytes()

    per_angle = 1024 * 1024 * (8 + 60 + 8 + 4 + 1)      # keys and ray records
    one = ws(360, 1)
    two = ws(360, 64)
    assert 64 * per_angle <= one < 2 * 64 * per_angle
    assert two >= 2 * 64 * per_angle                     # two sets of 64-angle batches
    assert ws(10, 64) < 11 * per_angle + (1 << 30)       # one batch of 10 angles, one set
    assert ws(0, 64) == 0


def test_sweep_point_order_checked_before_the_call(lib):
    # The library reads one order entry per point through a raw pointer, so
    # the binding refuses an order of the wrong type, size or layout before
    # it calls anything.
    from paper_2408_15583_gb300 import api
    import numpy as np
    import torch

    args = api.SweepArgs(np.full(4, 90.0), np.linspace(0, 90, 4), 64, 64, [0.0, 0.0, 0.0], 1.0,
                         np.linspace(8e9, 12e9, 8), 2)
    pos = torch.zeros(10, 3)
    for bad in (torch.arange(9, dtype=torch.int32),              # too short
                torch.arange(10, dtype=torch.int64),             # wrong type
                torch.arange(20, dtype=torch.int32)[::2]):       # not contiguous
        args.set_point_order(bad)
        with pytest.raises(ValueError, match="point order"):
            api.rcs_sweep(args, pos, pos, pos[:, 0], None, api.PeParams())
        with pytest.raises(ValueError, match="order_points"):
            api.order_points(pos, out=bad)


def test_outputs_checked_before_the_call(lib):
    # Outputs the library writes through raw pointers: the binding refuses a
    # wrong type, size or layout before any call.
    from paper_2408_15583_gb300 import api
    import numpy as np
    import torch

    h = api.alloc_hits(16, 1, "cpu", ids=False)
    ks = np.array([[0.0, 0.0, 1.0]], np.float32)
    fr = np.array([8e9, 9e9])
    for bad in (torch.empty(1, 2, 2, 3, 2, dtype=torch.float32),      # wrong type
                torch.empty(1, 3, 2, 3, 2, dtype=torch.float64)):     # wrong size
        with pytest.raises(ValueError, match="po_field: out"):
            api.po_field(h, 1, 16, ks, fr, out=bad)
    args = api.SweepArgs(np.full(4, 90.0), np.linspace(0, 90, 4), 64, 64, [0.0, 0.0, 0.0], 1.0,
                         fr, 2)
    pos = torch.zeros(10, 3)
    with pytest.raises(ValueError, match="rcs_sweep: E"):
        api.rcs_sweep(args, pos, pos, pos[:, 0], None, api.PeParams(),
                      E=torch.empty(4, 2, 2, 3, 2, dtype=torch.float64)[:, ::2])
    with pytest.raises(ValueError, match="rcs_sweep: sigma"):
        api.rcs_sweep(args, pos, pos, pos[:, 0], None, api.PeParams(),
                      sigma=torch.empty(4, 2, 2, dtype=torch.float64))


def test_workspace_queries(lib):
    from paper_2408_15583_gb300 import api
    vs = [api.view_from_angles(60, 45 + 90 * i, [0, 0, 0], 1.0, 512, 512) for i in range(8)]
    arr = api.views_to_array(vs)
    assert lib.pe_build_gfb_workspace(8, arr) >= 8 * 512 * 512 * 8
    g = lib.pe_geom_bytes(8, arr)
    assert g >= 8 * 512 * 512 * 32
    assert lib.pe_aggregate_workspace(8, arr, 256) >= 256 ** 3 * 8
    assert lib.pe_aggregate_workspace(8, arr, 257) == 0
    assert lib.pe_trace_workspace(8, arr) > 0
    assert lib.pe_trace_workspace(0, arr) == 0
    assert lib.pe_po_workspace(4, 1 << 20, 64) > 0
    assert lib.pe_po_workspace(0, 1 << 20, 64) == 0
    sw = api.SweepArgs([90.0] * 3, [0.0, 1.0, 2.0], 1024, 1024, [0, 0, 0], 1.1,
                       np.linspace(8e9, 12e9, 64), 2)
    assert sw.workspace_bytes() > 3 * 1024 * 1024 * 80
    bad = api.SweepArgs([90.0], [0.0], 1024, 1024, [0, 0, 0], -1.0, [1e9], 2)
    assert bad.workspace_bytes() == 0
    # PO at every bounce: hit records of every ray, a second Psi, the
    # per-bounce field and the PO partial sums
    eb = lib.pe_po_field_every_bounce_workspace(8, arr, 64)
    assert eb >= 8 * 512 * 512 * (60 + 8 + 4 + 1 + 1) + 8 * 64 * 12 * 8
    assert lib.pe_po_field_every_bounce_workspace(0, arr, 64) == 0
    assert lib.pe_po_field_every_bounce_workspace(8, arr, 0) == 0


def test_argument_errors_before_any_device_work(lib):
    from paper_2408_15583_gb300 import api
    v = api.views_to_array([api.view_from_angles(0, 0, [0, 0, 0], 1.0, 8, 8)])
    # zero views, too many views, bad mode: rejected synchronously
    assert lib.pe_build_gfb(v, 0, None, None, None, 0, 0, 0.0, None, 0, None, None, None,
                            None, None) == 1
    assert lib.pe_build_gfb(v, 65, None, None, None, 0, 0, 0.0, None, 0, None, None, None,
                            None, None) == 1
    assert lib.pe_build_gfb(v, 1, None, None, None, 0, 7, 0.0, None, 0, None, None, None,
                            None, None) == 1
    assert b"mode" in lib.pe_last_error()
    # workspace too small
    assert lib.pe_build_gfb(v, 1, None, None, None, 0, 0, 0.0, None, 0, None, None, None,
                            None, None) == 2
    assert lib.pe_view_from_angles(0.0, 0.0, None, 1.0, 8, 8, None) == 1
    # the batched entry points take one screen size per call
    mixed = api.views_to_array([api.view_from_angles(0, 0, [0, 0, 0], 1.0, 8, 8),
                                api.view_from_angles(0, 0, [0, 0, 0], 1.0, 8, 6)])
    assert lib.pe_build_gfb(mixed, 2, None, None, None, 0, 0, 0.0, None, 0, None, None, None,
                            None, None) == 1
    assert b"W x H" in lib.pe_last_error()
    assert lib.pe_build_gfb_topk(mixed, 2, None, 0, 0.1, 4, None, 0, None, None) == 1
    assert b"W x H" in lib.pe_last_error()
    prm, hits = api.PeParams(), api.PeHits()
    assert lib.pe_trace_bounces(mixed, 2, None, None, None, 1, C.byref(prm), None, 0,
                                C.byref(hits), None, None) == 1
    assert b"W x H" in lib.pe_last_error()
    assert lib.pe_trace_bounces(v, 1, None, None, None, 0, None, None, 0, None, None, None) == 1
    assert lib.pe_po_field(None, 1, 1, None, None, 1, None, 0, None, None) == 1
    fr = (C.c_double * 1)(3e9)
    assert lib.pe_po_field_every_bounce(mixed, 2, None, None, None, 2, C.byref(prm), fr, 1,
                                        None, 0, None, None) == 1
    assert lib.pe_nn_set_wait_limit(1 << 33) == 1


def test_probe_arguments_rejected_before_any_device_work(lib):
    assert lib.pe_probe_units(6, 1, 1, None, 0, None) == -1
    assert b"kind" in lib.pe_last_error()
    assert lib.pe_probe_units(0, 0, 1, None, 0, None) == -1
    assert lib.pe_probe_units(0, 1, 0, None, 0, None) == -1
    assert lib.pe_probe_units(3, 1, 1, None, 1 << 20, None) == -1
    assert b"scratch" in lib.pe_last_error()


def test_view_from_struct_round_trips_a_library_view(lib):
    from paper_2408_15583_gb300 import api
    a = api.view_from_angles(63.0, 211.0, [0.1, -0.2, 0.3], 1.7, 96, 64)
    b = api.view_from_struct(a.o, a.u, a.v, a.d, a.pitch, a.W, a.H)
    assert bytes(a) == bytes(b)


@pytest.mark.parametrize("G,tau", [(256, 3.0), (7, 2.5), (1, 3.0)])
def test_parameters_equal_the_oracles(lib, G, tau):
    # the library's fusion grid, epsilon and overlap radius (pipeline
    # default_params over api.make_params) are the oracle's (fuse_params,
    # default_eps from its own views), bit for bit as FP32 values; the GPU
    # parity tests build every oracle input on the oracle's side, so this
    # is where the two parameter paths meet
    import scenes
    from paper_2408_15583_gb300 import pipeline
    f32 = lambda x: np.float32(x).view(np.uint32)
    for sc in (scenes.dihedral(2000, seed=31), scenes.sphere(3000, 1.0),
               scenes.octar(3000, size=2.0, seed=13), scenes.plate(0.3, 0.2, 30, 20),
               scenes.Scene(pos=np.array([[0.01, -0.02, 0.03], [0.06, 0.01, -0.02]], np.float32),
                            nrm=np.array([[0.0, 0.6, 0.8], [0.8, 0.0, 0.6]], np.float32),
                            rad=np.array([0.05, 0.04], np.float32))):
        for W, H in ((80, 80), (64, 40)):
            vd = scenes.aggregation_views(sc, W, H)
            gv = pipeline.views_from_angles(vd.theta_deg, vd.phi_deg, vd.centre, vd.extent, W, H)
            prm = pipeline.default_params(sc.pos, gv, G=G, tau=tau)
            fp = oracle.fuse_params(sc, G, tau)
            eps = oracle.default_eps(oracle.gfb_views(vd, "fp32"))
            assert prm.fuse_grid == fp.G
            assert f32(prm.edge_tau) == f32(fp.tau)
            assert f32(prm.inv_voxel) == f32(fp.inv_vox)
            for k in range(3):
                assert f32(prm.bbox_min[k]) == f32(fp.bmin[k])
            assert f32(prm.eps) == f32(eps) and f32(prm.overlap_r) == f32(eps)
            assert prm.edge_mode == fp.edge_mode == 0
