"""ctypes declarations of the C ABI in ``include/pointemray.h``.

Loading fails loudly when the compiled library is missing: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpointemray.so")

PE_MAX_VIEWS = 16
PE_MAX_BATCH = 64
PE_STATS_WORDS = 8

STATUS = {0: "PE_OK", 1: "PE_EINVAL", 2: "PE_ENOMEM", 3: "PE_ECUDA", 4: "PE_ETIMEOUT",
          5: "PE_EOVERFLOW", 6: "PE_EUNSUPPORTED"}


class PeView(C.Structure):
    _fields_ = [("o", C.c_float * 3), ("u", C.c_float * 3), ("v", C.c_float * 3),
                ("d", C.c_float * 3), ("pitch", C.c_float), ("W", C.c_int32), ("H", C.c_int32)]


class PeParams(C.Structure):
    _fields_ = [("delta", C.c_float), ("eps", C.c_float), ("overlap_r", C.c_float),
                ("edge_tau", C.c_float), ("fuse_grid", C.c_int32), ("bbox_min", C.c_float * 3),
                ("inv_voxel", C.c_float), ("first_bounce_from_geom", C.c_int32),
                ("edge_mode", C.c_int32)]


class PeGeom(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("views", PeView * PE_MAX_VIEWS),
                ("blob_dev", C.c_void_p), ("blob_bytes", C.c_size_t),
                ("vgrid_min", C.c_float * 3), ("vgrid_cell", C.c_float), ("vgrid_n", C.c_int32)]


class PeHits(C.Structure):
    _fields_ = [("p", C.c_void_p), ("n", C.c_void_p), ("k", C.c_void_p), ("u", C.c_void_p),
                ("v", C.c_void_p), ("path", C.c_void_p), ("M", C.c_void_p), ("psi", C.c_void_p),
                ("ids", C.c_void_p), ("n_rays", C.c_int64), ("max_bounces", C.c_int32)]


class PeSweep(C.Structure):
    _fields_ = [("n_angles", C.c_int32), ("theta_deg", C.c_void_p), ("phi_deg", C.c_void_p),
                ("W", C.c_int32), ("H", C.c_int32), ("centre", C.c_double * 3),
                ("extent", C.c_double), ("n_freq", C.c_int32), ("freqs_hz", C.c_void_p),
                ("max_bounces", C.c_int32), ("angle_batch", C.c_int32),
                ("point_order", C.c_void_p)]


# name -> (restype, argtypes)
P = C.c_void_p
SIGNATURES = {
    "pe_abi_version": (C.c_int, []),
    "pe_probe_units": (C.c_int64, [C.c_int32, C.c_int32, C.c_int32, P, C.c_size_t, P]),
    "pe_kernel_launches": (C.c_int64, []),
    "pe_set_kernel_events": (C.c_int32, [C.c_char_p, P, C.c_int32]),
    "pe_last_error": (C.c_char_p, []),
    "pe_stream_check": (C.c_int, [P]),
    "pe_view_from_angles": (C.c_int, [C.c_double, C.c_double, P, C.c_double, C.c_int32,
                                      C.c_int32, P]),
    "pe_build_gfb_workspace": (C.c_size_t, [C.c_int32, P]),
    "pe_build_gfb": (C.c_int, [P, C.c_int32, P, P, P, C.c_int64, C.c_int32, C.c_float, P,
                               C.c_size_t, P, P, P, P, P]),
    "pe_geom_bytes": (C.c_size_t, [C.c_int32, P]),
    "pe_aggregate_workspace": (C.c_size_t, [C.c_int32, P, C.c_int32]),
    "pe_aggregate_views": (C.c_int, [P, C.c_int32, P, P, P, P, C.c_size_t, P, P]),
    "pe_trace_workspace": (C.c_size_t, [C.c_int32, P]),
    "pe_trace_bounces": (C.c_int, [P, C.c_int32, P, P, P, C.c_int32, P, P, C.c_size_t, P, P,
                                   P]),
    "pe_po_workspace": (C.c_size_t, [C.c_int32, C.c_int64, C.c_int32]),
    "pe_po_field": (C.c_int, [P, C.c_int32, C.c_int64, P, P, C.c_int32, P, C.c_size_t, P, P]),
    "pe_po_field_static": (C.c_int, [P, C.c_int32, C.c_int64, P, P, C.c_int32, P, P]),
    "pe_rcs_sweep_workspace": (C.c_size_t, [P]),
    "pe_rcs_sweep": (C.c_int, [P, P, P, P, C.c_int64, P, P, P, C.c_size_t, P, P, P, P]),
    # a8
    "pe_nn_gemm_workspace": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int64]),
    "pe_nn_gemm_path": (C.c_int32, [C.c_int32]),
    "pe_nn_set_wait_limit": (C.c_int, [C.c_int64]),
    "pe_point_attributes_workspace": (C.c_size_t, [C.c_int64]),
    "pe_order_points_workspace": (C.c_size_t, [C.c_int64]),
    "pe_order_points": (C.c_int, [P, C.c_int64, P, C.c_size_t, P, P]),
    "pe_po_field_bistatic_workspace": (C.c_size_t, [C.c_int32, C.c_int64, C.c_int32]),
    "pe_po_field_every_bounce_workspace": (C.c_size_t, [C.c_int32, P, C.c_int32]),
    "pe_po_field_every_bounce": (C.c_int, [P, C.c_int32, P, P, P, C.c_int32, P, P, C.c_int32, P,
                                           C.c_size_t, P, P]),
    "pe_po_field_bistatic": (C.c_int, [P, C.c_int32, C.c_int64, P, C.c_int32, P, C.c_float,
                                       C.c_int32, P, C.c_int32, P, C.c_size_t, P, P]),
    "pe_build_gfb_topk_workspace": (C.c_size_t, [C.c_int32, P, C.c_int64, C.c_float]),
    "pe_build_gfb_topk": (C.c_int, [P, C.c_int32, P, C.c_int64, C.c_float, C.c_int32, P, C.c_size_t,
                                    P, P]),
    "pe_point_attributes": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int32, P, P, C.c_size_t, P, P,
                                      P]),
    "pe_nn_transpose": (C.c_int, [P, C.c_int32, C.c_int32, P, P]),
    "pe_nn_gemm": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, P, C.c_int64, C.c_int64, P,
                             C.c_int64, C.c_int64, P, C.c_int64, C.c_int32, P, P, C.c_int64, P,
                             C.c_int64, C.c_int32, C.c_float, C.c_float, P, C.c_size_t, P]),
    "pe_nn_im2col3": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, C.c_int32, P]),
    "pe_nn_dwconv7": (C.c_int, [P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P]),
    "pe_nn_dwconv7_bwd_workspace": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "pe_nn_dwconv7_bwd": (C.c_int, [P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, P,
                                    P, C.c_size_t, P]),
    "pe_nn_layernorm": (C.c_int, [P, P, P, C.c_int64, C.c_int32, C.c_float, P, P, P, P]),
    "pe_nn_layernorm_bwd_workspace": (C.c_size_t, [C.c_int64, C.c_int32]),
    "pe_nn_layernorm_bwd": (C.c_int, [P, P, P, P, P, C.c_int64, C.c_int32, P, P, P, P,
                                      C.c_size_t, P]),
    "pe_nn_colsum_workspace": (C.c_size_t, [C.c_int64, C.c_int32]),
    "pe_nn_colsum": (C.c_int, [P, C.c_int64, C.c_int32, C.c_int64, P, C.c_int32, P, C.c_size_t,
                               P]),
    "pe_nn_gelu_bwd": (C.c_int, [P, P, C.c_int64, P, P]),
    "pe_nn_maxpool2": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P, C.c_int32,
                                 P]),
    "pe_nn_pixel_shuffle2": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P,
                                       C.c_int64, C.c_int32, C.c_int32, P]),
    "pe_nn_copy_channels": (C.c_int, [P, C.c_int64, C.c_int32, P, C.c_int64, C.c_int32,
                                      C.c_int64, C.c_int32, C.c_int32, P]),
    "pe_nn_to_bf16": (C.c_int, [P, C.c_int64, P, P]),
    "pe_nn_adamw": (C.c_int, [P, P, P, P, P, C.c_int64, C.c_float, C.c_float, C.c_float,
                              C.c_float, C.c_float, C.c_int32, P]),
    "pe_nn_unet_losses_workspace": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "pe_nn_unet_losses": (C.c_int, [P, P, P, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_float,
                                    C.c_float, P, P, P, P, P, P, C.c_size_t, P]),
    "pe_learned_pairs": (C.c_int, [P, C.c_int32, P, P, P, P, P, P, P, P, P]),
    "pe_gfb_hits": (C.c_int, [P, C.c_int32, P, P, P, P, C.c_float, P, P, P]),
}

_lib = None


def load():
    """Load libpointemray.so (build it first with ``paper_2408_15583_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"libpointemray.so is not built ({LIB_PATH}); run "
            "`python -c 'import __graft_entry__ as g; g.build()'` -- there is no CPU fallback")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PeError(RuntimeError):
    def __init__(self, status, where):
        msg = load().pe_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def check(status, where):
    if status != 0:
        raise PeError(status, where)
