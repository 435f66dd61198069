"""Convenience composition of the C-ABI calls for a scene (still only
argument marshalling: every step runs in the library's kernels)."""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import torch

from . import api
from ._lib import PeParams, PeView


def scene_to_device(scene, device="cuda:0"):
    pos = torch.from_numpy(np.ascontiguousarray(scene.pos, dtype=np.float32)).to(device)
    nrm = torch.from_numpy(np.ascontiguousarray(scene.nrm, dtype=np.float32)).to(device)
    rad = torch.from_numpy(np.ascontiguousarray(scene.rad, dtype=np.float32)).to(device)
    return pos, nrm, rad


def views_from_angles(theta_deg: Sequence[float], phi_deg: Sequence[float], centre, extent: float,
                      W: int, H: int) -> List[PeView]:
    return [api.view_from_angles(t, p, centre, extent, W, H) for t, p in zip(theta_deg, phi_deg)]


def default_params(pos: np.ndarray, gviews: Sequence[PeView], G: int = 256, tau: float = 3.0,
                   first_bounce_from_geom: bool = False, edge_mode: int = 0) -> PeParams:
    """epsilon = r = the smallest aggregation-view pitch (values the paper
    leaves open)."""
    lmin = float(min(v.pitch for v in gviews))
    return api.make_params(pos, lmin, lmin, G=G, tau=tau,
                           first_bounce_from_geom=first_bounce_from_geom, edge_mode=edge_mode)


def build_geometry(pos, nrm, rad, gviews: Sequence[PeView], params: PeParams, stream=None):
    """GFBs of the aggregation views (surfel splatting) fused into splats."""
    g = api.build_gfb(gviews, pos, nrm, rad, 0, 0.0, stream=stream, outputs=("nd", "mask"))
    geom = api.aggregate_views(gviews, g["nd"], g["mask"], params, stream=stream)
    return geom, g


def field_every_bounce(views, keys, nrm, geom, prm, mb: int, freqs_hz, stream=None):
    """PO at every bounce (instead of Eq. 14's last hit), one library call
    (``pe_po_field_every_bounce``): for b = 1..mb the rays traced to b
    bounces whose b-th hit is their last contribute Eq. 14 at that hit, Psi
    tested toward the monostatic receiver; the b fields are summed in the
    library.  Returns float64 [n_views, F, 2 pol, 3, re/im]."""
    return api.po_field_every_bounce(views, keys, nrm, geom, prm, mb, freqs_hz, stream=stream)
