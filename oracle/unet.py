"""FP64 CPU reference of the learned GFB completion network and its losses --
TEST INFRASTRUCTURE ONLY (imported by tests/, the smoke check and bench's CPU
legs, never by the product path).

Written with plain PyTorch CPU ops in float64 (autograd gives the reference
gradients), following the paper: a U-Net with ConvNeXt blocks in the encoder
(Sec. III-A, ref 49), max-pooling down, sub-pixel convolution up (ref 51), a
shared encoder and three decoders for depth, normal and hit mask, and the
losses of Eq. 17-21 with the factors of Eq. 21.  Fig. 3 (the exact structure)
is missing, so the structure is the reading documented with the parameter
shapes in scenes.unet_param_shapes.  Layout: NCHW internally; parameters in
the shared layout (3x3 conv [Cout,3,3,Cin], 1x1 [Cout,Cin], depthwise
[7,7,C]).
"""
from __future__ import annotations

import torch
import torch.nn.functional as F

HEADS = (("depth", 1), ("normal", 3), ("mask", 1))
LN_EPS = 1e-6
CROSS_EPS = 1e-12     # |a x b| = sqrt(|a x b|^2 + eps): smooth where a || b
DIV_EPS = 1e-8


def to_params(np_params, requires_grad=True):
    return {k: torch.tensor(v, dtype=torch.float64, requires_grad=requires_grad)
            for k, v in np_params.items()}


def conv3(x, w, b):
    return F.conv2d(x, w.permute(0, 3, 1, 2), b, padding=1)


def conv1(x, w, b):
    return F.conv2d(x, w[:, :, None, None], b)


def convnext(x, P, p):
    c = x.shape[1]
    y = F.conv2d(x, P[p + ".dw.w"].permute(2, 0, 1)[:, None], P[p + ".dw.b"], padding=3, groups=c)
    y = F.layer_norm(y.permute(0, 2, 3, 1), (c,), P[p + ".ln.g"], P[p + ".ln.b"], LN_EPS)
    y = y.permute(0, 3, 1, 2)
    y = F.gelu(conv1(y, P[p + ".pw1.w"], P[p + ".pw1.b"]))
    y = conv1(y, P[p + ".pw2.w"], P[p + ".pw2.b"])
    return x + y


def forward(P, x, n_levels=4, blocks=(2, 2, 2, 2)):
    """x: [B,1,H,W] normalised coarse depth -> dict of depth [B,1,H,W]
    (input + the depth head's correction), normal [B,3,H,W] (raw, uvw frame),
    mask logit [B,1,H,W]."""
    skips = []
    y = conv3(x, P["stem.w"], P["stem.b"])
    for lvl in range(n_levels):
        if lvl > 0:
            y = conv1(F.max_pool2d(y, 2), P[f"down{lvl}.w"], P[f"down{lvl}.b"])
        for k in range(blocks[lvl]):
            y = convnext(y, P, f"enc{lvl}.{k}")
        skips.append(y)
    out = {}
    for head, _ in HEADS:
        u = skips[-1]
        for lvl in range(n_levels - 2, -1, -1):
            u = F.pixel_shuffle(conv3(u, P[f"{head}.up{lvl}.w"], P[f"{head}.up{lvl}.b"]), 2)
            u = torch.cat([u, skips[lvl]], dim=1)
            u = conv1(u, P[f"{head}.fuse{lvl}.w"], P[f"{head}.fuse{lvl}.b"])
            u = convnext(u, P, f"{head}.blk{lvl}")
        out[head] = conv1(u, P[f"{head}.head.w"], P[f"{head}.head.b"])
    # the depth decoder refines the coarse depth: its head output is a
    # correction added to the input map (empty input pixels hold 0)
    out["depth"] = out["depth"] + x
    return out


def _cross_norm(a, b):
    c = torch.cross(a, b, dim=-1)
    return torch.sqrt((c * c).sum(-1) + CROSS_EPS)


def losses(out, d_gt, n_gt, m_gt, alpha=0.5, gamma=2.0):
    """Eq. 17-21.  d_gt [B,H,W] normalised depth, n_gt [B,H,W,3], m_gt [B,H,W]
    in {0,1}.  L1, L2, L4 are means over ground-truth hit pixels (L4 over hit
    pixels whose 4 neighbours are hits, interior only), L3 over all pixels;
    L4 compares (d_u, d_v, 1) vectors from central differences.
    Returns (L, [L1, L2, L3, L4])."""
    d = out["depth"][:, 0]
    n = out["normal"].permute(0, 2, 3, 1)
    z = out["mask"][:, 0]
    hit = m_gt > 0.5
    nh = hit.sum().clamp(min=1)
    L1 = ((d - d_gt) ** 2)[hit].sum() / nh
    cn = _cross_norm(n, n_gt) / (torch.linalg.norm(n, dim=-1) * torch.linalg.norm(n_gt, dim=-1) + DIV_EPS)
    L2 = cn[hit].sum() / nh
    logp = -F.softplus(-z)
    log1mp = -F.softplus(z)
    p = torch.sigmoid(z)
    foc = torch.where(hit, -alpha * (1 - p) ** gamma * logp, -(1 - alpha) * p ** gamma * log1mp)
    L3 = foc.mean()

    def grads(dd):
        gu = 0.5 * (dd[:, 1:-1, 2:] - dd[:, 1:-1, :-2])
        gv = 0.5 * (dd[:, 2:, 1:-1] - dd[:, :-2, 1:-1])
        return torch.stack([gu, gv, torch.ones_like(gu)], dim=-1)

    inner = hit[:, 1:-1, 1:-1] & hit[:, 1:-1, 2:] & hit[:, 1:-1, :-2] & hit[:, 2:, 1:-1] & hit[:, :-2, 1:-1]
    gp, gg = grads(d), grads(d_gt)
    c4 = _cross_norm(gp, gg) / (torch.linalg.norm(gp, dim=-1) * torch.linalg.norm(gg, dim=-1) + DIV_EPS)
    L4 = c4[inner].sum() / inner.sum().clamp(min=1)
    L = 1.0 * L1 + 0.5 * L2 + 1.0 * L3 + 0.5 * L4
    return L, [L1, L2, L3, L4]
