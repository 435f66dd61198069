"""Pins for the FP64 reference network and the Eq. 17-21 losses (CPU)."""
import math

import numpy as np
import torch

import scenes
from oracle import unet

W_SMALL = (2, 4, 4, 4)
B_SMALL = (1, 1, 1, 1)


def small_params(seed=0):
    return unet.to_params(scenes.unet_init(seed, W_SMALL, B_SMALL))


def test_shapes_and_heads():
    P = small_params()
    x = torch.rand(2, 1, 16, 16, dtype=torch.float64)
    out = unet.forward(P, x, blocks=B_SMALL)
    assert out["depth"].shape == (2, 1, 16, 16)
    assert out["normal"].shape == (2, 3, 16, 16)
    assert out["mask"].shape == (2, 1, 16, 16)


def test_depth_output_refines_the_input():
    # with the depth head zeroed, the refined depth is the coarse input
    P = small_params()
    P["depth.head.w"].data.zero_()
    P["depth.head.b"].data.zero_()
    x = torch.rand(1, 1, 8, 8, dtype=torch.float64)
    assert torch.equal(unet.forward(P, x, blocks=B_SMALL)["depth"], x)


def test_convnext_block_is_identity_with_zero_last_projection():
    P = small_params()
    P["enc0.0.pw2.w"].data.zero_()
    P["enc0.0.pw2.b"].data.zero_()
    x = torch.randn(1, 2, 8, 8, dtype=torch.float64)
    assert torch.equal(unet.convnext(x, P, "enc0.0"), x)


def test_depthwise_delta_kernel_and_layernorm_of_constant():
    c = 3
    P = {"b.dw.w": torch.zeros(7, 7, c, dtype=torch.float64), "b.dw.b": torch.full((c,), 0.5, dtype=torch.float64),
         "b.ln.g": torch.ones(c, dtype=torch.float64), "b.ln.b": torch.tensor([1.0, 2.0, 3.0], dtype=torch.float64)}
    P["b.dw.w"][3, 3, :] = 1.0
    x = torch.randn(1, c, 6, 6, dtype=torch.float64)
    y = torch.nn.functional.conv2d(x, P["b.dw.w"].permute(2, 0, 1)[:, None], P["b.dw.b"], padding=3,
                                   groups=c)
    assert torch.allclose(y, x + 0.5)
    # LayerNorm over channels of a per-pixel constant vector gives beta
    z = torch.full((1, 4, 4, c), 2.0, dtype=torch.float64)
    assert torch.allclose(torch.nn.functional.layer_norm(z, (c,), P["b.ln.g"], P["b.ln.b"], unet.LN_EPS),
                          P["b.ln.b"].expand(1, 4, 4, c))


def _maps(B=1, H=8, W=8):
    d_gt = torch.zeros(B, H, W, dtype=torch.float64)
    n_gt = torch.zeros(B, H, W, 3, dtype=torch.float64)
    n_gt[..., 2] = 1.0
    return d_gt, n_gt


def test_convnext_block_closed_form_gelu():
    # delta depthwise kernel, LayerNorm (gamma 1, beta 0) over the channel
    # pair (3, 1) -> (1, -1) (up to its 1e-6 epsilon), identity projections
    # through the first two of the 8 expansion channels: the block returns
    # x + GELU(LN(x)) with GELU(t) = t Phi(t), i.e. (3 + Phi(1), 1 - Phi(-1))
    c, h = 2, 8
    P = {"b.dw.w": torch.zeros(7, 7, c, dtype=torch.float64), "b.dw.b": torch.zeros(c, dtype=torch.float64),
         "b.ln.g": torch.ones(c, dtype=torch.float64), "b.ln.b": torch.zeros(c, dtype=torch.float64),
         "b.pw1.w": torch.zeros(h, c, dtype=torch.float64), "b.pw1.b": torch.zeros(h, dtype=torch.float64),
         "b.pw2.w": torch.zeros(c, h, dtype=torch.float64), "b.pw2.b": torch.zeros(c, dtype=torch.float64)}
    P["b.dw.w"][3, 3, :] = 1.0
    P["b.pw1.w"][0, 0] = P["b.pw1.w"][1, 1] = 1.0
    P["b.pw2.w"][0, 0] = P["b.pw2.w"][1, 1] = 1.0
    x = torch.empty(1, c, 5, 5, dtype=torch.float64)
    x[:, 0], x[:, 1] = 3.0, 1.0
    y = unet.convnext(x, P, "b")
    phi = lambda t: 0.5 * (1.0 + math.erf(t / math.sqrt(2.0)))
    assert torch.allclose(y[:, 0], torch.full_like(y[:, 0], 3.0 + phi(1.0)), atol=2e-6)
    assert torch.allclose(y[:, 1], torch.full_like(y[:, 1], 1.0 - phi(-1.0)), atol=2e-6)


def test_focal_loss_closed_values():
    # Eq. 19 with alpha = 0.5, gamma = 2 at p = 0.5: 0.5 * 0.25 * ln 2 for
    # either label
    d_gt, n_gt = _maps()
    out = {"depth": torch.zeros(1, 1, 8, 8, dtype=torch.float64),
           "normal": torch.zeros(1, 3, 8, 8, dtype=torch.float64),
           "mask": torch.zeros(1, 1, 8, 8, dtype=torch.float64)}
    out["normal"][:, 2] = 1.0
    for m in (0.0, 1.0):
        _, parts = unet.losses(out, d_gt, n_gt, torch.full((1, 8, 8), m, dtype=torch.float64))
        assert abs(parts[2].item() - 0.5 * 0.25 * math.log(2)) < 1e-12
    # confident and right -> ~0; confident and wrong -> large
    out["mask"][:] = 20.0
    _, parts = unet.losses(out, d_gt, n_gt, torch.ones(1, 8, 8, dtype=torch.float64))
    assert parts[2].item() < 1e-15
    _, parts = unet.losses(out, d_gt, n_gt, torch.zeros(1, 8, 8, dtype=torch.float64))
    assert abs(parts[2].item() - 0.5 * 20.0) < 1e-6
    # alpha weights the hit class and 1 - alpha the empty one (Eq. 19): at
    # p = 0.5 with alpha = 0.25, 0.25 * 0.25 ln 2 for a hit, 0.75 * 0.25 ln 2
    # for an empty pixel
    out["mask"][:] = 0.0
    for m, a_m in ((1.0, 0.25), (0.0, 0.75)):
        _, parts = unet.losses(out, d_gt, n_gt, torch.full((1, 8, 8), m, dtype=torch.float64),
                               alpha=0.25)
        assert abs(parts[2].item() - a_m * 0.25 * math.log(2)) < 1e-12


def test_normal_depth_and_gradient_losses_closed_values():
    d_gt, n_gt = _maps()
    m = torch.ones(1, 8, 8, dtype=torch.float64)
    out = {"depth": torch.full((1, 1, 8, 8), 0.25, dtype=torch.float64),
           "normal": torch.zeros(1, 3, 8, 8, dtype=torch.float64),
           "mask": torch.zeros(1, 1, 8, 8, dtype=torch.float64)}
    out["normal"][:, 0] = 2.0                       # orthogonal to n_gt: sin = 1
    L, parts = unet.losses(out, d_gt, n_gt, m)
    assert abs(parts[0].item() - 0.0625) < 1e-12    # Eq. 17: (0.25 - 0)^2
    assert abs(parts[1].item() - 1.0) < 1e-7        # Eq. 18 (up to the 1e-8 guard)
    assert parts[3].item() < 1e-5                   # Eq. 20: both gradients are (0,0,1)
    # Eq. 21 with the paper's factors 1, 0.5, 1, 0.5: the mask logit 0 gives
    # the focal value 0.5 * 0.25 ln 2 on every (hit) pixel
    assert abs(L.item() - (0.0625 + 0.5 * 1.0 + 0.5 * 0.25 * math.log(2))) < 1e-6
    out["normal"][:, 0] = 0.0
    out["normal"][:, 2] = 3.0                       # parallel: sin = 0
    _, parts = unet.losses(out, d_gt, n_gt, m)
    assert parts[1].item() < 1e-5
    # a depth ramp vs flat ground truth: (0.5,0,1) vs (0,0,1), sin = 0.5/sqrt(1.25)
    out["depth"][0, 0] = torch.arange(8, dtype=torch.float64)[None, :] * 0.5
    _, parts = unet.losses(out, d_gt, n_gt, m)
    assert abs(parts[3].item() - 0.5 / math.sqrt(1.25)) < 1e-7


def test_gradients_match_finite_differences():
    P = small_params(3)
    x = torch.rand(1, 1, 8, 8, dtype=torch.float64)
    d_gt = torch.rand(1, 8, 8, dtype=torch.float64)
    n_gt = torch.nn.functional.normalize(torch.randn(1, 8, 8, 3, dtype=torch.float64), dim=-1)
    m_gt = (torch.rand(1, 8, 8) > 0.3).double()
    names = ["stem.w", "enc0.0.pw1.w", "enc3.0.dw.w", "normal.fuse0.w", "mask.head.b", "depth.up1.w"]

    def f(*ts):
        Q = dict(P)
        for nm, t in zip(names, ts):
            Q[nm] = t
        L, _ = unet.losses(unet.forward(Q, x, blocks=B_SMALL), d_gt, n_gt, m_gt)
        return L

    assert torch.autograd.gradcheck(f, [P[nm].detach().clone().requires_grad_(True) for nm in names],
                                    eps=1e-6, atol=1e-5, rtol=1e-4)
