"""Learned GFB completion on the GPU: the coarse-depth -> dense GFB network of
PointEMRay (Sec. III-A, Fig. 2/3), trained with Eq. 17-21 and AdamW.

Every step runs in the library's kernels (``pe_nn_*``): this module only
sequences the calls, holds the buffers (torch tensors) and the tape of saved
activations.  Activations are BF16 NHWC, master weights FP32 in one flat
buffer (with a BF16 mirror for the tensor-core GEMMs), gradients FP32.

Structure (the paper's Fig. 3 is missing; parameter names/shapes are
``scenes.unet_param_shapes``): stem 3x3 conv; per level ConvNeXt blocks
(depthwise 7x7 -> LayerNorm -> 1x1 C->4C -> GELU -> 1x1 4C->C, residual);
max-pool + 1x1 conv between levels; three decoders (depth, normal in the uvw
frame, hit-mask logit), each: 3x3 conv to 4C -> pixel shuffle -> concat skip
-> 1x1 -> ConvNeXt block, per level; 1x1 heads (FP32 outputs).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Dict, List

import numpy as np
import torch

from . import _lib
from ._lib import check

BF16 = torch.bfloat16
F32 = torch.float32
HEADS = (("depth", 1), ("normal", 3), ("mask", 1))
LN_EPS = 1e-6


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Ops:
    """Thin wrappers of the layer entry points on one stream."""

    def __init__(self, device, stream=None):
        self.lib = _lib.load()
        self.dev = torch.device(device)
        self.stream = stream
        self._ws = torch.empty(0, dtype=torch.uint8, device=self.dev)

    def s(self):
        st = self.stream if self.stream is not None else torch.cuda.current_stream(self.dev)
        return C.c_void_p(st.cuda_stream)

    def ws(self, nbytes):
        if self._ws.numel() < nbytes:
            self._ws = torch.empty(int(nbytes * 1.25) + 4096, dtype=torch.uint8, device=self.dev)
        return self._ws

    # C[m,n] = sum_k A(m,k) B(k,n) with explicit element strides
    def gemm(self, M, N, K, A, sam, sak, B, sbk, sbn, Cout, ldc, bias=None, R=None, ldr=0,
             Z=None, ldz=0, gelu=False, alpha=1.0, beta=0.0, dgelu=False):
        nb = self.lib.pe_nn_gemm_workspace(M, N, K)
        ws = self.ws(nb)
        check(self.lib.pe_nn_gemm(M, N, K, _p(A), sam, sak, _p(B), sbk, sbn, _p(Cout), ldc,
                                  1 if Cout.dtype == F32 else 0, _p(bias), _p(R), ldr, _p(Z), ldz,
                                  2 if dgelu else (1 if gelu else 0), alpha, beta, _p(ws),
                                  ws.numel(), self.s()),
              "pe_nn_gemm")

    # y[P,N] = x[P,K] . W[N,K]^T (+ bias, + residual, gelu)
    def linear(self, x, ldx, W, bias, out, ldo, R=None, ldr=0, Z=None, gelu=False):
        P = out.shape[0]
        N, K = W.shape
        self.gemm(P, N, K, x, ldx, 1, W, 1, K, out, ldo, bias=bias, R=R, ldr=ldr, Z=Z,
                  ldz=N, gelu=gelu)

    def linear_bwd(self, dy, x, ldx, W, dx, ldd, dW, db, need_dx=True, gelu_z=None):
        """dy [P,N] (BF16, contiguous), x [P,K] with row stride ldx.  The data
        gradient reads W through its transpose, so both of its operands are
        K-contiguous (the layout of the tensor-core kernel); with gelu_z it
        is multiplied by GELU'(gelu_z) in the epilogue (the backward of a
        GELU applied to this layer's input)."""
        P, N = dy.shape
        K = W.shape[1]
        if need_dx:
            Wt = torch.empty(K, N, dtype=W.dtype, device=self.dev)
            check(self.lib.pe_nn_transpose(_p(W), N, K, _p(Wt), self.s()), "pe_nn_transpose")
            self.gemm(P, K, N, dy, N, 1, Wt, 1, N, dx, ldd, Z=gelu_z, ldz=K,
                      dgelu=gelu_z is not None)
        self.gemm(N, K, P, dy, 1, N, x, ldx, 1, dW, K)
        self.colsum(dy, P, N, N, db)

    def colsum(self, X, M, N, ld, out, accumulate=False):
        nb = self.lib.pe_nn_colsum_workspace(M, N)
        ws = self.ws(nb)
        check(self.lib.pe_nn_colsum(_p(X), M, N, ld, _p(out), 1 if accumulate else 0, _p(ws),
                                    ws.numel(), self.s()), "pe_nn_colsum")

    def im2col(self, x, B, H, W, Cc, col, backward=False):
        check(self.lib.pe_nn_im2col3(_p(x), B, H, W, Cc, _p(col), 1 if backward else 0, self.s()),
              "pe_nn_im2col3")

    def dw(self, x, w, b, B, H, W, Cc, y):
        check(self.lib.pe_nn_dwconv7(_p(x), _p(w), _p(b), B, H, W, Cc, _p(y), self.s()),
              "pe_nn_dwconv7")

    def dw_bwd(self, x, dy, w, B, H, W, Cc, dx, dw, db):
        nb = self.lib.pe_nn_dwconv7_bwd_workspace(B, H, W, Cc)
        ws = self.ws(nb)
        check(self.lib.pe_nn_dwconv7_bwd(_p(x), _p(dy), _p(w), B, H, W, Cc, _p(dx), _p(dw), _p(db),
                                         _p(ws), ws.numel(), self.s()), "pe_nn_dwconv7_bwd")

    def ln(self, x, g, b, P, Cc, y, mean, rstd):
        check(self.lib.pe_nn_layernorm(_p(x), _p(g), _p(b), P, Cc, LN_EPS, _p(y), _p(mean),
                                       _p(rstd), self.s()), "pe_nn_layernorm")

    def ln_bwd(self, dy, x, g, mean, rstd, P, Cc, dx, dg, db):
        nb = self.lib.pe_nn_layernorm_bwd_workspace(P, Cc)
        ws = self.ws(nb)
        check(self.lib.pe_nn_layernorm_bwd(_p(dy), _p(x), _p(g), _p(mean), _p(rstd), P, Cc, _p(dx),
                                           _p(dg), _p(db), _p(ws), ws.numel(), self.s()),
              "pe_nn_layernorm_bwd")

    def gelu_bwd(self, da, z, dz):
        check(self.lib.pe_nn_gelu_bwd(_p(da), _p(z), z.numel(), _p(dz), self.s()), "pe_nn_gelu_bwd")

    def maxpool(self, x, B, H, W, Cc, y, arg, backward=False):
        check(self.lib.pe_nn_maxpool2(_p(x), B, H, W, Cc, _p(y), _p(arg), 1 if backward else 0,
                                      self.s()), "pe_nn_maxpool2")

    def shuffle(self, src, B, H, W, Cc, dst, ld_big, off, backward=False):
        check(self.lib.pe_nn_pixel_shuffle2(_p(src), B, H, W, Cc, _p(dst), ld_big, off,
                                            1 if backward else 0, self.s()), "pe_nn_pixel_shuffle2")

    def copy(self, src, lds, soff, dst, ldd, doff, P, Cc, accumulate=False):
        check(self.lib.pe_nn_copy_channels(_p(src), lds, soff, _p(dst), ldd, doff, P, Cc,
                                           1 if accumulate else 0, self.s()), "pe_nn_copy_channels")

    def to_bf16(self, x, y):
        check(self.lib.pe_nn_to_bf16(_p(x), x.numel(), _p(y), self.s()), "pe_nn_to_bf16")


@dataclass
class Slot:
    off: int
    shape: tuple

    @property
    def n(self):
        return int(np.prod(self.shape))


class UNet:
    """Parameters, forward with a tape, backward, AdamW."""

    def __init__(self, params: Dict[str, np.ndarray], widths=(32, 64, 128, 256),
                 blocks=(2, 2, 2, 2), device="cuda:0", stream=None):
        self.widths, self.blocks = tuple(widths), tuple(blocks)
        self.L = len(widths)
        self.ops = Ops(device, stream)
        self.dev = self.ops.dev
        self.slots: Dict[str, Slot] = {}
        off = 0
        for k, v in params.items():
            self.slots[k] = Slot(off, tuple(v.shape))
            off += (v.size + 7) // 8 * 8          # 32-byte aligned views
        self.n_params = off
        flat = np.zeros(off, np.float32)
        for k, v in params.items():
            s = self.slots[k]
            flat[s.off:s.off + s.n] = v.ravel()
        self.master = torch.from_numpy(flat).to(self.dev)
        self.mirror = torch.empty(off, dtype=BF16, device=self.dev)
        self.grad = torch.zeros(off, dtype=F32, device=self.dev)
        self.m = torch.zeros(off, dtype=F32, device=self.dev)
        self.v = torch.zeros(off, dtype=F32, device=self.dev)
        self.ops.to_bf16(self.master, self.mirror)
        self.t = 0

    # parameter views
    def pf(self, name):
        s = self.slots[name]
        return self.master[s.off:s.off + s.n].view(s.shape)

    def pb(self, name):
        s = self.slots[name]
        return self.mirror[s.off:s.off + s.n].view(s.shape[0], -1)

    def g(self, name):
        s = self.slots[name]
        return self.grad[s.off:s.off + s.n].view(s.shape)

    def params_numpy(self):
        host = self.master.cpu().numpy()
        return {k: host[s.off:s.off + s.n].reshape(s.shape).copy() for k, s in self.slots.items()}

    # ------------------------------------------------------------------------
    def _empty(self, *shape, dtype=BF16):
        return torch.empty(shape, dtype=dtype, device=self.dev)

    def _block_fwd(self, x, p, B, H, W, Cc, tape):
        o = self.ops
        P = B * H * W
        a = self._empty(P, Cc)
        o.dw(x, self.pf(p + ".dw.w"), self.pf(p + ".dw.b"), B, H, W, Cc, a)
        bn = self._empty(P, Cc)
        mean = self._empty(P, dtype=F32)
        rstd = self._empty(P, dtype=F32)
        o.ln(a, self.pf(p + ".ln.g"), self.pf(p + ".ln.b"), P, Cc, bn, mean, rstd)
        z1 = self._empty(P, 4 * Cc)
        h = self._empty(P, 4 * Cc)
        o.linear(bn, Cc, self.pb(p + ".pw1.w"), self.pf(p + ".pw1.b"), h, 4 * Cc, Z=z1, gelu=True)
        y = self._empty(P, Cc)
        o.linear(h, 4 * Cc, self.pb(p + ".pw2.w"), self.pf(p + ".pw2.b"), y, Cc, R=x, ldr=Cc)
        tape.append(("block", p, (x, a, bn, mean, rstd, z1, h, B, H, W, Cc)))
        return y

    def _block_bwd(self, dy, rec):
        o = self.ops
        p, (x, a, bn, mean, rstd, z1, h, B, H, W, Cc) = rec
        P = B * H * W
        dz1 = self._empty(P, 4 * Cc)          # dL/dz1 = (dy . W2) * GELU'(z1), one GEMM
        o.linear_bwd(dy, h, 4 * Cc, self.pb(p + ".pw2.w"), dz1, 4 * Cc, self.g(p + ".pw2.w"),
                     self.g(p + ".pw2.b"), gelu_z=z1)
        dbn = self._empty(P, Cc)
        o.linear_bwd(dz1, bn, Cc, self.pb(p + ".pw1.w"), dbn, Cc, self.g(p + ".pw1.w"),
                     self.g(p + ".pw1.b"))
        da = self._empty(P, Cc)
        o.ln_bwd(dbn, a, self.pf(p + ".ln.g"), mean, rstd, P, Cc, da, self.g(p + ".ln.g"),
                 self.g(p + ".ln.b"))
        dx = self._empty(P, Cc)
        o.dw_bwd(x, da, self.pf(p + ".dw.w"), B, H, W, Cc, dx, self.g(p + ".dw.w"),
                 self.g(p + ".dw.b"))
        o.copy(dy, Cc, 0, dx, Cc, 0, P, Cc, accumulate=True)      # residual
        return dx

    def _conv3_fwd(self, x, name, B, H, W, Cin, Cout, tape):
        P = B * H * W
        col = self._empty(P, 9 * Cin)
        self.ops.im2col(x, B, H, W, Cin, col)
        y = self._empty(P, Cout)
        self.ops.linear(col, 9 * Cin, self.pb(name + ".w"), self.pf(name + ".b"), y, Cout)
        tape.append(("conv3", name, (col, B, H, W, Cin, Cout)))
        return y

    def _conv3_bwd(self, dy, rec, need_dx=True):
        name, (col, B, H, W, Cin, Cout) = rec
        P = B * H * W
        dcol = self._empty(P, 9 * Cin) if need_dx else None
        self.ops.linear_bwd(dy, col, 9 * Cin, self.pb(name + ".w"), dcol, 9 * Cin,
                            self.g(name + ".w").view(Cout, 9 * Cin), self.g(name + ".b"),
                            need_dx=need_dx)
        if not need_dx:
            return None
        dx = self._empty(P, Cin)
        self.ops.im2col(dcol, B, H, W, Cin, dx, backward=True)
        return dx

    # ------------------------------------------------------------------------
    def forward(self, x, B, H, W):
        """x: BF16 [B*H*W] normalised coarse depth.  Returns (outputs, tape):
        outputs['depth'] [P] FP32, ['normal'] [P,3] FP32, ['mask'] [P] FP32 logits."""
        assert H % (1 << (self.L - 1)) == 0 and W % (1 << (self.L - 1)) == 0
        o = self.ops
        tape: List = []
        c = self.widths
        y = self._conv3_fwd(x.view(-1, 1), "stem", B, H, W, 1, c[0], tape)
        skips = []
        dims = []
        h, w = H, W
        for lvl in range(self.L):
            if lvl > 0:
                pooled = self._empty(B * (h // 2) * (w // 2), c[lvl - 1])
                arg = self._empty(B * (h // 2) * (w // 2), c[lvl - 1], dtype=torch.uint8)
                o.maxpool(y, B, h, w, c[lvl - 1], pooled, arg)
                h, w = h // 2, w // 2
                y2 = self._empty(B * h * w, c[lvl])
                o.linear(pooled, c[lvl - 1], self.pb(f"down{lvl}.w"), self.pf(f"down{lvl}.b"), y2,
                         c[lvl])
                tape.append(("down", lvl, (pooled, arg, B, h, w)))
                y = y2
            for k in range(self.blocks[lvl]):
                y = self._block_fwd(y, f"enc{lvl}.{k}", B, h, w, c[lvl], tape)
            skips.append(y)
            dims.append((h, w))
        outs = {}
        dec_tapes = {}
        for head, nout in HEADS:
            dt: List = []
            u = skips[-1]
            for lvl in range(self.L - 2, -1, -1):
                hh, ww = dims[lvl + 1]
                up = self._conv3_fwd(u, f"{head}.up{lvl}", B, hh, ww, c[lvl + 1], 4 * c[lvl], dt)
                cat = self._empty(B * dims[lvl][0] * dims[lvl][1], 2 * c[lvl])
                o.shuffle(up, B, hh, ww, c[lvl], cat, 2 * c[lvl], 0)
                o.copy(skips[lvl], c[lvl], 0, cat, 2 * c[lvl], c[lvl], cat.shape[0], c[lvl])
                fu = self._empty(cat.shape[0], c[lvl])
                o.linear(cat, 2 * c[lvl], self.pb(f"{head}.fuse{lvl}.w"),
                         self.pf(f"{head}.fuse{lvl}.b"), fu, c[lvl])
                dt.append(("fuse", lvl, (cat, B, dims[lvl][0], dims[lvl][1], hh, ww)))
                u = self._block_fwd(fu, f"{head}.blk{lvl}", B, dims[lvl][0], dims[lvl][1], c[lvl], dt)
            out = self._empty(B * H * W, nout, dtype=F32)
            # the depth head refines the coarse input: correction + input
            o.linear(u, c[0], self.pb(f"{head}.head.w"), self.pf(f"{head}.head.b"), out, nout,
                     R=x if head == "depth" else None, ldr=1)
            dt.append(("head", head, (u,)))
            outs[head] = out if nout > 1 else out.view(-1)
            dec_tapes[head] = dt
        return outs, {"enc": tape, "dec": dec_tapes, "skips": skips, "dims": dims, "B": B}

    def backward(self, tape, grads: Dict[str, torch.Tensor]):
        """grads: FP32 dL/d(output) per head ([P] or [P,3]).  Fills self.grad."""
        o = self.ops
        c = self.widths
        B = tape["B"]
        dims = tape["dims"]
        self.grad.zero_()
        dskip = [torch.zeros_like(s) for s in tape["skips"]]
        for head, nout in HEADS:
            dt = tape["dec"][head]
            g32 = grads[head].reshape(-1, nout)
            gb = self._empty(g32.shape[0], nout)
            o.to_bf16(g32.contiguous(), gb)
            (_, _, (u,)) = dt[-1]
            du = self._empty(u.shape[0], c[0])
            o.linear_bwd(gb, u, c[0], self.pb(f"{head}.head.w"), du, c[0],
                         self.g(f"{head}.head.w"), self.g(f"{head}.head.b"))
            i = len(dt) - 2
            for lvl in range(0, self.L - 1):
                # records in reverse: block, fuse, conv3 (up)
                kind, p, rec = dt[i]
                assert kind == "block"
                dfu = self._block_bwd(du, (p, rec))
                kind, _, (cat, _, hh2, ww2, hh, ww) = dt[i - 1]
                assert kind == "fuse"
                P2 = cat.shape[0]
                dcat = self._empty(P2, 2 * c[lvl])
                o.linear_bwd(dfu, cat, 2 * c[lvl], self.pb(f"{head}.fuse{lvl}.w"), dcat, 2 * c[lvl],
                             self.g(f"{head}.fuse{lvl}.w"), self.g(f"{head}.fuse{lvl}.b"))
                o.copy(dcat, 2 * c[lvl], c[lvl], dskip[lvl], c[lvl], 0, P2, c[lvl], accumulate=True)
                dup = self._empty(B * hh * ww, 4 * c[lvl])
                o.shuffle(dcat, B, hh, ww, c[lvl], dup, 2 * c[lvl], 0, backward=True)
                kind, name, rec = dt[i - 2]
                assert kind == "conv3"
                du = self._conv3_bwd(dup, (name, rec))
                i -= 3
            o.copy(du, c[-1], 0, dskip[-1], c[-1], 0, du.shape[0], c[-1], accumulate=True)
        # encoder, deepest level first
        enc = tape["enc"]
        i = len(enc) - 1
        for lvl in range(self.L - 1, -1, -1):
            dy = dskip[lvl]
            for _ in range(self.blocks[lvl]):
                kind, p, rec = enc[i]
                assert kind == "block"
                dy = self._block_bwd(dy, (p, rec))
                i -= 1
            if lvl > 0:
                kind, _, (pooled, arg, _, h, w) = enc[i]
                assert kind == "down"
                dpool = self._empty(pooled.shape[0], c[lvl - 1])
                o.linear_bwd(dy, pooled, c[lvl - 1], self.pb(f"down{lvl}.w"), dpool, c[lvl - 1],
                             self.g(f"down{lvl}.w"), self.g(f"down{lvl}.b"))
                dfull = self._empty(B * 2 * h * 2 * w, c[lvl - 1])
                o.maxpool(dpool, B, 2 * h, 2 * w, c[lvl - 1], dfull, arg, backward=True)
                o.copy(dfull, c[lvl - 1], 0, dskip[lvl - 1], c[lvl - 1], 0, dfull.shape[0],
                       c[lvl - 1], accumulate=True)
                i -= 1
        kind, name, rec = enc[i]
        assert kind == "conv3" and name == "stem" and i == 0
        self._conv3_bwd(dy, (name, rec), need_dx=False)

    def adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.01):
        self.t += 1
        check(self.ops.lib.pe_nn_adamw(_p(self.master), _p(self.grad), _p(self.m), _p(self.v),
                                       _p(self.mirror), self.n_params, lr, beta1, beta2, eps,
                                       weight_decay, self.t, self.ops.s()), "pe_nn_adamw")

    def losses(self, outs, d_gt, n_gt, m_gt, B, H, W, alpha=0.5, gamma=2.0,
               lambdas=(1.0, 0.5, 1.0, 0.5)):
        lib = self.ops.lib
        P = B * H * W
        lam = torch.tensor(lambdas, dtype=F32)
        loss = torch.empty(5, dtype=F32, device=self.dev)
        gd = torch.empty(P, dtype=F32, device=self.dev)
        gn = torch.empty(P, 3, dtype=F32, device=self.dev)
        gz = torch.empty(P, dtype=F32, device=self.dev)
        nb = lib.pe_nn_unet_losses_workspace(B, H, W)
        ws = self.ops.ws(nb)
        check(lib.pe_nn_unet_losses(_p(outs["depth"]), _p(outs["normal"]), _p(outs["mask"]),
                                    _p(d_gt), _p(n_gt), _p(m_gt), B, H, W, alpha, gamma,
                                    lam.numpy().ctypes.data_as(C.c_void_p), _p(loss), _p(gd),
                                    _p(gn), _p(gz), _p(ws), ws.numel(), self.ops.s()),
              "pe_nn_unet_losses")
        return loss, {"depth": gd, "normal": gn, "mask": gz}

    def train_step(self, x, d_gt, n_gt, m_gt, B, H, W, lr):
        outs, tape = self.forward(x, B, H, W)
        loss, grads = self.losses(outs, d_gt, n_gt, m_gt, B, H, W)
        self.backward(tape, grads)
        self.adamw(lr)
        return loss


class GraphedUNet:
    """The U-Net's fixed-shape work as captured CUDA graphs: for training,
    forward + Eq. 17-21 losses + backward of a batch of B maps of H x W (one
    replay per step; the AdamW update runs after it as its own launch, since
    its step count and learning rate change every step); for inference, the
    forward pass alone.  Each call copies its inputs into the captured
    buffers and replays: the same kernels in the same order as the eager
    calls, so the results are the same bit for bit, without the host's
    per-layer launch work (about 1,260 launches per training step) between
    the kernels.  Captured once per shape, at the first call (after one eager
    warm-up pass that sizes the workspaces)."""

    def __init__(self, net: UNet, B: int, H: int, W: int):
        self.net, self.B, self.H, self.W = net, B, H, W
        P = B * H * W
        dev = net.dev
        self.x = torch.zeros(P, dtype=BF16, device=dev)
        self.d_gt = torch.zeros(P, dtype=F32, device=dev)
        self.n_gt = torch.zeros(P, 3, dtype=F32, device=dev)
        self.m_gt = torch.zeros(P, dtype=F32, device=dev)
        self._train = None
        self._infer = None

    def _fwd_bwd(self):
        net = self.net
        outs, tape = net.forward(self.x, self.B, self.H, self.W)
        loss, grads = net.losses(outs, self.d_gt, self.n_gt, self.m_gt, self.B, self.H, self.W)
        net.backward(tape, grads)
        return loss

    def _capture(self, fn):
        side = torch.cuda.Stream(self.net.dev)
        side.wait_stream(torch.cuda.current_stream(self.net.dev))
        with torch.cuda.stream(side):
            fn()                                  # eager warm-up: workspaces at full size
        torch.cuda.current_stream(self.net.dev).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            out = fn()
        return g, out

    def train_step(self, x, d_gt, n_gt, m_gt, lr):
        """One training step (the graph, then AdamW); returns the loss vector."""
        self.x.copy_(x)
        self.d_gt.copy_(d_gt)
        self.n_gt.copy_(n_gt)
        self.m_gt.copy_(m_gt)
        if self._train is None:
            # the warm-up inside the capture runs forward and backward once;
            # its gradients are overwritten by the replay below
            self._train = self._capture(self._fwd_bwd)
        g, loss = self._train
        g.replay()
        self.net.adamw(lr)
        return loss

    def forward(self, x):
        """Inference: the outputs dict of the captured forward pass (its
        tensors are overwritten by the next call)."""
        self.x.copy_(x)
        if self._infer is None:
            self._infer = self._capture(
                lambda: self.net.forward(self.x, self.B, self.H, self.W)[0])
        g, outs = self._infer
        g.replay()
        return outs


def lr_schedule(step, steps_per_epoch, lr0=1e-4, floor=1e-6):
    """The paper's schedule (Sec. IV-A): start at 1e-4, halve every ten
    epochs, never below 1e-6."""
    return max(floor, lr0 * 0.5 ** (step // max(1, 10 * steps_per_epoch)))
