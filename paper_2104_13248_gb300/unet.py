"""Few-view correction network: a 3-level 3-D residual U-Net on libbp's kernels.

The network maps a back-projection from 1/6 of the views to the full-view
FDK: out = input + net(input). Levels at 16/32/64 channels with 3x3x3
convolutions and ReLU:

    e1a (1 -> 16) [, e1b (16 -> 16)]               = s1   level 1
    pool, e2a (16 -> 32), e2b (32 -> 32)           = s2   level 2
    pool, e3a (32 -> 64), e3b (64 -> 64)                  level 3
    u3 (64 -> 32, linear), upsample + s2           = a2
    d2 (32 -> 32), u2 (32 -> 16, linear), upsample + s1 = a1
    [d1 (16 -> 16),] head (1x1x1, 16 -> 1) + input

The two bracketed full-resolution convolutions are optional (UNet(e1b=,
d1=)) and off by default: at 256^3 they cost 1.1 of the 2.7 ms of an
inference, and without them the network, trained four times as long,
reaches about the same held-out error (RMSE ratio 0.39 against 0.36).

The skip connections add (a projection to the finer level's width, nearest
upsampling, then the sum), so every level-1 convolution has 16 input and 16
output channels. The one-channel input layer (cnn_stem_forward, or
cnn_stem_pool_forward with the first pooling) puts its taps into the GEMM's
K dimension instead of channels, the output head is the usual U-Net 1x1x1 projection
(cnn_head1_*); every other convolution is a BF16 implicit GEMM on the
tensor cores with FP32 accumulation (cnn_conv3d_* in include/unet.h).
Activations and their gradients are BF16 channels-last tensors; the master
weights, weight gradients and Adam moments FP32. Forward and backward are
written out layer by layer (the kernels are not torch operators). The paper
has no learned component; this serves the few-view workload.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from . import _lib
from ._lib import check

# (name, cin, cout) of the convolutions; e1a (cin 1) is the CUDA-core input layer
LAYERS = [("e1a", 1, 16), ("e1b", 16, 16), ("e2a", 16, 32), ("e2b", 32, 32), ("e3a", 32, 64),
          ("e3b", 64, 64), ("u3", 64, 32), ("d2", 32, 32), ("u2", 32, 16), ("d1", 16, 16)]
LINEAR = {"u3", "u2"}   # projections before an additive skip: no ReLU
HEAD_CIN = 16


def _p(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def conv_flops(shape, e1b: bool = False, d1: bool = False) -> float:
    """Multiply-adds x 2 of one forward pass at volume shape (N, D, H, W)."""
    n, d, h, w = shape
    v1 = n * d * h * w
    v2, v3 = v1 / 8, v1 / 64
    macs = 27 * (v1 * (1 * 16 + 16 * 16 * (int(e1b) + int(d1))) +
                 v2 * (16 * 32 + 32 * 32 + 32 * 32 + 32 * 16) +
                 v3 * (32 * 64 + 64 * 64 + 64 * 32)) + v1 * HEAD_CIN
    return 2.0 * macs


class UNet:
    def __init__(self, seed: int = 0, device: str = "cuda", e1b: bool = False, d1: bool = False):
        self.device = torch.device(device)
        self.has_e1b, self.has_d1 = e1b, d1
        self.layers = [l for l in LAYERS if (l[0] != "e1b" or e1b) and (l[0] != "d1" or d1)]
        self.off = {}
        n = 0
        for name, cin, cout in self.layers:
            self.off[name] = (n, n + cout * 27 * cin, cin, cout)   # weight start, bias start
            n += cout * 27 * cin + cout
        self.n_conv = n
        self.head_off = n
        n += HEAD_CIN + 1
        self.n_params = n
        g = torch.Generator().manual_seed(seed)
        p = torch.zeros(n, dtype=torch.float32)
        for name, cin, cout in self.layers:
            w0, b0, _, _ = self.off[name]
            std = math.sqrt((1.0 if name in LINEAR else 2.0) / (27 * cin))
            p[w0:b0] = torch.randn(cout * 27 * cin, generator=g) * std
        p[self.head_off:self.head_off + HEAD_CIN] = torch.randn(HEAD_CIN, generator=g) * 0.02
        self.params = p.to(self.device)
        self.params16 = self.params.to(torch.bfloat16)   # BF16 copy read by the kernels
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        largest = max(27 * cin * cout for _, cin, cout in self.layers)
        self.wt = torch.empty(largest, dtype=torch.bfloat16, device=self.device)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.device)
        self._bufs = {}

    # parameter views ------------------------------------------------------
    def w16(self, name):
        w0, b0, _, _ = self.off[name]
        return self.params16[w0:b0]

    def bias(self, name):
        _, b0, _, cout = self.off[name]
        return self.params[b0:b0 + cout]

    def gw(self, name):
        w0, b0, _, _ = self.off[name]
        return self.grads[w0:b0]

    def gb(self, name):
        _, b0, _, cout = self.off[name]
        return self.grads[b0:b0 + cout]

    def head_w(self):
        return self.params[self.head_off:self.head_off + HEAD_CIN]

    def head_b(self):
        return self.params[self.head_off + HEAD_CIN:self.head_off + HEAD_CIN + 1]

    def state_dict(self) -> dict:
        return {"params": self.params.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "t": self.t}

    def load_state_dict(self, sd: dict):
        self.params.copy_(sd["params"].to(self.device))
        self.params16.copy_(self.params.to(torch.bfloat16))
        self.m.copy_(sd["m"].to(self.device))
        self.v.copy_(sd["v"].to(self.device))
        self.t = int(sd["t"])

    # activation buffers ---------------------------------------------------
    def _buffers(self, shape, train: bool):
        key = (tuple(shape), train)
        if key in self._bufs:
            return self._bufs[key]
        n, d, h, w = shape
        if d % 4 or h % 4 or w % 4:
            raise ValueError("volume dimensions must be multiples of 4")
        bf = dict(dtype=torch.bfloat16, device=self.device)
        s1, s2, s3 = (n, d, h, w), (n, d // 2, h // 2, w // 2), (n, d // 4, h // 4, w // 4)
        B = {"e1a": torch.empty(s1 + (16,), **bf), "s1": torch.empty(s1 + (16,), **bf),
             "p1": torch.empty(s2 + (16,), **bf), "e2a": torch.empty(s2 + (32,), **bf),
             "s2": torch.empty(s2 + (32,), **bf), "p2": torch.empty(s3 + (32,), **bf),
             "e3a": torch.empty(s3 + (64,), **bf), "e3b": torch.empty(s3 + (64,), **bf),
             "r3": torch.empty(s3 + (32,), **bf), "a2": torch.empty(s2 + (32,), **bf),
             "d2": torch.empty(s2 + (32,), **bf), "r2": torch.empty(s2 + (16,), **bf),
             "a1": torch.empty(s1 + (16,), **bf), "d1": torch.empty(s1 + (16,), **bf),
             "out": torch.empty(s1, dtype=torch.float32, device=self.device)}
        if train:
            # g_a1 / g_a2 also collect the gradients of the skips s1 / s2
            B.update({"g_out": torch.empty(s1, dtype=torch.float32, device=self.device),
                      "g_d1": torch.empty(s1 + (16,), **bf), "g_a1": torch.empty(s1 + (16,), **bf),
                      "g_r2": torch.empty(s2 + (16,), **bf), "g_d2": torch.empty(s2 + (32,), **bf),
                      "g_a2": torch.empty(s2 + (32,), **bf), "g_r3": torch.empty(s3 + (32,), **bf),
                      "g_e3b": torch.empty(s3 + (64,), **bf), "g_e3a": torch.empty(s3 + (64,), **bf),
                      "g_p2": torch.empty(s3 + (32,), **bf), "g_e2a": torch.empty(s2 + (32,), **bf),
                      "g_p1": torch.empty(s2 + (16,), **bf), "g_e1a": torch.empty(s1 + (16,), **bf)})
        self._bufs[key] = B
        return B

    # kernels ----------------------------------------------------------------
    def _conv(self, name, x, xcs, xoff, y, ycs, yoff, dims):
        _, _, cin, cout = self.off[name]
        n, d, h, w = dims
        relu = int(name not in LINEAR)
        if cin == 1:
            check(_lib.load().cnn_stem_forward(_p(x), _p(self.w16(name)), _p(self.bias(name)), _p(y), ycs, yoff,
                                               n, d, h, w, cout, relu, _stream()))
            return
        check(_lib.load().cnn_conv3d_forward(_p(x), xcs, xoff, _p(self.w16(name)), _p(self.bias(name)),
                                             _p(y), ycs, yoff, 0, n, d, h, w, cin, cout, relu, _stream()))

    def _conv_bwd(self, name, x, xcs, xoff, g, gcs, goff, dx, dxcs, dxoff, dims):
        _, _, cin, cout = self.off[name]
        n, d, h, w = dims
        lib = _lib.load()
        if cin == 1:
            check(lib.cnn_stem_wgrad(_p(x), _p(g), gcs, goff, _p(self.gw(name)), _p(self.gb(name)),
                                     n, d, h, w, cout, _stream()))
            return
        check(lib.cnn_conv3d_wgrad(_p(x), xcs, xoff, _p(g), gcs, goff, _p(self.gw(name)), _p(self.gb(name)),
                                   n, d, h, w, cin, cout, _stream()))
        if dx is not None:
            check(lib.cnn_conv3d_dgrad(_p(g), gcs, goff, _p(self.w16(name)), _p(self.wt), _p(dx), dxcs, dxoff,
                                       n, d, h, w, cin, cout, _stream()))

    def _relu_bwd(self, g, y, nvox, c):
        check(_lib.load().cnn_relu_backward(_p(g), c, 0, _p(y), c, 0, nvox, c, _stream()))

    def forward(self, x: torch.Tensor, train: bool = False) -> torch.Tensor:
        """x: FP32 [N, D, H, W] (or [D, H, W]); returns x + net(x) (FP32)."""
        squeeze = x.dim() == 3
        if squeeze:
            x = x.unsqueeze(0)
        x = x.contiguous()
        n, d, h, w = x.shape
        B = self._buffers((n, d, h, w), train)
        self._x = x
        lib = _lib.load()
        st = _stream()
        l1, l2, l3 = (n, d, h, w), (n, d // 2, h // 2, w // 2), (n, d // 4, h // 4, w // 4)
        if self.has_e1b:
            self._conv("e1a", x, 1, 0, B["e1a"], 16, 0, l1)
            self._conv("e1b", B["e1a"], 16, 0, B["s1"], 16, 0, l1)
            check(lib.cnn_maxpool2_forward(_p(B["s1"]), 16, 0, _p(B["p1"]), *l1, 16, st))
        else:
            # the input layer writes s1 and its pooling p1 in one pass
            check(lib.cnn_stem_pool_forward(_p(x), _p(self.w16("e1a")), _p(self.bias("e1a")), _p(B["s1"]), 16, 0,
                                            _p(B["p1"]), n, d, h, w, 16, 1, st))
        self._conv("e2a", B["p1"], 16, 0, B["e2a"], 32, 0, l2)
        self._conv("e2b", B["e2a"], 32, 0, B["s2"], 32, 0, l2)
        check(lib.cnn_maxpool2_forward(_p(B["s2"]), 32, 0, _p(B["p2"]), *l2, 32, st))
        self._conv("e3a", B["p2"], 32, 0, B["e3a"], 64, 0, l3)
        self._conv("e3b", B["e3a"], 64, 0, B["e3b"], 64, 0, l3)
        self._conv("u3", B["e3b"], 64, 0, B["r3"], 32, 0, l3)
        check(lib.cnn_upsample2_add_forward(_p(B["r3"]), _p(B["s2"]), 32, 0, _p(B["a2"]), 32, 0, *l3, 32, st))
        self._conv("d2", B["a2"], 32, 0, B["d2"], 32, 0, l2)
        self._conv("u2", B["d2"], 32, 0, B["r2"], 16, 0, l2)
        fused = False
        if not self.has_d1 and not train:
            # the head reads up(r2) + s1 straight from its operands (bit for bit the two calls below)
            check(lib.cnn_upsample2_add_head1_forward(_p(B["r2"]), _p(B["s1"]), 16, 0, _p(self.head_w()),
                                                      _p(self.head_b()), _p(x), _p(B["out"]), *l2, 16, st))
            out = B["out"]
            return out[0] if squeeze else out
        check(lib.cnn_upsample2_add_forward(_p(B["r2"]), _p(B["s1"]), 16, 0, _p(B["a1"]), 16, 0, *l2, 16, st))
        if not self.has_d1:
            # the head reads a1 directly
            check(lib.cnn_head1_forward(_p(B["a1"]), 16, _p(self.head_w()), _p(self.head_b()), _p(x),
                                        _p(B["out"]), n * d * h * w, HEAD_CIN, st))
            fused = True
        if not train and not fused:
            # d1 and the head in one kernel where the persistent tcgen05 convolution takes the layer
            r = lib.cnn_conv3d_forward_head(_p(B["a1"]), 16, 0, _p(self.w16("d1")), _p(self.bias("d1")),
                                            _p(self.head_w()), _p(self.head_b()), _p(x), _p(B["out"]),
                                            n, d, h, w, 16, 16, 1, st)
            if r != _lib.BP_ERR_UNSUPPORTED:
                check(r)
                fused = True
        if not fused:
            self._conv("d1", B["a1"], 16, 0, B["d1"], 16, 0, l1)
            check(lib.cnn_head1_forward(_p(B["d1"]), 16, _p(self.head_w()), _p(self.head_b()), _p(x),
                                        _p(B["out"]), n * d * h * w, HEAD_CIN, st))
        out = B["out"]
        return out[0] if squeeze else out

    def backward(self, g_out: torch.Tensor):
        """Accumulate parameter gradients for dL/d(out) = g_out (FP32, shape of out)."""
        x = self._x
        n, d, h, w = x.shape
        B = self._buffers((n, d, h, w), True)
        lib = _lib.load()
        st = _stream()
        l1, l2, l3 = (n, d, h, w), (n, d // 2, h // 2, w // 2), (n, d // 4, h // 4, w // 4)
        v1, v2, v3 = n * d * h * w, n * d * h * w // 8, n * d * h * w // 64
        gw_head = self.grads[self.head_off:self.head_off + HEAD_CIN]
        gb_head = self.grads[self.head_off + HEAD_CIN:self.head_off + HEAD_CIN + 1]
        if self.has_d1:
            check(lib.cnn_head1_backward(_p(B["d1"]), 16, _p(self.head_w()), _p(g_out.contiguous()), _p(B["g_d1"]),
                                         16, _p(gw_head), _p(gb_head), v1, HEAD_CIN, st))
            self._relu_bwd(B["g_d1"], B["d1"], v1, 16)
            self._conv_bwd("d1", B["a1"], 16, 0, B["g_d1"], 16, 0, B["g_a1"], 16, 0, l1)
        else:
            check(lib.cnn_head1_backward(_p(B["a1"]), 16, _p(self.head_w()), _p(g_out.contiguous()), _p(B["g_a1"]),
                                         16, _p(gw_head), _p(gb_head), v1, HEAD_CIN, st))
        # a1 = up(r2) + s1: g_r2 sums the eight children, g_s1 starts as g_a1
        check(lib.cnn_upsample2_backward(_p(B["g_a1"]), 16, 0, _p(B["g_r2"]), *l2, 16, st))
        self._conv_bwd("u2", B["d2"], 32, 0, B["g_r2"], 16, 0, B["g_d2"], 32, 0, l2)
        self._relu_bwd(B["g_d2"], B["d2"], v2, 32)
        self._conv_bwd("d2", B["a2"], 32, 0, B["g_d2"], 32, 0, B["g_a2"], 32, 0, l2)
        check(lib.cnn_upsample2_backward(_p(B["g_a2"]), 32, 0, _p(B["g_r3"]), *l3, 32, st))
        self._conv_bwd("u3", B["e3b"], 64, 0, B["g_r3"], 32, 0, B["g_e3b"], 64, 0, l3)
        self._relu_bwd(B["g_e3b"], B["e3b"], v3, 64)
        self._conv_bwd("e3b", B["e3a"], 64, 0, B["g_e3b"], 64, 0, B["g_e3a"], 64, 0, l3)
        self._relu_bwd(B["g_e3a"], B["e3a"], v3, 64)
        self._conv_bwd("e3a", B["p2"], 32, 0, B["g_e3a"], 64, 0, B["g_p2"], 32, 0, l3)
        # s2 feeds the pool and the skip: the pooled branch's gradient is added to g_a2
        check(lib.cnn_maxpool2_backward(_p(B["s2"]), 32, 0, _p(B["g_p2"]), _p(B["g_a2"]), 32, 0, *l2, 32, st))
        self._relu_bwd(B["g_a2"], B["s2"], v2, 32)
        self._conv_bwd("e2b", B["e2a"], 32, 0, B["g_a2"], 32, 0, B["g_e2a"], 32, 0, l2)
        self._relu_bwd(B["g_e2a"], B["e2a"], v2, 32)
        self._conv_bwd("e2a", B["p1"], 16, 0, B["g_e2a"], 32, 0, B["g_p1"], 16, 0, l2)
        check(lib.cnn_maxpool2_backward(_p(B["s1"]), 16, 0, _p(B["g_p1"]), _p(B["g_a1"]), 16, 0, *l1, 16, st))
        self._relu_bwd(B["g_a1"], B["s1"], v1, 16)
        if self.has_e1b:
            self._conv_bwd("e1b", B["e1a"], 16, 0, B["g_a1"], 16, 0, B["g_e1a"], 16, 0, l1)
            self._relu_bwd(B["g_e1a"], B["e1a"], v1, 16)
            self._conv_bwd("e1a", x, 1, 0, B["g_e1a"], 16, 0, None, 0, 0, l1)
        else:
            self._conv_bwd("e1a", x, 1, 0, B["g_a1"], 16, 0, None, 0, 0, l1)

    def adam_step(self, lr: float = 1e-3, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.t += 1
        check(_lib.load().cnn_adam(_p(self.params), _p(self.grads), _p(self.m), _p(self.v), _p(self.params16),
                                   self.n_params, ctypes.c_float(lr), ctypes.c_float(b1), ctypes.c_float(b2),
                                   ctypes.c_float(eps), self.t, _stream()))

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float = 1e-3) -> float:
        """One forward, MSE loss, backward and Adam step; returns the loss."""
        out = self.forward(x, train=True)
        if x.dim() == 3:
            out = out.unsqueeze(0)
            target = target.unsqueeze(0)
        B = self._buffers(tuple(out.shape), True)
        self.loss_buf.zero_()
        check(_lib.load().cnn_mse(_p(out), _p(target.contiguous()), _p(B["g_out"]), _p(self.loss_buf),
                                  out.numel(), _stream()))
        self.backward(B["g_out"])
        self.adam_step(lr)
        return float(self.loss_buf.item()) / out.numel()


__all__ = ["UNet", "LAYERS", "conv_flops"]
