"""Learned denoiser of harmonic radiance maps: a U-Net on the hand-written BF16 tensor-core kernels.

The forward and adjoint MC (Secs. 3-4) deliver per-pixel Fourier coefficients a_0, a_n, b_n
(Eqs. 8-11) whose noise falls like 1/sqrt(N_p).  The denoiser maps a low-packet-count map
(2K+1 channels) to an estimate of the high-count map, trained on pairs the MC itself generates;
full-count MC remains the reference that measures its error.  (The paper has no learned part.)

Architecture: 4 levels with 32/64/128/256 channels, two 3x3 convolutions + ReLU per level,
2x2 average pooling down, nearest 2x up-sampling + skip concatenation up, a 1x1 output head, and
a residual output y = x + f(x).  Inputs are scaled per sample by 1 / mean(a_0).  Every operation
runs in libmcr kernels (include/mcr_denoise.h): convolutions, input gradients and weight
gradients on tcgen05 tensor cores (BF16 operands, FP32 accumulation), the rest memory-bound.
"""
from __future__ import annotations

import math

import torch

from . import denoise_ops as ops
from .denoise_ops import Act


def r64(c):
    return (c + 63) // 64 * 64


def r16(c):
    return (c + 15) // 16 * 16


def r8(c):
    return (c + 7) // 8 * 8


class Conv:
    """One convolution layer: FP32 master weights [cout][taps][cin] + bias, Adam state, and the
    BF16 copies for the forward pass ([n_pad][taps][cin_pad]) and the input-gradient pass
    ([r16(cin)][taps][r64(cout)], taps flipped)."""

    def __init__(self, name, cin, cout, taps, relu, gen, device, init_std=None):
        self.name, self.cin, self.cout, self.taps, self.relu = name, cin, cout, taps, relu
        self.cin_pad, self.n_pad, self.dz_stride = r64(cin), r16(cout), r64(cout)
        std = init_std if init_std is not None else math.sqrt(2.0 / (taps * cin))
        w = torch.randn(cout, taps, cin, generator=gen) * std
        self.w = w.to(device)
        self.b = torch.zeros(cout, device=device)
        self.m, self.v = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.gw, self.gb = torch.zeros_like(self.w), torch.zeros_like(self.b)
        self.wf = torch.zeros(self.n_pad, taps, self.cin_pad, dtype=torch.bfloat16, device=device)
        self.wd = torch.zeros(r16(cin), taps, self.dz_stride, dtype=torch.bfloat16, device=device)
        self.refresh()

    def refresh(self):
        """Write the BF16 copies from the master weights (no update)."""
        ops.adam(self.w, self.m, self.v, self.gw, self.cout, self.taps, self.cin, 0.0, 0.9, 0.999, 1e-8, 0,
                 self.wf, self.cin_pad, self.wd, self.dz_stride)

    def step(self, lr, t, b1=0.9, b2=0.999, eps=1e-8):
        ops.adam(self.w, self.m, self.v, self.gw, self.cout, self.taps, self.cin, lr, b1, b2, eps, t, self.wf,
                 self.cin_pad, self.wd, self.dz_stride)
        ops.adam_bias(self.b, self.mb, self.vb, self.gb, lr, b1, b2, eps, t)

    def adam_entry(self):
        """This layer's descriptor for the multi-tensor Adam step (``ops.adam_table``)."""
        return (self.w, self.m, self.v, self.gw, self.wf, self.cin_pad, self.wd, self.dz_stride, self.cout, self.taps,
                self.cin, self.b, self.mb, self.vb, self.gb)

    def forward(self, x: torch.Tensor, out: Act, f32: bool = False):
        assert x.shape[3] == self.cin_pad, (self.name, x.shape, self.cin_pad)
        ops.conv(x, self.wf, self.cout, out.t, taps=self.taps, bias=self.b, relu=self.relu, out_off=out.off,
                 cin=self.cin)

    def input_grad(self, dz: torch.Tensor, dx: torch.Tensor, mask: torch.Tensor | None):
        """dx[..., :cin] = conv(dz, flipped W^T), times (mask > 0) if a mask is given."""
        for c0 in range(0, self.cin, 256):
            n = min(256, self.cin - c0)
            ops.conv(dz, self.wd[c0:c0 + r16(n)], n, dx, taps=self.taps, mask=mask, mask_off=c0, out_off=c0,
                     cin=self.cout)


LAYERS = [  # name, input, output (buffer, offset), cin, cout, taps, relu
    ("e0a", "x0", ("e0a", 0), "in", 0, 9, True),
    ("e0b", "e0a", ("cat0", 64), 0, 0, 9, True),
    ("e1a", "p0", ("e1a", 0), 0, 1, 9, True),
    ("e1b", "e1a", ("cat1", 128), 1, 1, 9, True),
    ("e2a", "p1", ("e2a", 0), 1, 2, 9, True),
    ("e2b", "e2a", ("cat2", 256), 2, 2, 9, True),
    ("ma", "p2", ("ma", 0), 2, 3, 9, True),
    ("mb", "ma", ("mb", 0), 3, 3, 9, True),
    ("d2a", "cat2", ("d2a", 0), "32", 2, 9, True),
    ("d2b", "d2a", ("d2b", 0), 2, 2, 9, True),
    ("d1a", "cat1", ("d1a", 0), "21", 1, 9, True),
    ("d1b", "d1a", ("d1b", 0), 1, 1, 9, True),
    ("d0a", "cat0", ("d0a", 0), "10", 0, 9, True),
    ("d0b", "d0a", ("d0b", 0), 0, 0, 9, True),
    ("out", "d0b", ("out", 0), 0, "in", 1, False),
]


class UNet:
    """4-level U-Net on (2K+1)-channel harmonic maps, trained and run with libmcr kernels only."""

    def __init__(self, in_ch: int = 33, base: int = 32, seed: int = 0, device="cuda"):
        self.in_ch = in_ch
        self.ch = [base, 2 * base, 4 * base, 8 * base]
        assert base % 32 == 0 and 8 * base <= 256, "channel counts must fit one MMA N (<= 256)"
        gen = torch.Generator().manual_seed(seed)
        self.device = torch.device(device)

        def chans(spec):
            if spec == "in":
                return in_ch
            if isinstance(spec, int):
                return self.ch[spec]
            return self.ch[int(spec[0])] + self.ch[int(spec[1])]

        self._adam = None  # multi-tensor Adam descriptors, built on the first step
        self.layers = {}
        for name, src, dst, ci, co, taps, relu in LAYERS:
            std = 1e-3 if name == "out" else None
            self.layers[name] = Conv(name, chans(ci), chans(co), taps, relu, gen, self.device, init_std=std)
        self.t = 0
        self._shape = None

    # ------------------------------------------------------------------ buffers
    def _alloc(self, B, H, W):
        if self._shape == (B, H, W):
            return
        assert H % 8 == 0 and W % 8 == 0 and W // 8 >= 16, "levels need W/8 >= 16"
        dev, c = self.device, self.ch
        z = lambda h, w, s: torch.zeros(B, h, w, s, dtype=torch.bfloat16, device=dev)
        L = [(H, W), (H // 2, W // 2), (H // 4, W // 4), (H // 8, W // 8)]
        a = {}
        a["x0"] = z(*L[0], r64(self.in_ch))
        a["e0a"] = z(*L[0], r64(c[0]))
        a["cat0"] = z(*L[0], r64(c[1] + c[0]))
        a["p0"] = z(*L[1], r64(c[0]))
        a["e1a"] = z(*L[1], r64(c[1]))
        a["cat1"] = z(*L[1], r64(c[2] + c[1]))
        a["p1"] = z(*L[2], r64(c[1]))
        a["e2a"] = z(*L[2], r64(c[2]))
        a["cat2"] = z(*L[2], r64(c[3] + c[2]))
        a["p2"] = z(*L[3], r64(c[2]))
        a["ma"] = z(*L[3], r64(c[3]))
        a["mb"] = z(*L[3], r64(c[3]))
        a["d2a"] = z(*L[2], r64(c[2]))
        a["d2b"] = z(*L[2], r64(c[2]))
        a["d1a"] = z(*L[1], r64(c[1]))
        a["d1b"] = z(*L[1], r64(c[1]))
        a["d0a"] = z(*L[0], r64(c[0]))
        a["d0b"] = z(*L[0], r64(c[0]))
        a["out"] = torch.zeros(B, *L[0], r8(self.in_ch), device=dev)
        self.a = a
        # gradients: dZ of every layer (stride r64(cout)) and the routed input gradients
        g = {name: torch.zeros(B, *L[self._level(name)], r64(lay.cout), dtype=torch.bfloat16, device=dev)
             for name, lay in self.layers.items()}
        g["dcat0"], g["dcat1"], g["dcat2"] = (torch.zeros_like(a["cat0"]), torch.zeros_like(a["cat1"]),
                                              torch.zeros_like(a["cat2"]))
        g["dp0"], g["dp1"], g["dp2"] = torch.zeros_like(a["p0"]), torch.zeros_like(a["p1"]), torch.zeros_like(a["p2"])
        self.g = g
        P = B * H * W
        self.target = torch.zeros(B, H, W, self.in_ch, device=dev)
        self.loss = torch.zeros((), dtype=torch.float64, device=dev)
        self.pred = torch.zeros(B, self.in_ch, H, W, device=dev)
        self._shape = (B, H, W)

    @staticmethod
    def _level(name):
        return {"e0a": 0, "e0b": 0, "e1a": 1, "e1b": 1, "e2a": 2, "e2b": 2, "ma": 3, "mb": 3, "d2a": 2, "d2b": 2,
                "d1a": 1, "d1b": 1, "d0a": 0, "d0b": 0, "out": 0}[name]

    # ------------------------------------------------------------------ passes
    def load(self, x: torch.Tensor, scale: torch.Tensor, target: torch.Tensor | None = None):
        """x, target: channel-major fp32 [B][in_ch][H][W] maps; scale: fp32 [B] per-sample factors."""
        B, C, H, W = x.shape
        assert C == self.in_ch
        self._alloc(B, H, W)
        ops.pack_input(x.contiguous(), scale, self.a["x0"])
        if target is not None:
            ops.pack_target(target.contiguous(), scale, self.target)

    def forward(self):
        """The network on the loaded input; returns the NHWC fp32 output of the 1x1 head."""
        self._trunk()
        a, o = self.a, self.layers["out"]
        ops.conv(a["d0b"], o.wf, o.cout, a["out"], taps=1, bias=o.b, relu=False)
        return a["out"]

    def _trunk(self):
        """Every layer but the 1x1 output head (its input is a["d0b"])."""
        a, L, c = self.a, self.layers, self.ch
        L["e0a"].forward(a["x0"], Act(a["e0a"], c[0]))
        L["e0b"].forward(a["e0a"], Act(a["cat0"], c[0], c[1]))
        ops.pool2(Act(a["cat0"], c[0], c[1]), Act(a["p0"], c[0]))
        L["e1a"].forward(a["p0"], Act(a["e1a"], c[1]))
        L["e1b"].forward(a["e1a"], Act(a["cat1"], c[1], c[2]))
        ops.pool2(Act(a["cat1"], c[1], c[2]), Act(a["p1"], c[1]))
        L["e2a"].forward(a["p1"], Act(a["e2a"], c[2]))
        L["e2b"].forward(a["e2a"], Act(a["cat2"], c[2], c[3]))
        ops.pool2(Act(a["cat2"], c[2], c[3]), Act(a["p2"], c[2]))
        L["ma"].forward(a["p2"], Act(a["ma"], c[3]))
        L["mb"].forward(a["ma"], Act(a["mb"], c[3]))
        ops.up2(Act(a["mb"], c[3]), Act(a["cat2"], c[3], 0))
        L["d2a"].forward(a["cat2"], Act(a["d2a"], c[2]))
        L["d2b"].forward(a["d2a"], Act(a["d2b"], c[2]))
        ops.up2(Act(a["d2b"], c[2]), Act(a["cat1"], c[2], 0))
        L["d1a"].forward(a["cat1"], Act(a["d1a"], c[1]))
        L["d1b"].forward(a["d1a"], Act(a["d1b"], c[1]))
        ops.up2(Act(a["d1b"], c[1]), Act(a["cat0"], c[1], 0))
        L["d0a"].forward(a["cat0"], Act(a["d0a"], c[0]))
        L["d0b"].forward(a["d0a"], Act(a["d0b"], c[0]))

    def _wgrad(self, lay: Conv, dz: torch.Tensor, x: Act):
        # straight from the NHWC activations (MN-major operands, no transposed copies)
        ops.wgrad_nhwc(Act(dz, lay.cout), x, lay.taps, lay.gw, db=lay.gb)  # + the bias gradient

    def backward(self):
        """Gradients of the loss computed by the last ``loss()`` into every layer's gw, gb."""
        a, g, L, c = self.a, self.g, self.layers, self.ch
        chain = [  # layer, its input (Act), input-gradient destination, ReLU mask of the input
            ("out", Act(a["d0b"], c[0]), g["d0b"], a["d0b"]),
            ("d0b", Act(a["d0a"], c[0]), g["d0a"], a["d0a"]),
            ("d0a", Act(a["cat0"], c[1] + c[0]), g["dcat0"], None),
        ]
        for name, x, dx, mask in chain:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.up2_bwd(Act(g["dcat0"], c[1], 0), Act(a["d1b"], c[1]), Act(g["d1b"], c[1]))
        for name, x, dx, mask in [("d1b", Act(a["d1a"], c[1]), g["d1a"], a["d1a"]),
                                  ("d1a", Act(a["cat1"], c[2] + c[1]), g["dcat1"], None)]:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.up2_bwd(Act(g["dcat1"], c[2], 0), Act(a["d2b"], c[2]), Act(g["d2b"], c[2]))
        for name, x, dx, mask in [("d2b", Act(a["d2a"], c[2]), g["d2a"], a["d2a"]),
                                  ("d2a", Act(a["cat2"], c[3] + c[2]), g["dcat2"], None)]:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.up2_bwd(Act(g["dcat2"], c[3], 0), Act(a["mb"], c[3]), Act(g["mb"], c[3]))
        for name, x, dx, mask in [("mb", Act(a["ma"], c[3]), g["ma"], a["ma"]),
                                  ("ma", Act(a["p2"], c[2]), g["dp2"], None)]:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.pool2_bwd(Act(g["dp2"], c[2]), Act(g["dcat2"], c[2], c[3]), Act(a["cat2"], c[2], c[3]),
                      Act(g["e2b"], c[2]))
        for name, x, dx, mask in [("e2b", Act(a["e2a"], c[2]), g["e2a"], a["e2a"]),
                                  ("e2a", Act(a["p1"], c[1]), g["dp1"], None)]:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.pool2_bwd(Act(g["dp1"], c[1]), Act(g["dcat1"], c[1], c[2]), Act(a["cat1"], c[1], c[2]),
                      Act(g["e1b"], c[1]))
        for name, x, dx, mask in [("e1b", Act(a["e1a"], c[1]), g["e1a"], a["e1a"]),
                                  ("e1a", Act(a["p0"], c[0]), g["dp0"], None)]:
            self._wgrad(L[name], g[name], x)
            L[name].input_grad(g[name], dx, mask)
        ops.pool2_bwd(Act(g["dp0"], c[0]), Act(g["dcat0"], c[0], c[1]), Act(a["cat0"], c[0], c[1]),
                      Act(g["e0b"], c[0]))
        self._wgrad(L["e0b"], g["e0b"], Act(a["e0a"], c[0]))
        L["e0b"].input_grad(g["e0b"], g["e0a"], a["e0a"])
        self._wgrad(L["e0a"], g["e0a"], Act(a["x0"], self.in_ch))

    def loss_and_grad_seed(self):
        """Residual MSE of the last forward pass against the loaded target; seeds the backward pass."""
        ops.mse(self.a["out"], self.a["x0"], self.target, self.in_ch, self.g["out"], self.loss)
        return self.loss

    def step(self, lr: float):
        """One Adam step of every layer (weights, biases, bf16 copies) in one launch."""
        self.t += 1
        if self._adam is None:
            self._adam = ops.adam_table([lay.adam_entry() for lay in self.layers.values()])
        ops.adam_multi(self._adam, lr, 0.9, 0.999, 1e-8, self.t)

    def train_step(self, x, scale, target, lr):
        """One Adam step on the residual MSE against scale * target; returns the loss (device FP64).
        The head's epilogue computes the loss and its gradient seed from the channel-major target
        (no packed target copy, no fp32 network output)."""
        self.load(x, scale)
        self._trunk()
        o = self.layers["out"]
        ops.conv_head(self.a["d0b"], o.wf, o.cout, o.b, self.a["x0"], scale, target=target.contiguous(),
                      dout=self.g["out"], loss=self.loss)
        self.backward()
        self.step(lr)
        return self.loss

    def predict(self, x: torch.Tensor, scale: torch.Tensor) -> torch.Tensor:
        """Denoised channel-major maps [B][in_ch][H][W] (unscaled), written by the head's epilogue."""
        self.load(x, scale)
        self._trunk()
        o = self.layers["out"]
        ops.conv_head(self.a["d0b"], o.wf, o.cout, o.b, self.a["x0"], scale, pred=self.pred)
        return self.pred

    # ------------------------------------------------------------------ state
    def state(self):
        return {name: (lay.w.detach().cpu().clone(), lay.b.detach().cpu().clone()) for name, lay in self.layers.items()}

    def set_state(self, state):
        for name, (w, b) in state.items():
            self.layers[name].w.copy_(w.to(self.device))
            self.layers[name].b.copy_(b.to(self.device))
            self.layers[name].refresh()


def sample_scale(x: torch.Tensor) -> torch.Tensor:
    """Per-sample scale 1 / mean(a_0) (channel 0) so that inputs have unit mean fluence."""
    x = x.contiguous()
    scale = torch.empty(x.shape[0], device=x.device, dtype=torch.float32)
    ops.sample_scale(x, scale)
    return scale
