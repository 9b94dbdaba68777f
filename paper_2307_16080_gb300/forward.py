"""A chained forward through the 20-layer ResNet-style conv stack, built from
library calls only (nk_conv2d_nhwc_hwcf with BF16 outputs and fused
programs; no arithmetic here).

The producer -> consumer chain is that of the lowered Linear layer of
Sec. 2.1.2 (the contraction's output feeds the next op), with the
conv_2d_nhwc_hwcf of Sec. 4.1 as the op:

  stage 56x56 (64 channels):   x -> 3x3 -> 3x3 -> 3x3 -> 3x3
  each later stage (128 @ 28, 256 @ 14, 512 @ 7), input s:
      a = 3x3 stride 2 (s)            BF16, bias + ReLU
      p = 1x1 stride 2 (s)            FP32, bias (the projection shortcut)
      b = 3x3 (a), c = 3x3 (b)        BF16, bias + ReLU
      d = ReLU(3x3 (c) + bias + p)    BF16: a fused ADD of p, then ReLU
  head: 1x1 512 -> 512 on the last d   FP32, bias + ReLU

Every BF16 output is the epilogue's FP32 value rounded once (RNE), and the
next layer reads it as its BF16 input: the FP32 -> BF16 hand-off of a real
forward is paid inside the producing kernel.  The layer list is
synth.resnet_stack(batch), in the same order.
"""
from __future__ import annotations

import math

import torch

from . import nk, synth


class ResNetStack:
    """Weights packed to BF16 once; activations in preallocated buffers, so
    run() issues 20 library calls that a CUDA graph can capture."""

    def __init__(self, batch: int, device, seed: int = synth.SEED_COSTMODEL, schedules=None):
        self.batch = batch
        self.dev = torch.device(device)
        self.layers = synth.resnet_stack(batch)
        self.calls = []       # (I, W, O, stride, pad, bias, ew, relu, schedule, ws)
        self.flop = 0.0
        self.kernels = 0
        self.weights32, self.bias32 = [], []
        for li, L in enumerate(self.layers):
            w = synth.normal(seed, 2 * li, (L["KH"], L["KW"], L["C"], L["F"]),
                             sigma=math.sqrt(2.0 / (L["KH"] * L["KW"] * L["C"])))
            b = synth.uniform(seed, 2 * li + 1, (L["F"],), -0.1, 0.1)
            self.weights32.append(w)
            self.bias32.append(b)
        self.schedules = schedules or [None] * len(self.layers)
        self.x = None

    @staticmethod
    def _out_hw(L):
        return (L["H"] + 2 * L["pad"] - L["KH"]) // L["stride"] + 1

    def bind(self, x: torch.Tensor):
        """x: BF16 NHWC [batch, 56, 56, 64] input.  Builds every call."""
        assert x.dtype == torch.bfloat16 and tuple(x.shape) == (self.batch, 56, 56, 64)
        self.x = x
        self.calls, self.outputs = [], []
        cur, stage_in = x, x
        proj = None
        for li, (L, sched) in enumerate(zip(self.layers, self.schedules)):
            oh = self._out_hw(L)
            wp = nk.nk_conv2d_pack_weights(torch.from_numpy(self.weights32[li]).to(self.dev))
            bias = torch.from_numpy(self.bias32[li]).to(self.dev)
            st, pad = (L["stride"],) * 2, (L["pad"],) * 4
            role = self.role(li)
            if role == "projection":
                src, out = stage_in, torch.empty(self.batch, oh, oh, L["F"], device=self.dev)
                relu, ew = False, None
            elif role == "head":
                src, out = cur, torch.empty(self.batch, oh, oh, L["F"], device=self.dev)
                relu, ew = True, None
            elif role == "residual":
                src = cur
                out = torch.empty(self.batch, oh, oh, L["F"], device=self.dev, dtype=torch.bfloat16)
                relu, ew = False, [("add", proj), ("relu",)]
            else:   # "plain" or "downsample"
                src = stage_in if role == "downsample" else cur
                out = torch.empty(self.batch, oh, oh, L["F"], device=self.dev, dtype=torch.bfloat16)
                relu, ew = True, None
            ws = nk.workspace(nk.nk_conv2d_workspace_size(src, wp, out, st, (1, 1), pad, "bf16", sched), self.dev)
            self.calls.append((src, wp, out, st, pad, bias, ew, relu, sched, ws))
            self.outputs.append(out)
            self.flop += 2.0 * self.batch * oh * oh * L["F"] * L["KH"] * L["KW"] * L["C"]
            if role == "projection":
                proj = out
            else:
                cur = out
                if role in ("residual",) or (role == "plain" and li == 3):
                    stage_in = out
        # one kernel per layer, plus the reduce of a split-K schedule
        from . import nk_tune as nt
        self.kernels = 0
        for L, sched in zip(self.layers, self.schedules):
            s = sched or nt.nk_default_schedule(nt.conv_problem(L["N"], L["H"], L["W"], L["C"], L["F"], L["KH"],
                                                                L["KW"], L["stride"], L["pad"]))
            self.kernels += 2 if s[5] > 1 else 1
        return self

    def role(self, li: int) -> str:
        """Position of layer li in the chain (the stack's fixed order)."""
        if li < 4:
            return "plain"
        if li == 19:
            return "head"
        k = (li - 4) % 5
        return ("downsample", "projection", "plain", "plain", "residual")[k]

    def run(self, stream=None):
        for (src, wp, out, st, pad, bias, ew, relu, sched, ws) in self.calls:
            nk.nk_conv2d_nhwc_hwcf(src, wp, out, st, (1, 1), pad, "bf16", bias=bias, relu=relu, ew=ew,
                                   schedule=sched, ws=ws, stream=stream)

    def layer_inputs(self, li: int):
        """(input tensor, residual operand or None) of layer li, as bound."""
        src, _, _, _, _, _, ew, _, _, _ = self.calls[li]
        return src, (ew[0][1] if ew else None)

