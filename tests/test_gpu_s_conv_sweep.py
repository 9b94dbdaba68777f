"""Seeded sweep of random small convolutions through the built-in dispatch
(the schedule a caller gets without tuning), bitwise against the oracle.

Each geometry draws N, H, W, C, F, KH, KW, stride, dilation and four
independent pads, so the dispatcher lands on every kernel family: per-tap
(any stride), plain and stacked windows, whole-width stacked tiles, split-K.
Entries are small integers (FP32, BF16; BF16 outputs compared after the
oracle's own rounding) or half-integers with amax 3.5 (E4M3 quantised per
call: scale 128, exact codes), so every result is exact whatever the order.
Outputs sit inside canary-filled buffers, so a write past either end of the
tensor (a ragged last tile) fails too.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, Canary

pytestmark = pytest.mark.gpu

NGEOM = 120


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _geometries():
    u = synth.uniform01(171, 0, 12 * NGEOM)
    out = []
    for g in range(NGEOM):
        r = u[12 * g: 12 * g + 12]
        kh, kw = 1 + int(r[0] * 4), 1 + int(r[1] * 4)
        sh, sw = 1 + int(r[2] * 2), 1 + int(r[3] * 2)
        dh, dw = (1 + int(r[4] * 2), 1 + int(r[5] * 2)) if sh == 1 and sw == 1 else (1, 1)
        pad = (int(r[6] * kh), int(r[7] * kh), int(r[8] * kw), int(r[9] * kw))
        h = (kh - 1) * dh + 1 + int(r[10] * 20)
        w = (kw - 1) * dw + 1 + int(r[11] * 20)
        n = 1 + int(r[0] * 10) % 3
        c = [3, 8, 16, 40, 64, 72, 128, 136][int(r[5] * 8)]
        f = [5, 16, 24, 64, 72, 130][int(r[9] * 6)]
        out.append((n, h, w, c, f, kh, kw, (sh, sw), (dh, dw), pad))
    return out


GEOMS = _geometries()


def _out_shape(n, h, w, f, kh, kw, st, dl, pad):
    oh = O.conv_out_size(h, kh, st[0], dl[0], pad[0], pad[1])
    ow = O.conv_out_size(w, kw, st[1], dl[1], pad[2], pad[3])
    return (n, oh, ow, f)


@pytest.mark.parametrize("prec,odt", [("f32", torch.float32), ("bf16", torch.float32), ("bf16", torch.bfloat16),
                                      ("fp8", torch.float32)])
def test_random_convolutions_bitwise(nk, prec, odt):
    ran, bad = 0, []
    for gi, (n, h, w, c, f, kh, kw, st, dl, pad) in enumerate(GEOMS):
        shape = _out_shape(n, h, w, f, kh, kw, st, dl, pad)
        if min(shape) < 1:
            continue
        I = synth.small_ints(172, 2 * gi, (n, h, w, c))
        W = synth.small_ints(172, 2 * gi + 1, (kh, kw, c, f))
        if prec == "fp8":   # half-integers with amax 3.5 in both: scale 128, exact E4M3 codes
            I, W = I / 2, W / 2
            I.flat[0], W.flat[0] = 3.5, -3.5
        R = O.conv2d_nhwc_hwcf(I, W, st, dl, pad)
        if odt == torch.bfloat16:
            R = O.bf16_rn(R)
        can = Canary(shape, odt)   # contiguous NHWC inside sentinels: catches writes past either end
        out = can.t
        try:
            nk.nk_conv2d_nhwc_hwcf(torch.from_numpy(I).to(DEV), torch.from_numpy(W).to(DEV), out, stride=st,
                                   dilation=dl, pad=pad, precision=prec)
            nk.nk_sync_status()
        except nk.NkError as e:
            if prec == "fp8" or odt == torch.bfloat16:   # paths with documented shape limits
                continue
            raise AssertionError(f"geometry {gi} {GEOMS[gi]}: {e}")
        ran += 1
        can.check()
        if not np.array_equal(out.float().cpu().numpy(), R):
            bad.append(gi)
    assert not bad, f"{len(bad)} geometries differ, first {[GEOMS[i] for i in bad[:3]]}"
    assert ran >= NGEOM // 2, ran
