"""Seeded sweep of E4M3 convolutions on pre-quantised operands (filters
packed once by nk_conv2d_pack_weights_fp8, the input quantised by nk_amax +
nk_cast_fp8), through the built-in dispatch, bitwise against the oracle,
with canary-padded outputs.

Half-integer entries with |x| <= 3.5 and amax 3.5 in both operands give the
scale 448 / 3.5 = 128, and every x * 128 is an E4M3 code, so quantisation
is exact and the FP32 result (sum of code products times 1 / 128^2) is
exact too.  C >= 128 reaches the E4M3 stacked window kernel (stride 1,
2 <= KW <= 4), C = 64 the per-tap kernel; outputs FP32 or BF16.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, Canary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _case(i):
    u = synth.uniform01(221, i, 14)
    kh, kw = 2 + int(u[0] * 3), 2 + int(u[1] * 3)
    dl = (1 + int(u[2] * 2), 1) if u[3] < 0.3 else (1, 1)
    pad = (int(u[4] * kh), int(u[5] * kh), int(u[6] * kw), int(u[7] * kw))
    h = (kh - 1) * dl[0] + 1 + int(u[8] * 16)
    w = (kw - 1) * dl[1] + 1 + int(u[9] * 16)
    n = 1 + int(u[10] * 4)
    c = [64, 128, 136, 256][int(u[11] * 4)]
    f = [16, 40, 64, 96, 130][int(u[12] * 5)]
    return n, h, w, c, f, kh, kw, dl, pad


@pytest.mark.parametrize("i", range(40))
def test_prequantised_e4m3_conv_bitwise(nk, i):
    n, h, w, c, f, kh, kw, dl, pad = _case(i)
    I = synth.small_ints(222, 2 * i, (n, h, w, c)) / 2
    W = synth.small_ints(222, 2 * i + 1, (kh, kw, c, f)) / 2
    I.flat[0], W.flat[0] = 3.5, -3.5
    iq, si = nk.quantize_nhwc_fp8(torch.from_numpy(I).to(DEV))
    wq, sw = nk.nk_conv2d_pack_weights_fp8(torch.from_numpy(W).to(DEV))
    s_i, s_w = float(si.item()), float(sw.item())
    assert s_i == 128.0 and s_w == 128.0
    R = O.conv2d_nhwc_hwcf(I, W, (1, 1), dl, pad)
    shape = R.shape
    for odt in (torch.float32, torch.bfloat16):
        can = Canary(shape, odt)
        nk.nk_conv2d_nhwc_hwcf(iq, wq, can.t, dilation=dl, pad=pad, precision="fp8", scale_i=s_i, scale_w=s_w)
        nk.nk_sync_status()
        can.check()
        want = O.bf16_rn(R) if odt == torch.bfloat16 else R
        np.testing.assert_array_equal(can.t.float().cpu().numpy(), want, err_msg=str((i, n, h, w, c, f, kh, kw, dl,
                                                                                      pad, str(odt))))
