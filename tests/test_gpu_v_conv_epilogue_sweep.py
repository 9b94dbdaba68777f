"""Seeded sweeps of convolution epilogues and of grouped convolutions,
bitwise against the oracle, with canary-padded outputs.

* nk_conv2d_nhwc_hwcf through the built-in dispatch with a random
  epilogue: bias, ReLU, accumulate (beta = 1 on the output's own values) and
  the residual program ADD t, RELU, into FP32 or BF16 outputs.  The oracle
  applies them in the order the API defines: ReLU?(beta*O_in + conv + bias),
  then the program, then (BF16 outputs) one rounding.
* nk_conv2d_grouped_plan_*: 1-8 uneven convolutions per launch (strides,
  dilation, pads, ragged C and F), each with its own bias / ReLU /
  accumulate, under the default and an explicit tile.

Entries are small integers, so every result is exact whatever the order.
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


def _geometry(u, strided):
    kh, kw = (3, 3) if u[0] < 0.6 else (1 + int(u[0] * 4), 1 + int(u[1] * 4))
    st = (2, 2) if strided else (1, 1)
    dl = (1, 1) if strided or u[2] < 0.7 else (2, 1)
    pad = (int(u[3] * kh), int(u[4] * kh), int(u[5] * kw), int(u[6] * kw))
    h = (kh - 1) * dl[0] + 1 + int(u[7] * 24)
    w = (kw - 1) * dl[1] + 1 + int(u[8] * 24)
    n = 1 + int(u[9] * 3)
    c = [8, 16, 40, 64, 128, 136][int(u[10] * 6)]
    f = [8, 16, 24, 64, 72, 128][int(u[11] * 6)]
    return n, h, w, c, f, kh, kw, st, dl, pad


def _out_shape(n, h, w, f, kh, kw, st, dl, pad):
    return (n, O.conv_out_size(h, kh, st[0], dl[0], pad[0], pad[1]),
            O.conv_out_size(w, kw, st[1], dl[1], pad[2], pad[3]), f)


@pytest.mark.parametrize("case", range(48))
def test_random_conv_epilogues_bitwise(nk, case):
    u = synth.uniform01(201, case, 20)
    n, h, w, c, f, kh, kw, st, dl, pad = _geometry(u, strided=u[12] < 0.25)
    shape = _out_shape(n, h, w, f, kh, kw, st, dl, pad)
    odt = torch.bfloat16 if u[13] < 0.5 else torch.float32
    I = synth.small_ints(202, 2 * case, (n, h, w, c))
    W = synth.small_ints(202, 2 * case + 1, (kh, kw, c, f))
    bias = synth.small_ints(203, case, (f,)) if u[14] < 0.6 else None
    relu = bool(u[15] < 0.5)
    acc = bool(u[16] < 0.3)
    resid = u[17] < 0.4
    O_in = synth.small_ints(204, case, shape)
    T = synth.small_ints(205, case, shape)
    can = Canary(shape, odt)
    if acc:
        can.t.copy_(torch.from_numpy(O_in).to(DEV).to(odt))
    ew = [("add", torch.from_numpy(T).to(DEV)), ("relu",)] if resid else None
    nk.nk_conv2d_nhwc_hwcf(torch.from_numpy(I).to(DEV), torch.from_numpy(W).to(DEV), can.t, stride=st, dilation=dl,
                           pad=pad, precision="bf16", bias=torch.from_numpy(bias).to(DEV) if bias is not None else None,
                           relu=relu, accumulate=acc, ew=ew)
    nk.nk_sync_status()
    can.check()
    R = O.conv2d_fused(I, W, "bf16", st, dl, pad, o_in=O_in if acc else None, bias=bias, relu=relu,
                       beta=1.0 if acc else 0.0, ew=[("add", T), ("relu",)] if resid else None)
    if odt == torch.bfloat16:
        R = O.bf16_rn(R)
    np.testing.assert_array_equal(can.t.float().cpu().numpy(), R,
                                  err_msg=str((case, shape, kh, kw, st, dl, pad, str(odt), bias is not None, relu, acc,
                                               resid)))


@pytest.mark.parametrize("i", range(12))
def test_random_grouped_convolutions_bitwise(nk, i):
    u = synth.uniform01(211, i, 1 + 20 * 8)
    G = 1 + int(u[0] * 8)
    convs, want, cans = [], [], []
    for g in range(G):
        r = u[1 + 20 * g: 21 + 20 * g]
        n, h, w, c, f, kh, kw, st, dl, pad = _geometry(r, strided=r[12] < 0.3)
        shape = _out_shape(n, h, w, f, kh, kw, st, dl, pad)
        I = synth.small_ints(212 + i, 2 * g, (n, h, w, c))
        W = synth.small_ints(212 + i, 2 * g + 1, (kh, kw, c, f))
        bias = synth.small_ints(230 + i, g, (f,)) if r[14] < 0.6 else None
        relu, acc = bool(r[15] < 0.5), bool(r[16] < 0.3)
        O_in = synth.small_ints(240 + i, g, shape)
        can = Canary(shape)
        cans.append((can, O_in, acc))
        convs.append(dict(I=torch.from_numpy(I).to(DEV).to(torch.bfloat16),
                          W=nk.nk_conv2d_pack_weights(torch.from_numpy(W).to(DEV)), O=can.t, stride=st, dilation=dl,
                          pad=pad, bias=torch.from_numpy(bias).to(DEV) if bias is not None else None, relu=relu,
                          accumulate=acc))
        want.append(O.epilogue(O.conv2d_nhwc_hwcf(I, W, st, dl, pad), O_in if acc else None, bias, relu,
                               beta=1.0 if acc else 0.0))
    groups, G = nk.make_conv_groups(convs)
    for sched in [None, (128, 128, 64, 1, 3, 1)]:
        for can, O_in, acc in cans:
            can.t.copy_(torch.from_numpy(O_in).to(DEV))
        plan = nk.nk_conv2d_grouped_plan_create(groups, G, schedule=sched)
        nk.nk_grouped_plan_run(plan)
        nk.nk_sync_status()
        nk.nk_grouped_plan_destroy(plan)
        for g, (can, _, _) in enumerate(cans):
            can.check()
            np.testing.assert_array_equal(can.t.cpu().numpy(), want[g], err_msg=str((i, g, sched)))
