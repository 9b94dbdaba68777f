"""No kernel writes outside its output: every family writes into an output
view that sits inside a sentinel-filled buffer (tests.gpu_util.Canary), on
ragged shapes and padded row strides, and the sentinels must survive.  The
stand-in for a memory checker, which is closed on this machine; the values
themselves are checked against the FP64 oracle as well."""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import Canary, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


MM = [("f32", None), ("f32", (64, 64, 16, 1, 2, 3)), ("bf16", None), ("bf16", (128, 64, 64, 1, 3, 3)),
      ("bf16", (256, 512, 64, 2, 4, 1)), ("bf16", (256, 128, 64, 1, 3, 1)), ("fp8", (128, 128, 128, 1, 4, 1)),
      ("bf16x3", (256, 128, 64, 2, 3, 1))]


@pytest.mark.parametrize("prec,sched", MM)
@pytest.mark.parametrize("N,ldc", [(260, 273), (259, 260), (257, 264), (256, 264)])
def test_matmul_writes_only_its_output(nk, prec, sched, N, ldc):
    """Padded rows (the gaps are canaries); ldc a multiple of 4 floats with
    N % 4 != 0 must not take the TMA-store epilogue, whose clipping works in
    16-byte granules."""
    M, K = 300, 200
    A = synth.small_ints(140, 1, (M, K))
    B = synth.small_ints(140, 2, (K, N))
    if prec == "fp8":   # half-integers up to 3.5 with amax 3.5: exact E4M3 codes
        A, B = A / 2, B / 2
        A.flat[0], B.flat[0] = 3.5, 3.5
    c = Canary((M, N), strides=(ldc, 1))   # padded rows: gaps between them are canaries too
    nk.nk_matmul(dev(A), dev(B), c.t, precision=prec, schedule=sched, bias=dev(np.ones(N, np.float32)))
    nk.nk_sync_status()
    c.check()
    np.testing.assert_array_equal(host(c.t), O.matmul_precision(A, B, prec) + 1.0)


CONV = [(None, torch.float32), ((128, 64, 64, 1, 3, 1), torch.float32), ((128, 64, 64, 1, 3, 3), torch.bfloat16),
        ((128, 64, 576, 1, 2, 1), torch.float32), ((128, 64, 192, 1, 1, 1), torch.bfloat16),
        ((256, 64, 192, 1, 4, 1), torch.float32), ((256, 64, 192, 1, 4, 1), torch.bfloat16)]


@pytest.mark.parametrize("sched,odt", CONV)
def test_conv_writes_only_its_output(nk, sched, odt):
    N, H, Wd, C, F = 2, 13, 15, 64, 40
    I = synth.small_ints(141, 1, (N, H, Wd, C))
    W = synth.small_ints(141, 2, (3, 3, C, F))
    c = Canary((N, H, Wd, F), odt)
    nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), c.t, pad=(1, 1, 1, 1), precision="bf16", schedule=sched, relu=True)
    nk.nk_sync_status()
    c.check()
    R = O.epilogue(O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)), relu=True)
    np.testing.assert_array_equal(c.t.float().cpu().numpy(), O.bf16_rn(R) if odt == torch.bfloat16 else R)


def test_fp8_window_conv_writes_only_its_output(nk):
    N, H, Wd, C, F = 2, 11, 12, 128, 40
    I = synth.small_ints(142, 1, (N, H, Wd, C)) / 2
    W = synth.small_ints(142, 2, (3, 3, C, F)) / 2
    I.flat[0], W.flat[0] = 3.5, 3.5
    c = Canary((N, H, Wd, F))
    try:
        nk.nk_conv2d_nhwc_hwcf(dev(I), dev(W), c.t, pad=(1, 1, 1, 1), precision="fp8",
                               schedule=(256, 64, 384, 1, 3, 1))
    except nk.NkError as e:
        if e.status == -7:   # no room for this schedule's layout on this shape
            pytest.skip(str(e))
        raise
    nk.nk_sync_status()
    c.check()
    np.testing.assert_array_equal(host(c.t), O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)))


# per-lane stores (rows not 16-byte multiples), and TMA stores clipped at
# each group's ragged edges (every row a 16-byte multiple)
GROUP_SETS = [[(130, 70, 96), (33, 257, 64), (256, 128, 160), (1, 16, 48)],
              [(130, 72, 96), (33, 260, 64), (256, 132, 160), (1, 16, 48), (97, 300, 32)]]


@pytest.mark.parametrize("shapes", GROUP_SETS)
def test_grouped_gemm_writes_only_its_outputs(nk, shapes):
    As = [synth.small_ints(143, 2 * g, (M, K)) for g, (M, N, K) in enumerate(shapes)]
    Bs = [synth.small_ints(143, 2 * g + 1, (K, N)) for g, (M, N, K) in enumerate(shapes)]
    cans = [Canary((M, N)) for (M, N, K) in shapes]
    a16 = [dev(a).to(torch.bfloat16) for a in As]
    bt16 = [dev(np.ascontiguousarray(b.T)).to(torch.bfloat16) for b in Bs]
    groups, G = nk.make_groups(a16, bt16, [c.t for c in cans])
    for sched in [None, (128, 64, 0, 1, 0, 0), (128, 256, 0, 1, 4, 0), (256, 128, 0, 2, 0, 0)]:
        plan = nk.nk_grouped_plan_create(groups, G, schedule=sched)
        nk.nk_grouped_plan_run(plan)
        nk.nk_sync_status()
        nk.nk_grouped_plan_destroy(plan)
        for c, a, b in zip(cans, As, Bs):
            c.check()
            np.testing.assert_array_equal(host(c.t), O.matmul(a, b))


def test_direct_conv_and_casts_write_only_their_outputs(nk):
    inp = synth.small_ints(144, 1, (2, 1, 37, 53))
    ker = synth.small_ints(144, 2, (3, 1, 3, 3))
    c = Canary((2, 3, 35, 51))
    nk.nk_conv2d_nchw_fchw(dev(inp), dev(ker), c.t)
    nk.nk_sync_status()
    c.check()
    x = synth.normal(145, 0, (37, 45))
    cb = Canary((37, 45), torch.bfloat16, strides=(56, 1))
    nk.nk_cast_bf16(dev(x), cb.t)
    cb.check()
    ct = Canary((45, 37), torch.bfloat16, strides=(40, 1))
    nk.nk_cast_bf16(dev(x), ct.t, transpose=True)
    ct.check()
    np.testing.assert_array_equal(ct.t.float().cpu().numpy(), O.bf16_rn(x).T)
    amax = dev(np.array([np.abs(x).max()], np.float32))
    c8 = Canary((37, 45), torch.uint8, strides=(48, 1))
    nk.nk_cast_fp8(dev(x), amax, c8.t)
    c8.check()
