"""GPU parity of the direct NCHW / FCHW convolution (the layout of Listing
"2dnchwconv") against the FP64 oracle's loop nest, including the tuning
experiment's workload (1, 1, 1280, 1280) with Ci = 1, Co = 3, 3 x 3."""
import os

import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _nchw_ref(I, K, st, dl, pad):
    return O.conv2d_nhwc_hwcf(I.transpose(0, 2, 3, 1), K.transpose(2, 3, 1, 0), st, dl, pad).transpose(0, 3, 1, 2)


def _run(nk, I, K, st=(1, 1), dl=(1, 1), pad=(0, 0, 0, 0), **kw):
    R = _nchw_ref(I, K, st, dl, pad)
    out = kw.pop("out", None)
    out = torch.empty(*R.shape, device=DEV) if out is None else out
    nk.nk_conv2d_nchw_fchw(dev(I), dev(K), out, stride=st, dilation=dl, pad=pad, **kw)
    nk.nk_sync_status()
    return host(out), R


def test_paper_workload_ones_closed_form(nk):
    got, _ = _run(nk, np.ones((1, 1, 1280, 1280), np.float32), np.ones((3, 1, 3, 3), np.float32))
    assert got.shape == (1, 3, 1278, 1278)
    assert np.all(got == 9.0)


def test_paper_workload_normal(nk):
    I = synth.normal(90, 0, (1, 1, 1280, 1280))
    K = synth.normal(90, 1, (3, 1, 3, 3))
    got, R = _run(nk, I, K)
    assert O.rel_frobenius(got, R) <= 1e-6


def test_matches_listing_loop_nest_bitwise(nk):
    I = synth.small_ints(91, 0, (2, 3, 9, 70))
    K = synth.small_ints(91, 1, (5, 3, 3, 3))
    got, _ = _run(nk, I, K)
    np.testing.assert_array_equal(got, O.conv2d_nchw_fchw_loops(I, K))


@pytest.mark.parametrize("case", [
    ((1, 2, 33, 130), (12, 2, 3, 3), (2, 2), (1, 1), (1, 1, 1, 1)),
    ((2, 5, 20, 65), (3, 5, 5, 5), (1, 1), (2, 2), (2, 3, 1, 0)),
    ((1, 1, 17, 200), (9, 1, 1, 7), (1, 2), (1, 1), (0, 0, 3, 3)),
    ((3, 4, 40, 40), (16, 4, 3, 3), (1, 1), (1, 1), (0, 0, 0, 0)),
])
def test_variants_small_ints_bitwise(nk, case):
    ish, ksh, st, dl, pad = case
    I = synth.small_ints(92, ish[3], ish)
    K = synth.small_ints(92, ksh[0], ksh)
    got, R = _run(nk, I, K, st, dl, pad)
    np.testing.assert_array_equal(got, R)


@pytest.mark.parametrize("case", [
    # stride 1, dilation 1, 1x1 / 3x3 / 5x5: the register-streaming kernel
    ((1, 1, 21, 1283), (3, 1, 3, 3), (1, 1), (1, 1), (0, 0, 0, 0)),     # odd widths: 8-byte-aligned rows
    ((2, 3, 13, 37), (10, 3, 3, 3), (1, 1), (1, 1), (1, 2, 0, 1)),      # 3 channel groups, uneven padding
    ((1, 2, 19, 45), (5, 2, 5, 5), (1, 1), (1, 1), (2, 2, 2, 2)),
    ((2, 4, 7, 530), (6, 4, 1, 1), (1, 1), (1, 1), (0, 0, 0, 0)),       # rows wider than one CTA
    ((1, 1, 6, 6), (3, 1, 3, 3), (1, 1), (1, 1), (3, 3, 3, 3)),         # output mostly padding
    # one input channel: the rotating-accumulator kernel
    ((2, 1, 30, 77), (7, 1, 5, 5), (1, 1), (1, 1), (2, 1, 2, 0)),       # 2 channel groups, 5x5
    ((1, 1, 9, 300), (5, 1, 1, 1), (1, 1), (1, 1), (0, 0, 0, 0)),
    ((3, 1, 2, 9), (3, 1, 3, 3), (1, 1), (1, 1), (1, 1, 1, 1)),         # fewer rows than taps
])
def test_streaming_kernel_small_ints_bitwise(nk, case):
    ish, ksh, st, dl, pad = case
    I = synth.small_ints(95, ish[3], ish)
    K = synth.small_ints(95, ksh[0], ksh)
    got, R = _run(nk, I, K, st, dl, pad)
    np.testing.assert_array_equal(got, R)


def test_paper_workload_batch16(nk):
    """16 images of the tuning experiment's shape (larger than L2)."""
    I = synth.normal(96, 0, (16, 1, 1280, 1280))
    K = synth.normal(96, 1, (3, 1, 3, 3))
    got, R = _run(nk, I, K)
    assert O.rel_frobenius(got, R) <= 1e-6


def test_epilogue_bias_relu_accumulate(nk):
    I = synth.normal(93, 0, (2, 3, 30, 90))
    K = synth.normal(93, 1, (6, 3, 3, 3))
    bias = synth.uniform(93, 2, (6,), -1, 1)
    R0 = _nchw_ref(I, K, (1, 1), (1, 1), (1, 1, 1, 1))
    C0 = synth.uniform(93, 3, R0.shape)
    out = dev(C0)
    nk.nk_conv2d_nchw_fchw(dev(I), dev(K), out, pad=(1, 1, 1, 1), bias=dev(bias), relu=True, accumulate=True)
    nk.nk_sync_status()
    R = np.maximum(R0 + C0 + bias[None, :, None, None], 0.0)
    assert O.rel_frobenius(host(out), R) <= 1e-6
