"""Programmatic dependent launch: chains of dependent calls stay exact.

With nk_set_pdl(1) (the default) each kernel may start its set-up while the
kernel before it on the stream is finishing, and waits on the device before
it touches global memory.  A missing wait would show up as a race between
neighbouring kernels, so these chains put every kind of neighbour hazard in
a row:

- read after write: each layer reads the previous layer's output;
- write after read: with two ping-pong activation buffers, layer i+1 writes
  the buffer layer i read, and every layer re-uses one workspace, so the
  next layer's operand casts (or split-K partials) overwrite what the
  previous layer's contraction (or reduce) is still reading.

The final activation must be bitwise the same with PDL off and on, called
one by one and replayed from a CUDA graph; each layer of a separate
snapshot run matches the FP64 oracle applied to that layer's own input.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

from gpu_util import dev, host

pytestmark = pytest.mark.gpu

TOL_SAME_INPUTS = {"f32": 1e-5, "bf16": 1e-5, "fp8": 1e-5, "bf16x3": 2e-5}


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as nk
    nk.lib()
    yield nk
    nk.nk_set_pdl(True)


def _run_variants(nk, make_forward, out_of):
    """Final outputs of: PDL off eager, PDL on eager, PDL on graph, PDL off graph."""
    outs = []
    for pdl, graph in ((False, False), (True, False), (True, True), (False, True)):
        nk.nk_set_pdl(pdl)
        forward = make_forward()
        if graph:
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                forward()   # warm-up outside capture (per-device set-up)
                torch.cuda.synchronize()
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    forward()
            torch.cuda.current_stream().wait_stream(s)
            for _ in range(3):
                g.replay()
        else:
            for _ in range(3):
                forward()
        nk.nk_sync_status()
        outs.append(host(out_of()).copy())
    nk.nk_set_pdl(True)
    return outs


@pytest.mark.parametrize("prec,sched", [
    ("bf16", None),
    ("bf16", (256, 256, 64, 2, 4, 1)),   # CTA pair
    ("fp8", None),
    ("bf16x3", None),
    ("f32", (64, 64, 16, 1, 2, 4)),      # CUDA-core split-K + reduce
])
def test_matmul_chain_pdl_bitwise(nk, prec, sched):
    n, layers = 384, 6
    X0 = synth.uniform(71, 0, (n, n))
    Ws = [synth.uniform(71, 1 + i, (n, n)) * np.float32(1.7 / np.sqrt(n)) for i in range(layers)]
    bias = [synth.uniform(71, 20 + i, (n,), -0.1, 0.1) for i in range(layers)]
    ws_t = [dev(W) for W in Ws]
    b_t = [dev(b) for b in bias]
    bufs = [torch.empty(n, n, device="cuda"), torch.empty(n, n, device="cuda")]
    x0 = dev(X0)   # device copy made once: no host transfer inside graph capture
    ws = nk.workspace(nk.nk_matmul_workspace_size(bufs[0], ws_t[0], bufs[1], prec, sched), "cuda")

    def make_forward():
        def forward():
            bufs[0].copy_(x0)
            for i in range(layers):
                nk.nk_matmul(bufs[i % 2], ws_t[i], bufs[(i + 1) % 2], precision=prec, bias=b_t[i], relu=True,
                             schedule=sched, ws=ws)
        return forward

    outs = _run_variants(nk, make_forward, lambda: bufs[layers % 2])
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])

    # Snapshot run (PDL on): every layer against the oracle on its own input.
    x = dev(X0)
    for i in range(layers):
        y = torch.empty(n, n, device="cuda")
        nk.nk_matmul(x, ws_t[i], y, precision=prec, bias=b_t[i], relu=True, schedule=sched, ws=ws)
        nk.nk_sync_status()
        R = O.epilogue(O.matmul_precision(host(x), Ws[i], prec), bias=bias[i], relu=True)
        assert O.rel_frobenius(host(y), R) <= TOL_SAME_INPUTS[prec], (i, prec)
        x = y
    np.testing.assert_array_equal(host(x), outs[0])


@pytest.mark.parametrize("prec,packed,sched", [
    ("bf16", False, None),
    ("bf16", True, None),
    ("bf16", True, (128, 64, 576, 1, 1, 1)),   # shared-window kernel, one window slot
    ("fp8", False, None),
    ("f32", False, None),
])
def test_conv_chain_pdl_bitwise(nk, prec, packed, sched):
    N, H, C, layers = 2, 20, 64, 4
    I0 = synth.half_normal(72, 0, (N, H, H, C))
    Ws = [synth.normal(72, 1 + i, (3, 3, C, C), sigma=float(np.sqrt(2.0 / (9 * C)))) for i in range(layers)]
    bias = [synth.uniform(72, 10 + i, (C,), -0.1, 0.1) for i in range(layers)]
    w_t = [nk.nk_conv2d_pack_weights(dev(W)) if packed else dev(W) for W in Ws]
    b_t = [dev(b) for b in bias]
    pad = (1, 1, 1, 1)
    if packed:   # BF16 activations in, FP32 out: each layer's output is cast by a separate pass
        bufs = [torch.empty(N, H, H, C, device="cuda", dtype=torch.bfloat16) for _ in range(2)]
        out = torch.empty(N, H, H, C, device="cuda")
    else:
        bufs = [torch.empty(N, H, H, C, device="cuda") for _ in range(2)]
        out = None
    i0 = dev(I0).to(bufs[0].dtype)
    ws = nk.workspace(nk.nk_conv2d_workspace_size(bufs[0], w_t[0], out if packed else bufs[1], (1, 1), (1, 1),
                                                  pad, prec, sched), "cuda")

    def layer(x, i, y):
        nk.nk_conv2d_nhwc_hwcf(x, w_t[i], y, pad=pad, precision=prec, bias=b_t[i], relu=True, schedule=sched,
                               ws=ws)

    def make_forward():
        def forward():
            bufs[0].copy_(i0)
            for i in range(layers):
                if packed:
                    layer(bufs[i % 2], i, out)
                    bufs[(i + 1) % 2].copy_(out)
                else:
                    layer(bufs[i % 2], i, bufs[(i + 1) % 2])
        return forward

    outs = _run_variants(nk, make_forward, lambda: out if packed else bufs[layers % 2])
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])

    x = dev(I0).to(bufs[0].dtype)
    for i in range(layers):
        y = torch.empty(N, H, H, C, device="cuda")
        layer(x, i, y)
        nk.nk_sync_status()
        xin = host(x.float())
        R = O.epilogue(O.conv2d_precision(xin, Ws[i], prec, pad=pad), bias=bias[i], relu=True)
        assert O.rel_frobenius(host(y), R) <= TOL_SAME_INPUTS[prec], (i, prec)
        x = y.to(bufs[0].dtype)
    np.testing.assert_array_equal(host(y), outs[0])


def test_pdl_switch_round_trip(nk):
    assert nk.nk_get_pdl()
    nk.nk_set_pdl(False)
    assert not nk.nk_get_pdl()
    nk.nk_set_pdl(True)
    assert nk.nk_get_pdl()
