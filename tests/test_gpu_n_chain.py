"""GPU parity of the chained ResNet-style forward (paper_2307_16080_gb300.forward).

Every layer reads the BF16 output its predecessor wrote.  Layer by layer,
the GPU output is compared with the FP64 oracle run on that layer's own GPU
input (the BF16 values the previous kernel stored, the packed BF16 weights
= bf16_rn of the FP32 weights, the FP32 bias and, for a stage's last layer,
the FP32 projection it adds).  A BF16 output is the FP32 epilogue value
rounded once, so elementwise |out - exact| <= 2^-9 |out| + (FP32
accumulation error), i.e. a relative Frobenius error of at most 2^-9 + 1e-5;
the FP32 outputs (projections, head) keep the 1e-5 bound.  A CUDA-graph
replay of the whole forward reproduces the eager result bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

pytestmark = pytest.mark.gpu

BF16_BOUND = 2.0 ** -9 + 1e-5


@pytest.fixture(scope="module")
def fwd():
    import paper_2307_16080_gb300.forward as f
    import paper_2307_16080_gb300.nk as nk
    nk.lib()
    return f


def _h(t):
    return t.float().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("batch", [1, 2])
def test_chained_forward_layer_by_layer(fwd, batch):
    import paper_2307_16080_gb300.nk as nk
    net = fwd.ResNetStack(batch, "cuda")
    x = torch.from_numpy(synth.half_normal(120, batch, (batch, 56, 56, 64))).cuda().to(torch.bfloat16)
    net.bind(x)
    net.run()
    nk.nk_sync_status()
    for li, L in enumerate(net.layers):
        src, res = net.layer_inputs(li)
        out = net.outputs[li]
        st, pad = (L["stride"],) * 2, (L["pad"],) * 4
        acc = O.conv2d_nhwc_hwcf(_h(src), O.bf16_rn(net.weights32[li]), st, (1, 1), pad)
        role = net.role(li)
        if role == "residual":
            R = O.ew_program(O.epilogue(acc, bias=net.bias32[li]), [("add", _h(res)), ("relu",)])
        else:
            R = O.epilogue(acc, bias=net.bias32[li], relu=role != "projection")
        err = O.rel_frobenius(_h(out), R)
        bound = BF16_BOUND if out.dtype == torch.bfloat16 else 1e-5
        assert err <= bound, (li, role, err)
        if out.dtype == torch.bfloat16:   # the stored values are BF16 roundings of FP32 results
            assert np.array_equal(O.bf16_rn(_h(out)), _h(out))


def test_chained_forward_graph_replay_is_bitwise(fwd):
    import paper_2307_16080_gb300.nk as nk
    net = fwd.ResNetStack(4, "cuda")
    x = torch.from_numpy(synth.half_normal(121, 0, (4, 56, 56, 64))).cuda().to(torch.bfloat16)
    net.bind(x)
    net.run()
    torch.cuda.synchronize()
    eager = [o.clone() for o in net.outputs]
    for o in net.outputs:
        o.fill_(float("nan"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            net.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    nk.nk_sync_status()
    for a, b in zip(eager, net.outputs):
        assert torch.equal(a, b)
    assert net.kernels >= 20
