"""The split-K matmul that allocates nothing, checked against nk_matmul.

nk_matmul_f32_splitk_noalloc serves callers that cannot allocate device
memory (for instance code running inside an allocator callback): its split-K
partials live in a fixed array inside the library.  Called twice in a row
through the C ABI -- the second call reuses the array the first one left
behind -- each result must match nk_matmul with the same split on the same
inputs within the FP32 tolerance, and the device's free memory and torch's
allocator counters must not move across those calls.  This file is
collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

pytestmark = pytest.mark.gpu


def _memory_state():
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    return free, torch.cuda.memory_allocated(), torch.cuda.memory_reserved()


def test_noalloc_split_k_matches_nk_matmul_twice():
    import paper_2307_16080_gb300.nk as nk
    nk.lib()
    sms = nk.nk_device_info()[0]
    cases = [(300, 260, 2000, 4), (128, 512, 4096, 8)]
    inputs = []
    for M, N, K, split in cases:
        A, B = synth.matmul_uniform(M, N, K, seed=90 + split)
        a = torch.from_numpy(A).cuda()
        b = torch.from_numpy(B).cuda()
        c_ref = torch.empty(M, N, device="cuda")
        tile = 64 if ((M + 127) // 128) * ((N + 127) // 128) < sms else 128
        nk.nk_matmul(a, b, c_ref, precision="f32", schedule=(tile, tile, 16, 1, 2, split))
        c = torch.full((M, N), float("nan"), device="cuda")
        inputs.append((A, B, a, b, c, c_ref, split))
    # A first call may load the library's kernels (and with them the static
    # array) onto the device; the calls measured below come after it.
    A, B, a, b, c, c_ref, split = inputs[0]
    nk.nk_matmul_f32_splitk_noalloc(a, b, c, split)
    nk.nk_sync_status()
    before = _memory_state()
    for A, B, a, b, c, c_ref, split in inputs:   # two calls in a row
        c.fill_(float("nan"))
        nk.nk_matmul_f32_splitk_noalloc(a, b, c, split)
    nk.nk_sync_status()
    assert _memory_state() == before, "the no-allocation entry point changed device memory use"
    for A, B, a, b, c, c_ref, split in inputs:
        got, ref = c.cpu().numpy(), c_ref.cpu().numpy()
        assert O.rel_frobenius(got, ref) <= 1e-5
        assert O.rel_frobenius(got, O.matmul(A, B)) <= 1e-5


def test_noalloc_rejects_oversize_without_launch():
    import paper_2307_16080_gb300.nk as nk
    a = torch.empty(2048, 64, device="cuda")
    b = torch.empty(64, 2048, device="cuda")
    c = torch.empty(2048, 2048, device="cuda")
    with pytest.raises(nk.NkError) as e:
        nk.nk_matmul_f32_splitk_noalloc(a, b, c, 2)   # 2 * 2048 * 2048 > 4 Mi floats
    assert e.value.status == -4
