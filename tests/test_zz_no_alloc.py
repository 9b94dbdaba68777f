"""The split-K matmul that allocates nothing, checked against nk_matmul.

nk_matmul_f32_splitk_noalloc serves callers that cannot allocate device
memory (for instance code running inside an allocator callback): its split-K
partials live in a fixed array inside the library.  Called twice in a row
through the C ABI -- the second call reuses the array the first one left
behind -- each result must match nk_matmul with the same split on the same
inputs within the FP32 tolerance.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_split_k_matches_nk_matmul_twice():
    import paper_2307_16080_gb300.nk as nk
    nk.lib()
    cases = [(300, 260, 2000, 4), (128, 512, 4096, 8)]
    for M, N, K, split in cases:
        A, B = synth.matmul_uniform(M, N, K, seed=90 + split)
        a = torch.from_numpy(A).cuda()
        b = torch.from_numpy(B).cuda()
        c_ref = torch.empty(M, N, device="cuda")
        tile = 64 if ((M + 127) // 128) * ((N + 127) // 128) < 152 else 128
        nk.nk_matmul(a, b, c_ref, precision="f32", schedule=(tile, tile, 16, 1, 2, split))
        c = torch.full((M, N), float("nan"), device="cuda")
        nk.nk_matmul_f32_splitk_noalloc(a, b, c, split)
        nk.nk_sync_status()
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
