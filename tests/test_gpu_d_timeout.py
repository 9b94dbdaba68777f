"""Failure detection without a GPU fault: every device wait in the tensor-core
kernels is bounded.  Shrinking the spin budget to one poll makes the waits
run out on purpose; the kernel must then drain its own copies and MMAs, free
TMEM, exit, and the host must report NK_ERR_TIMEOUT -- after which the same
context keeps working."""
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


def test_wait_budget_exhaustion_reports_timeout_and_context_survives(nk):
    M, N, K = 512, 768, 4096
    A, B = synth.matmul_uniform(M, N, K, seed=80)
    a, b = dev(A), dev(B)
    c = torch.empty(M, N, device=DEV)
    sched = (128, 256, 64, 1, 4, 1)
    nk.nk_set_wait_budget(1)
    try:
        nk.nk_matmul(a, b, c, precision="bf16", schedule=sched)
        with pytest.raises(nk.NkError) as e:
            nk.nk_sync_status()
        assert e.value.status == -6
    finally:
        nk.nk_set_wait_budget(0)
    nk.nk_sync_status()          # flag was cleared by the previous report
    nk.nk_matmul(a, b, c, precision="bf16", schedule=sched)
    nk.nk_sync_status()
    assert O.rel_frobenius(host(c), O.matmul_precision(A, B, "bf16")) <= 1e-5


@pytest.mark.parametrize("sched", [(128, 64, 576, 1, 2, 1),    # shared window, taps in K
                                   (128, 64, 192, 1, 2, 1)])   # stacked kernel rows
def test_window_conv_wait_budget_exhaustion(nk, sched):
    """The same for the window convolution kernels: a timeout is reported,
    and the next call on the same context is exact."""
    I = synth.small_ints(81, 0, (4, 24, 24, 64))
    W = synth.small_ints(81, 1, (3, 3, 64, 64))
    i, w = dev(I), dev(W)
    out = torch.empty(4, 24, 24, 64, device=DEV)
    nk.nk_set_wait_budget(1)
    try:
        nk.nk_conv2d_nhwc_hwcf(i, w, out, pad=(1, 1, 1, 1), precision="bf16", schedule=sched)
        with pytest.raises(nk.NkError) as e:
            nk.nk_sync_status()
        assert e.value.status == -6
    finally:
        nk.nk_set_wait_budget(0)
    nk.nk_sync_status()
    nk.nk_conv2d_nhwc_hwcf(i, w, out, pad=(1, 1, 1, 1), precision="bf16", schedule=sched)
    nk.nk_sync_status()
    np.testing.assert_array_equal(host(out), O.conv2d_nhwc_hwcf(I, W, pad=(1, 1, 1, 1)))
