"""Argument validation happens on the host, before any device call: a
malformed request returns its own status and message even on a machine
without a GPU, and a well-formed one reaches the device check (NK_ERR_CUDA
here) -- never a CPU fallback.  Host tensors stand in for device memory;
validation reads only their descriptors."""
import pytest
import torch

nk = pytest.importorskip("paper_2307_16080_gb300.nk")

INVALID, UNSUPPORTED, CUDA = -1, -2, -5


def _status(fn):
    with pytest.raises(nk.NkError) as e:
        fn()
    assert nk.last_error(), "no message for a non-OK status"
    return e.value.status


def z(*shape, dtype=torch.float32):
    return torch.zeros(*shape, dtype=dtype)


@pytest.mark.parametrize("case,want", [
    (lambda: nk.nk_matmul(z(4, 5), z(6, 7), z(4, 7)), INVALID),                      # K mismatch
    (lambda: nk.nk_matmul(z(4, 5), z(5, 7), z(4, 8)), INVALID),                      # C shape
    (lambda: nk.nk_matmul(z(4, 5), z(5, 7), z(4, 7, dtype=torch.bfloat16), "bf16"), UNSUPPORTED),
    (lambda: nk.nk_matmul(z(4, 5), z(5, 7, dtype=torch.bfloat16), z(4, 7), "bf16"), INVALID),
    (lambda: nk.nk_matmul(z(4, 8, dtype=torch.bfloat16), z(8, 8, dtype=torch.bfloat16), z(4, 8), "f32"),
     INVALID),                                                                        # BF16 with F32 precision
])
def test_matmul_rejects_on_the_host(case, want):
    assert _status(case) == want


def test_matmul_unknown_precision():
    t = nk.as_nk_tensor
    a, b, c = z(4, 5), z(5, 7), z(4, 7)
    st = nk.lib().nk_matmul(nk.ctypes.byref(t(a)), nk.ctypes.byref(t(b)), nk.ctypes.byref(t(c)), 9, None, None,
                            None, 0, None)
    assert st == INVALID and nk.last_error()


@pytest.mark.parametrize("case,want", [
    (lambda: nk.nk_conv2d_nhwc_hwcf(z(1, 8, 8, 16), z(3, 3, 8, 4), z(1, 6, 6, 4)), INVALID),      # C mismatch
    (lambda: nk.nk_conv2d_nhwc_hwcf(z(1, 8, 8, 16), z(3, 3, 16, 4), z(1, 8, 8, 4)), INVALID),     # O extent
    (lambda: nk.nk_conv2d_nhwc_hwcf(z(1, 8, 8, 16), z(3, 3, 16, 4), z(1, 4, 6, 6).permute(0, 2, 3, 1)),
     UNSUPPORTED),                                                                               # O not NHWC
])
def test_conv_rejects_on_the_host(case, want):
    assert _status(case) == want


def test_well_formed_calls_reach_the_device_check():
    """Through the C ABI directly (NULL stream): the binding would ask
    PyTorch for the current CUDA stream first."""
    t, ref = nk.as_nk_tensor, nk.ctypes.byref
    a, b, c = z(4, 5), z(5, 7), z(4, 7)
    assert nk.lib().nk_matmul(ref(t(a)), ref(t(b)), ref(t(c)), 0, None, None, None, 0, None) == CUDA
    assert nk.last_error()
    i, w, o = z(1, 8, 8, 16), z(3, 3, 16, 4), z(1, 6, 6, 4)
    st, dl, pd = nk._conv_args((1, 1), (1, 1), (0, 0, 0, 0))
    assert nk.lib().nk_conv2d_nhwc_hwcf(ref(t(i)), ref(t(w)), ref(t(o)), st, dl, pd, 0, None, None, None, 0,
                                        None) == CUDA
    assert nk.last_error()
