"""The canary-padded output helper catches writes outside a view (checked on
CPU tensors, so the GPU out-of-bounds tests rest on a tested detector)."""
import pytest
import torch

from tests.gpu_util import Canary


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.uint8])
def test_writes_inside_the_view_pass(dtype):
    c = Canary((5, 7), dtype, strides=(9, 1), pad=64, device="cpu")
    c.t.fill_(1)
    c.check()


@pytest.mark.parametrize("where", ["before", "gap", "after"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.uint8])
def test_writes_outside_the_view_fail(dtype, where):
    c = Canary((5, 7), dtype, strides=(9, 1), pad=64, device="cpu")
    c.t.fill_(1)
    k = {"before": 63, "gap": 64 + 7, "after": 64 + 4 * 9 + 7}[where]   # raw indices outside the view
    c.buf[k] = 2
    with pytest.raises(AssertionError, match="outside the output"):
        c.check()


def test_transposed_view_covers_exactly_its_elements():
    c = Canary((3, 4), strides=(1, 5), pad=16, device="cpu")   # column-major with a padded leading dim
    c.t.copy_(torch.arange(12.0).reshape(3, 4))
    c.check()
    assert int(c.inside.sum()) == 12
