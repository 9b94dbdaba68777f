"""FP32 -> BF16 and FP32 -> E4M3 conversions of the operand-prep kernels,
bitwise against the oracle's own rounding over every rounding class.

The inputs are every value of the high 16 bits of an FP32 word (sign,
exponent, the mantissa bits either format keeps, its round bit and the
upper sticky bits) combined with a set of low halves: 0, 1, just below,
at and just above the half-way point of a BF16 ulp, all ones, and seeded
random halves.  So every sign, binade and tie / above / below case of
round-to-nearest-even is exercised, for normal and subnormal results, with
E4M3 saturation at +-448 (scale 1), in 65536 x 16 patterns per
conversion.  Codes are compared as bits, so the sign of zero counts.
"""
import numpy as np
import pytest
import torch

import oracle.nk_oracle as O
from paper_2307_16080_gb300 import synth
from tests.gpu_util import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nk():
    import paper_2307_16080_gb300.nk as m
    m.lib()
    return m


def _patterns():
    lo = [0x0000, 0x0001, 0x7FFF, 0x8000, 0x8001, 0xFFFF]
    lo += [int(v) & 0xFFFF for v in synth.raw_u64(151, 0, 10)]
    hi = np.arange(1 << 16, dtype=np.uint32)
    bits = (hi[:, None] << np.uint32(16)) | np.array(lo, dtype=np.uint32)[None, :]
    x = bits.reshape(-1).view(np.float32)
    return x[np.isfinite(x)]


def _bf16_bits(values):
    """Expected BF16 bit patterns of exactly representable values (float64)."""
    return (np.asarray(values, np.float64).astype(np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def test_bf16_cast_every_rounding_class_bitwise(nk):
    x = _patterns()
    n = x.size // 1024 * 1024
    x2 = x[:n].reshape(-1, 1024)
    out = torch.empty(x2.shape, dtype=torch.bfloat16, device=DEV)
    nk.nk_cast_bf16(torch.from_numpy(x2).to(DEV), out)
    torch.cuda.synchronize()
    got = out.view(torch.int16).cpu().numpy().view(np.uint16)
    want = _bf16_bits(O.bf16_rn(x2))
    bad = np.flatnonzero(got.reshape(-1) != want.reshape(-1))
    assert bad.size == 0, (bad.size, hex(x2.reshape(-1)[bad[0]].view(np.uint32)), hex(got.reshape(-1)[bad[0]]),
                           hex(want.reshape(-1)[bad[0]]))


def test_e4m3_cast_every_rounding_class_bitwise(nk):
    x = _patterns()
    n = x.size // 1024 * 1024
    x2 = x[:n].reshape(-1, 1024)
    amax = torch.tensor([448.0], device=DEV)   # scale 448 / 448 = 1: the codes round x itself
    q = torch.empty(x2.shape, dtype=torch.uint8, device=DEV)
    s_out = torch.empty(1, device=DEV)
    nk.nk_cast_fp8(torch.from_numpy(x2).to(DEV), amax, q, scale_out=s_out)
    torch.cuda.synchronize()
    assert s_out.item() == 1.0
    got = q.view(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
    got_neg = (q.cpu().numpy() & 0x80) != 0
    want = O.fp8_quantize(x2, np.float32(1.0))
    np.testing.assert_array_equal(got, want)
    # the sign of zero: E4M3 keeps it (code 0x80 for -0)
    zero = want == 0
    np.testing.assert_array_equal(got_neg[zero], np.signbit(want[zero]))
