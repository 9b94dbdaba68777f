"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import torch

DEV = "cuda"


def dev(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def colmajor(x: np.ndarray) -> torch.Tensor:
    """A device tensor with x's values and column-major strides."""
    return dev(np.ascontiguousarray(x.T)).t()


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


# Canary-padded outputs: a stand-in for a memory checker.  The view a kernel
# writes lives inside a larger buffer whose every other element holds a NaN
# with a payload no kernel produces; check() fails on any write outside the
# view (before it, after it, or in the gaps its strides leave).
_SENT = {torch.float32: (torch.int32, 0x7FC0DEAD), torch.bfloat16: (torch.int16, 0x7FAB),
         torch.uint8: (torch.uint8, 0xA5)}


class Canary:
    def __init__(self, shape, dtype=torch.float32, strides=None, pad=4096, device=DEV):
        shape = tuple(int(s) for s in shape)
        if strides is None:
            strides, acc = [], 1
            for s in reversed(shape):
                strides.append(acc)
                acc *= s
            strides = tuple(reversed(strides))
        self.shape, self.strides, self.pad, self.dtype = shape, tuple(strides), pad, dtype
        span = 1 + sum((s - 1) * st for s, st in zip(shape, strides))
        itype, bits = _SENT[dtype]
        nbits = 8 * torch.tensor([], dtype=itype).element_size()
        if itype != torch.uint8 and bits >= 2 ** (nbits - 1):   # the signed integer with these bits
            bits -= 2 ** nbits
        raw = torch.full((2 * pad + span,), bits, dtype=itype, device=device)
        self.raw = raw
        self.buf = raw.view(dtype)
        self.t = self.buf[pad:].as_strided(shape, strides)
        idx = np.zeros(1, dtype=np.int64)
        for s, st in zip(shape, strides):
            idx = (idx[:, None] + np.arange(s, dtype=np.int64)[None, :] * st).reshape(-1)
        self.inside = np.zeros(raw.numel(), dtype=bool)
        self.inside[pad + idx] = True
        self.sentinel = raw[0].item()

    def check(self):
        if self.raw.is_cuda:
            torch.cuda.synchronize()
        r = self.raw.cpu().numpy()
        bad = np.flatnonzero((r != self.sentinel) & ~self.inside)
        assert bad.size == 0, f"{bad.size} elements written outside the output (first at {int(bad[0]) - self.pad})"
