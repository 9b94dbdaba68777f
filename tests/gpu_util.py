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
