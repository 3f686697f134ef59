"""Helpers shared by the GPU parity tests (marshalling only)."""

import numpy as np
import torch

MASK = (1 << 64) - 1


def to_device(bits, misalign: int = 0) -> torch.Tensor:
    """float64 CUDA tensor holding the given bit patterns; misalign=1 shifts the
    start by 8 bytes so the data pointer is not 16-byte aligned."""
    a = np.ascontiguousarray(np.asarray(bits, dtype=np.uint64)).view(np.int64)
    t = torch.empty(a.size + misalign, dtype=torch.int64, device="cuda")
    if a.size:
        t[misalign:].copy_(torch.from_numpy(a))
    return t[misalign:].view(torch.float64)


def bits_of(t: torch.Tensor) -> np.ndarray:
    return t.detach().view(torch.int64).cpu().numpy().view(np.uint64)


def out_slot() -> torch.Tensor:
    return torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")


def f2b(x: float) -> int:
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])
