"""Helpers shared by the GPU tests (marshalling only)."""
import numpy as np
import torch


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def bf16_round(x):
    """float64 values rounded to the nearest bfloat16 (ties to even), returned
    as float64: inputs that a bf16 rounding leaves unchanged."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    keep = np.uint64(45)                      # float64 keeps 52 fraction bits, bfloat16 7
    bias = np.uint64((1 << 44) - 1) + ((b >> keep) & np.uint64(1))
    return ((b + bias) & ~np.uint64((1 << 45) - 1)).view(np.float64)
