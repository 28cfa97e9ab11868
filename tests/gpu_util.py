"""Helpers of the GPU tests: tensors in the layouts the C ABI takes."""
import numpy as np


def dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def normwise(a, b):
    """max |a - b| / max |b| (per field), the error measure of the tolerances."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def state_tensors(U, dtype):
    """(4, ny, nx) numpy state -> four contiguous device tensors (halo 0)."""
    return [to_dev(U[f], dtype) for f in range(4)]


def empty_like_state(ts):
    import torch
    return [torch.empty_like(t) for t in ts]
