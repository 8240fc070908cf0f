"""Helpers shared by the GPU tests (device buffers through torch, nothing else)."""
import numpy as np

U53 = 2.0 ** -53


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a, ld=None):
    """Copy a 2-D numpy block to a CUDA tensor with leading dimension ld (>= cols)."""
    torch = torch_cuda()
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    rows, cols = a.shape
    ld = ld or cols
    t = torch.zeros((rows, ld), dtype=torch.float64, device="cuda")
    t[:, :cols] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t


def host(t, cols=None):
    x = t.detach().cpu().numpy()
    return x if cols is None else x[:, :cols]


def dev_i32(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def gamma(n):
    """Classical bound n*u/(1 - n*u) on the relative error of an n-term dot product."""
    return n * U53 / (1 - n * U53)
