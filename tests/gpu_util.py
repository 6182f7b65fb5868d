"""Helpers shared by the GPU parity tests (conversion between the oracle's
NumPy layouts and the binding's CUDA tensors)."""
import numpy as np


def dev():
    import torch
    from paper_2012_00506_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


def to_dev(a, device):
    """NumPy band (n, ldab) or block (n, m) column-major -> CUDA tensor (band as is; block as (m, n))."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


def block_to_dev(X, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to(device)


def block_from_dev(T):
    return np.asfortranarray(T.detach().cpu().numpy().T)
