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


def orth_tol(n, arith):
    """Tolerance on ||X^H X - I||_max for Ritz vectors of length n: the worst-case rounding bound
    n u of an n-term dot product in the arithmetic of the Rayleigh-Ritz products -- u = 2^-53 for
    FP64 (plain path, arith 1), 2^-48 for float-float (arith 0, ~48-bit products), 2^-47 for the
    bf16 digit products on the tensor cores (arith 2, 47-bit fixed point per row)."""
    u = {1: 2.0 ** -53, 0: 2.0 ** -48, 2: 2.0 ** -47}[arith]
    return n * u
