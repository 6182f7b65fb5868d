"""Tall block products of the Rayleigh-Ritz step on the tensor cores (bf16 digit products,
FP64-class accuracy) against FP64 products of the same operands.

The digit scheme is exact up to the rounding of the digits (2^-48 of each row's maximum), the
dropped digit pairs (d+d' > 6) and the FP32 rounding of the accumulator of the trailing levels, so
the error of every entry must stay at FP64 level relative to the norms of its two columns (5e-15
here).  An inexact accumulation of the leading levels would show up near 1e-7, and stopping at
digit level 5 leaves a bias near 5e-14 on Gram diagonals.  Sizes span several 128 x 32 tiles,
ragged block widths (1, 37, 130, 267), reduction lengths that are not multiples of the 32-element
stage, and a reduction long enough to need several split-K ranges.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    from gpu_util import dev
    dev()
    import paper_2012_00506_gb300 as pk
    return pk


def _blocks(n, sizes, cplx, seed, scales=True):
    g = np.random.default_rng(seed)
    M = int(sum(sizes))
    X = g.normal(size=(M, n))
    if cplx:
        X = X + 1j * g.normal(size=(M, n))
    if scales:  # columns of very different magnitude (each digit row has its own scale)
        X *= (10.0 ** g.uniform(-6, 6, size=M))[:, None]
    return X


def _rel_err(C, Cref, na, nb):
    return np.max(np.abs(C - Cref) / np.outer(na, nb))


def _t(pk, X):
    import torch
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n", [1000, 8192])
def test_gram_tensor_matches_fp64(pk, cplx, n):
    sizes = [1, 37, 130, 267]
    X = _blocks(n, sizes, cplx, 11 + n)
    out = pk.block_gemm(pk.GEMM_GRAM, _t(pk, X), sizes, arith=pk.RR_TENSOR)
    off = 0
    worst = 0.0
    for t, m in enumerate(sizes):
        A = X[off: off + m].T            # n x m
        ref = A.conj().T @ A
        C = out[t].cpu().numpy()
        nrm = np.linalg.norm(A, axis=0)
        worst = max(worst, _rel_err(C, ref, nrm, nrm))
        assert np.array_equal(C, C.conj().T)          # Hermitian by construction
        off += m
    print("gram", cplx, n, worst)
    assert worst < 5e-15


@pytest.mark.parametrize("cplx", [True, False])
def test_projection_tensor_matches_fp64(pk, cplx):
    n, sizes = 8192, [267, 250, 64]
    X = _blocks(n, sizes, cplx, 5)
    Y = _blocks(n, sizes, cplx, 6)
    out = pk.block_gemm(pk.GEMM_AHB, _t(pk, X), sizes, B=_t(pk, Y), arith=pk.RR_TENSOR)
    off = 0
    for t, m in enumerate(sizes):
        A, B = X[off: off + m].T, Y[off: off + m].T
        err = _rel_err(out[t].cpu().numpy(), A.conj().T @ B, np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0))
        print("ahb", cplx, m, err)
        assert err < 5e-15
        off += m


@pytest.mark.parametrize("cplx", [True, False])
@pytest.mark.parametrize("n", [1000, 8192])
def test_update_tensor_matches_fp64(pk, cplx, n):
    sizes = [1, 37, 267]
    X = _blocks(n, sizes, cplx, 21, scales=False)
    g = np.random.default_rng(22)
    Ts = []
    for m in sizes:
        T = g.normal(size=(m, m)) + (1j * g.normal(size=(m, m)) if cplx else 0)
        T = np.triu(T) if m == 37 else T           # triangular factor (explicit CholQR pass)
        T[:, :1] *= 1e8                             # columns of very different magnitude
        Ts.append(T)
    out = pk.block_gemm(pk.GEMM_UPDATE, _t(pk, X), sizes, B=[_t(pk, T) for T in Ts], arith=pk.RR_TENSOR)
    got = out.cpu().numpy()
    off = 0
    for t, m in enumerate(sizes):
        A = X[off: off + m].T
        ref = A @ Ts[t]
        C = got[off: off + m].T
        # row i of A times column j of T: relative to |A(i, :)| |T(:, j)|
        err = np.max(np.abs(C - ref) / np.outer(np.linalg.norm(A, axis=1), np.linalg.norm(Ts[t], axis=0)))
        print("update", cplx, n, m, err)
        # few terms keep the full digit rounding of both factors (2 x 2^-47 relative for m = 1)
        assert err < 3e-14
        off += m


def test_long_reduction_split_k(pk):
    """2n = 80000 elements: five split-K ranges of at most 16384, each with exact integer sums."""
    n, sizes = 40000, [40, 70]
    X = _blocks(n, sizes, True, 31, scales=False)
    out = pk.block_gemm(pk.GEMM_GRAM, _t(pk, X), sizes, arith=pk.RR_TENSOR)
    off = 0
    for t, m in enumerate(sizes):
        A = X[off: off + m].T
        nrm = np.linalg.norm(A, axis=0)
        err = _rel_err(out[t].cpu().numpy(), A.conj().T @ A, nrm, nrm)
        print("split-k", m, err)
        assert err < 5e-15
        off += m


def test_tensor_agrees_with_floatfloat_and_fp64(pk):
    n, sizes = 4096, [100, 33]
    X = _blocks(n, sizes, True, 41, scales=False)
    r = {a: pk.block_gemm(pk.GEMM_GRAM, _t(pk, X), sizes, arith=a) for a in (pk.RR_TENSOR, pk.RR_FLOATFLOAT,
                                                                             pk.RR_FP64)}
    for t in range(len(sizes)):
        ref = r[pk.RR_FP64][t].cpu().numpy()
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(r[pk.RR_TENSOR][t].cpu().numpy() - ref)) <= 1e-14 * scale
        assert np.max(np.abs(r[pk.RR_FLOATFLOAT][t].cpu().numpy() - ref)) <= 5e-13 * scale


@pytest.mark.parametrize("cplx", [True, False])
def test_update_with_badly_scaled_columns(pk, cplx):
    """X = Q T with columns of Q spanning 16 decades and T undoing the scaling (the
    shape of Q R^{-1} on a filtered basis): the columns are equilibrated before the
    digit split, so X keeps FP64-class accuracy relative to |U(i,:)| |W(:,j)|."""
    n, m = 4096, 96
    g = np.random.default_rng(51)
    U = g.normal(size=(n, m)) + (1j * g.normal(size=(n, m)) if cplx else 0)
    W = g.normal(size=(m, m)) + (1j * g.normal(size=(m, m)) if cplx else 0)
    s = 10.0 ** g.uniform(-16, 0, size=m)
    Q = U * s[None, :]
    T = W / s[:, None]
    out = pk.block_gemm(pk.GEMM_UPDATE, _t(pk, np.ascontiguousarray(Q.T)), [m], B=[_t(pk, T)], arith=pk.RR_TENSOR)
    X = out.cpu().numpy().T
    ref = U @ W
    err = np.max(np.abs(X - ref) / np.outer(np.linalg.norm(U, axis=1), np.linalg.norm(W, axis=0)))
    print("update scaled", cplx, err)
    assert err < 1e-14


@pytest.mark.parametrize("cplx,n,b,m", [(True, 8192, 64, 267), (False, 1000, 7, 37), (True, 333, 40, 5),
                                        (False, 2000, 32, 150)])
def test_band_product_tensor_matches_fp64(pk, cplx, n, b, m):
    """Y = B X on the tensor cores (128-row tiles of the band over their window) against the
    FP64 band product: every entry within 1e-13 |B(i,:)| max|X(:,j)| (the digits of a row of B
    and of a column of X carry 2^-47 of their maxima; 2b+1 such terms add up); ragged n, b not
    a multiple of 32, windows that start before row 0 and end past row n."""
    import synth
    ab = synth.random_band(n, b, 61 + n, cplx)
    g = np.random.default_rng(62)
    X = g.normal(size=(m, n)) + (1j * g.normal(size=(m, n)) if cplx else 0)
    Y = pk.band_matmul_tc(_t(pk, ab), _t(pk, X)).cpu().numpy()
    Bd = synth.band_to_dense(ab)
    ref = X @ Bd.T                      # rows of the (m, n) layout: (B x_j)^T
    scale = np.outer(np.max(np.abs(X), axis=1), np.linalg.norm(Bd, axis=1))
    err = np.max(np.abs(Y - ref) / scale)
    print("band", cplx, n, b, m, err)
    assert err < 1e-13
