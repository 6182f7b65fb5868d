"""FP64 CPU oracle of the learned slice proposer -- TEST INFRASTRUCTURE.

Only ``tests/`` may import this module.  It restates, in plain NumPy FP64,
what the library's proposer computes, so that the CUDA kernels can be compared
with it element by element.  The proposer itself is not in arXiv 2012.00506:
the paper slices by inertia counts (Section 3.2), names density-of-states
estimates for a first partition (Section 3.1) and lists equal eigenvalue
counts per slice among its partition objectives (Section 3.1).

* ``splitmix64``, ``probes``  Vigna's SplitMix64 (state += 0x9e3779b97f4a7c15,
                              then z ^= z >> 30; z *= 0xbf58476d1ce4e5b9;
                              z ^= z >> 27; z *= 0x94d049bb133111eb;
                              z ^= z >> 31) and the Rademacher probes drawn from
                              its low bit.
* ``features``                diagonal histogram over the Gershgorin interval,
                              the interval's centre and radius, and Chebyshev
                              moments of the scaled band estimated with the
                              probes (kernel polynomial method: stochastic
                              trace of T_k by the three-term recurrence).
* ``forward``, ``loss_and_grad``  the network 98 -> 256 -> 256 -> 256 -> 64
                              (ReLU), softmax, cumulative sums, mean squared
                              error, and its gradient by reverse-mode
                              differentiation written out by hand.
* ``adam_step``               Adam (Kingma and Ba, 2015) with bias correction.

Pins: ``tests/test_oracle_slicer.py`` (closed forms on diagonal bands, an
eigendecomposition route for the moments, central finite differences for the
gradient, the uniform output of a zero network, the first-step closed form of
Adam, published SplitMix64 outputs).
"""
from __future__ import annotations

import numpy as np

from . import band_matvec, gershgorin

N_FEAT, N_HID, N_OUT, N_BINS, N_MOM, N_PROBES = 98, 256, 64, 64, 32, 8
DIMS = (N_FEAT, N_HID, N_HID, N_HID, N_OUT)
_M64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One SplitMix64 output for input state ``x`` (Python integers, mod 2^64)."""
    x = (x + 0x9E3779B97F4A7C15) & _M64
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def probes(n: int, seed: int) -> np.ndarray:
    """n x 8 Rademacher probes: entry (i, p) = +1 if splitmix64(seed + p n + i) is even, else -1."""
    Z = np.empty((n, N_PROBES))
    for p in range(N_PROBES):
        for i in range(n):
            Z[i, p] = -1.0 if splitmix64((seed + p * n + i) & _M64) & 1 else 1.0
    return Z


def histogram(d: np.ndarray, lo: float, hi: float) -> np.ndarray:
    """64-bin histogram of the values d over [lo, hi] as fractions; out-of-range values clamp."""
    w = (hi - lo) / N_BINS
    h = np.zeros(N_BINS)
    for x in d:
        k = 0
        if w > 0:
            t = np.floor((x - lo) / w)
            k = 0 if t < 0 else (N_BINS - 1 if t > N_BINS - 1 else int(t))
        h[k] += 1
    return h / d.size


def chebyshev_moments(ab: np.ndarray, lo: float, hi: float, Z: np.ndarray) -> np.ndarray:
    """mu_k = (1/(n P)) sum_p z_p^H T_k(Bs) z_p, k = 0..31, Bs = (B - c I)/r."""
    n = ab.shape[0]
    c, r = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if not r > 0:
        r = 1.0
    scaled = lambda X: (band_matvec(ab, X) - c * X) / r  # noqa: E731
    T0 = Z.astype(np.complex128)
    T1 = scaled(T0)
    mu = np.zeros(N_MOM)
    mu[0] = np.sum(np.real(np.conj(Z) * T0)) / (n * N_PROBES)
    mu[1] = np.sum(np.real(np.conj(Z) * T1)) / (n * N_PROBES)
    for k in range(2, N_MOM):
        T2 = 2.0 * scaled(T1) - T0
        mu[k] = np.sum(np.real(np.conj(Z) * T2)) / (n * N_PROBES)
        T0, T1 = T1, T2
    return mu


def features(ab: np.ndarray, seed: int) -> np.ndarray:
    """The 98 features of the band, FP64."""
    n = ab.shape[0]
    lo, hi = gershgorin(ab)
    s = max(abs(lo), abs(hi))
    if not s > 0:
        s = 1.0
    f = np.zeros(N_FEAT)
    f[:N_BINS] = histogram(np.real(ab[:, 0]), lo, hi)
    f[64] = 0.5 * (lo + hi) / s
    f[65] = 0.5 * (hi - lo) / s
    f[66:] = chebyshev_moments(ab, lo, hi, probes(n, seed))
    return f


def unpack(params: np.ndarray):
    """[(W (out x in), bias)] views of the parameter vector (per layer: W row-major, then bias)."""
    out, off = [], 0
    p = np.asarray(params, dtype=np.float64)
    for l in range(4):
        fi, fo = DIMS[l], DIMS[l + 1]
        W = p[off: off + fo * fi].reshape(fo, fi)
        off += fo * fi
        b = p[off: off + fo]
        off += fo
        out.append((W, b))
    return out


def forward(params: np.ndarray, X: np.ndarray, keep: bool = False):
    """Boundaries (batch, 63): cumulative sums of the softmax of the network's logits."""
    h = np.asarray(X, dtype=np.float64).reshape(-1, N_FEAT)
    acts = [h]
    layers = unpack(params)
    for l, (W, b) in enumerate(layers):
        a = h @ W.T + b
        h = np.maximum(a, 0.0) if l < 3 else a
        acts.append(h)
    z = h - h.max(axis=1, keepdims=True)
    e = np.exp(z)
    p = e / e.sum(axis=1, keepdims=True)
    c = np.cumsum(p, axis=1)[:, : N_OUT - 1]
    return (c, p, acts) if keep else c


def loss_and_grad(params: np.ndarray, X: np.ndarray, T: np.ndarray):
    """L = mean over batch and boundaries of (c - t)^2, and dL/dparams (same layout)."""
    c, p, acts = forward(params, X, keep=True)
    T = np.asarray(T, dtype=np.float64).reshape(c.shape)
    B = c.shape[0]
    scale = 1.0 / (B * (N_OUT - 1))
    loss = float(np.sum((c - T) ** 2) * scale)
    dc = np.zeros((B, N_OUT))
    dc[:, : N_OUT - 1] = 2.0 * (c - T) * scale
    dp = np.cumsum(dc[:, ::-1], axis=1)[:, ::-1]            # dL/dp_j = sum_{k >= j} dL/dc_k
    dz = p * (dp - np.sum(p * dp, axis=1, keepdims=True))   # softmax Jacobian
    layers = unpack(params)
    grads = [None] * 4
    g = dz
    for l in range(3, -1, -1):
        W, _ = layers[l]
        x_in = acts[l]
        grads[l] = (g.T @ x_in, g.sum(axis=0))
        if l > 0:
            g = (g @ W) * (acts[l] > 0)
    flat = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in grads])
    return loss, flat


def adam_step(p, g, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update with bias correction; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def equal_count_targets(ab: np.ndarray, nslices: int = 64) -> np.ndarray:
    """The proposer's regression targets from the exact spectrum (dense eigvalsh of the
    band): boundary k (k = 1..nslices-1) is the midpoint of eigenvalues t-1 and t,
    t = floor(k n / nslices + 1/2) clipped to [1, n-1], normalised to the Gershgorin
    interval and clipped to [0, 1]."""
    n, ldab = ab.shape
    A = np.zeros((n, n), dtype=ab.dtype)
    for d in range(ldab):                       # lower band storage: ab[j, d] = B(j + d, j)
        j = np.arange(n - d)
        A[j + d, j] = ab[: n - d, d]
        if d:
            A[j, j + d] = np.conj(ab[: n - d, d])
    ev = np.linalg.eigvalsh(A)
    lo, hi = gershgorin(ab)
    span = hi - lo if hi > lo else 1.0
    out = np.zeros(nslices - 1)
    for k in range(1, nslices):
        t = min(max((2 * k * n + nslices) // (2 * nslices), 1), n - 1)
        out[k - 1] = min(max((0.5 * (ev[t - 1] + ev[t]) - lo) / span, 0.0), 1.0)
    return out

