"""Learned slice proposal -- Python side of the C ABI's proposer entry points.

The paper partitions the spectrum with inertia counts (Section 3.2) and
suggests density-of-states estimates when no earlier spectrum is available
(Section 3.1).  Here a small FP32 network (98 -> 256 -> 256 -> 256 -> 64)
maps cheap band statistics (diagonal histogram, Gershgorin interval, KPM
Chebyshev moments) to the equal-count slice boundaries; the library validates
each boundary with an exact inertia count and re-places the misses by
multisection.  Everything numeric runs in ``libpdeshep.so``; this module
marshals tensors, initialises parameters, asks the library for the training
labels (pdeshep_equal_count_targets) and stores weights.

Weights file: ``<path>.bin`` holds the raw little-endian float32 parameter
vector, ``<path>.json`` a header with the architecture and training metadata.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from dataclasses import dataclass

import numpy as np

from . import _band_args, _check, _np_ptr, _ptr, _stream, _torch, _workspace, load

N_FEAT = 98
N_HIDDEN = 256
N_OUT = 64
N_BOUNDS = N_OUT - 1
DIMS = (N_FEAT, N_HIDDEN, N_HIDDEN, N_HIDDEN, N_OUT)


def param_count() -> int:
    return int(load().pdeshep_mlp_param_count())


def layer_offsets():
    """[(W offset, bias offset, out, in)] for the four layers of the parameter vector."""
    off = 0
    out = []
    for l in range(4):
        fi, fo = DIMS[l], DIMS[l + 1]
        out.append((off, off + fo * fi, fo, fi))
        off += fo * fi + fo
    return out


def init_params(seed: int = 0, device="cuda", last_scale: float = 0.1):
    """He-normal weights, zero biases; the output layer scaled by ``last_scale``
    so that an untrained network proposes nearly equal widths."""
    torch = _torch()
    g = np.random.Generator(np.random.PCG64(int(seed)))
    p = np.zeros(param_count(), dtype=np.float32)
    for l, (wo, bo, fo, fi) in enumerate(layer_offsets()):
        w = g.normal(0.0, np.sqrt(2.0 / fi), size=(fo, fi))
        if l == 3:
            w *= last_scale
        p[wo: wo + fo * fi] = w.reshape(-1)
    return torch.from_numpy(p).to(device)


def features(band, seed: int = 0, b=None, stream=None):
    """98 float32 features of the band (see ``pdeshep_slice_features``)."""
    torch = _torch()
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    out = torch.empty(N_FEAT, dtype=torch.float32, device=band.device)
    ws = _workspace(lib.pdeshep_slice_features_workspace_size(n, cplx), band.device)
    st = lib.pdeshep_slice_features(n, b, cplx, _ptr(band), ldab, C.c_uint64(int(seed) & (2**64 - 1)), _ptr(out),
                                    _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_slice_features", st)
    return out


def _as_f32(t):
    torch = _torch()
    return t.to(torch.float32).contiguous()


def mlp_forward(params, X, stream=None):
    """Predicted boundaries (batch, 63) for features X (batch, 98)."""
    torch = _torch()
    lib = load()
    X = _as_f32(X.reshape(-1, N_FEAT))
    B = X.shape[0]
    out = torch.empty((B, N_BOUNDS), dtype=torch.float32, device=X.device)
    ws = _workspace(lib.pdeshep_mlp_workspace_size(B), X.device)
    st = lib.pdeshep_mlp_forward(_ptr(params), B, _ptr(X), _ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_mlp_forward", st)
    return out


def mlp_grad(params, X, T, stream=None):
    """(dL/dparams, L) for features X (batch, 98) and targets T (batch, 63)."""
    torch = _torch()
    lib = load()
    X = _as_f32(X.reshape(-1, N_FEAT))
    T = _as_f32(T.reshape(-1, N_BOUNDS))
    B = X.shape[0]
    grad = torch.empty_like(params)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    ws = _workspace(lib.pdeshep_mlp_workspace_size(B), X.device)
    st = lib.pdeshep_mlp_grad(_ptr(params), B, _ptr(X), _ptr(T), _ptr(grad), _ptr(loss), _ptr(ws), ws.numel(),
                              _stream(stream))
    _check("pdeshep_mlp_grad", st)
    return grad, loss


class Trainer:
    """Adam on the network parameters; every step runs in the library's kernels."""

    def __init__(self, params, lr: float = 1e-3, max_batch: int = 256):
        torch = _torch()
        self.params = params
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.lr = float(lr)
        self.t = 0
        self.ws = _workspace(load().pdeshep_mlp_workspace_size(int(max_batch)), params.device)
        self.max_batch = int(max_batch)
        self.loss = torch.zeros(1, dtype=torch.float32, device=params.device)

    def step(self, X, T, stream=None):
        lib = load()
        X = _as_f32(X.reshape(-1, N_FEAT))
        T = _as_f32(T.reshape(-1, N_BOUNDS))
        B = X.shape[0]
        assert B <= self.max_batch
        self.t += 1
        st = lib.pdeshep_mlp_train_step(_ptr(self.params), _ptr(self.m), _ptr(self.v), self.t, C.c_float(self.lr),
                                        B, _ptr(X), _ptr(T), _ptr(self.loss), _ptr(self.ws), self.ws.numel(),
                                        _stream(stream))
        _check("pdeshep_mlp_train_step", st)
        return self.loss


def equal_count_targets(band, nslices: int = N_OUT, rtol: float = 1e-7, b=None, stream=None, fanout: int = 8):
    """Training labels: the equal-count boundaries k n / nslices (k = 1..nslices-1), each the
    midpoint of the enclosures of eigenvalues t-1 and t (t = round(k n / nslices)), found by
    inertia bisection and normalised to the Gershgorin interval (pdeshep_equal_count_targets)."""
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    out = np.zeros(nslices - 1, dtype=np.float32)
    ws = _workspace(lib.pdeshep_equal_count_targets_workspace_size(n, b, cplx, nslices, fanout), band.device)
    st = lib.pdeshep_equal_count_targets(n, b, cplx, _ptr(band), ldab, int(nslices), float(rtol), int(fanout),
                                         _np_ptr(out), _ptr(ws), ws.numel(), _stream(stream))
    _check("pdeshep_equal_count_targets", st)
    return out


def train(bands, steps: int = 2000, batch: int = 64, lr: float = 1e-3, seed: int = 0, params=None,
          feature_seed: int = 0, log_every: int = 0, label_rtol: float = 1e-7):
    """Train on a list of bands (CUDA tensors).  Returns (params, losses, (X, T)).
    ``label_rtol``: relative accuracy of the eigenvalue enclosures behind the labels
    (regression targets only: 1e-4 of the spectrum is far below the network's error)."""
    torch = _torch()
    device = bands[0].device
    X = torch.stack([features(bd, seed=feature_seed) for bd in bands])
    T = torch.from_numpy(np.stack([equal_count_targets(bd, rtol=label_rtol) for bd in bands])).to(device)
    if params is None:
        params = init_params(seed, device)
    tr = Trainer(params, lr=lr, max_batch=batch)
    g = np.random.Generator(np.random.PCG64(int(seed) + 1))
    losses = []
    for s in range(steps):
        sel = torch.from_numpy(g.choice(len(bands), size=min(batch, len(bands)), replace=False)).to(device)
        loss = tr.step(X[sel], T[sel])
        if log_every and (s % log_every == 0 or s == steps - 1):
            losses.append((s, float(loss.item())))
    return tr.params, losses, (X, T)


@dataclass
class Proposal:
    bounds: np.ndarray        # nslices + 1 ascending shifts
    counts: np.ndarray        # exact eigenvalue count per slice
    used_fallback: int        # boundaries whose proposed count missed the target
    inertia_evals: int        # shifts evaluated (validation + fix-up)
    proposed_counts: np.ndarray = None  # exact count below each proposed boundary, before the fix-up


def propose_slices(band, params=None, nslices: int = N_OUT, frac=(0.0, 1.0), count_tol: int = 0,
                   fanout: int = 8, seed: int = 0, b=None, stream=None) -> Proposal:
    """Equal-count slices (see ``pdeshep_propose_slices``); ``params=None`` proposes
    equal widths over the Gershgorin interval instead of the network's boundaries."""
    lib = load()
    n, b, cplx, ldab = _band_args(band, b)
    bounds = np.zeros(nslices + 1)
    counts = np.zeros(nslices, dtype=np.int32)
    used = C.c_int32()
    evals = C.c_int64()
    proposed = np.zeros(nslices + 1, dtype=np.int64)
    ws = _workspace(lib.pdeshep_propose_workspace_size(n, b, cplx, nslices, fanout), band.device)
    st = lib.pdeshep_propose_slices(n, b, cplx, _ptr(band), ldab, _ptr(params),
                                    C.c_uint64(int(seed) & (2**64 - 1)), float(frac[0]), float(frac[1]),
                                    int(nslices), int(count_tol), int(fanout), _np_ptr(bounds), _np_ptr(counts),
                                    C.byref(used), C.byref(evals), _np_ptr(proposed), _ptr(ws), ws.numel(),
                                    _stream(stream))
    _check("pdeshep_propose_slices", st)
    return Proposal(bounds, counts, int(used.value), int(evals.value), proposed)


def save_params(path: str, params, meta: dict | None = None):
    """Write ``path.bin`` (float32 parameters) and ``path.json`` (header)."""
    p = params.detach().to("cpu").numpy().astype("<f4")
    with open(path + ".bin", "wb") as f:
        f.write(p.tobytes())
    head = {"format": "pdeshep-slicer-mlp", "dims": list(DIMS), "param_count": int(p.size),
            "activation": "relu", "head": "softmax-cumsum", "dtype": "float32-le"}
    head.update(meta or {})
    with open(path + ".json", "w") as f:
        json.dump(head, f, indent=1)


def load_params(path: str, device="cuda"):
    torch = _torch()
    with open(path + ".json") as f:
        head = json.load(f)
    if head.get("format") != "pdeshep-slicer-mlp" or list(head.get("dims", [])) != list(DIMS):
        raise ValueError(f"{path}.json: not a weights file of this network")
    p = np.fromfile(path + ".bin", dtype="<f4")
    if p.size != param_count():
        raise ValueError(f"{path}.bin: {p.size} parameters, expected {param_count()}")
    return torch.from_numpy(p.astype(np.float32)).to(device), head
