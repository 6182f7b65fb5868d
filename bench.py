#!/usr/bin/env python3
"""Benchmark: eigenpairs/s at residual <= 1e-10 for banded FEAST spectrum slicing.

Workload (the SCF-like sequence of complex Hermitian bands): n = 8192,
semi-bandwidth b = 64, B_{k+1} = B_k + 1e-3 E_k (E_k random Hermitian band,
entries N(0,1)); eight slices cover the lowest 20% of the spectrum (1638
eigenpairs); Ne = 8 Gauss-Legendre nodes per slice on an ellipse (ratio 0.3);
m0 = max(ceil(1.3 m_i), m_i + 10); every step is warm-started from the previous
step's eigenvectors and re-sliced at gap midpoints of the previous eigenvalues
(counts validated by exact inertia inside the call).

One timed step = one call of pdeshep_band_slice on the next matrix of the
sequence (inertia counts of all slices, complex64 shifted band LU and solves
with FP64 residual refinement, CholQR2 and Rayleigh-Ritz with FP64-class
products (tensor-core digit products for the tall and band products), until
every slice has its exact count of eigenpairs at residual <= 1e-10).  Inputs
are resident in HBM when timing starts; the factors (about 1.2 GB) exceed L2.

Also reported: the plain FP64 path on the same steps, an end-to-end variant
through the C ABI with host buffers, the dominant kernel group's achieved
throughput against its roofline, SM clocks sampled during the timed region, and
the CPU oracle on a bounded sample (--impl reference times only that).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

N, BW, NSLICE, NE, EPS, RHO = 8192, 64, 8, 8, 1e-3, 0.3
NEV = int(0.2 * N)  # 1638
TOL = 1e-10
SEED = synth.config_seed(2)
WORKLOAD = ("SCF sequence of complex Hermitian bands n=8192 b=64 (B_k+1 = B_k + 1e-3 E_k), 8 slices "
            "over the lowest 20% (1638 eigenpairs), Ne=8, m0=max(1.3m, m+10), warm start")
METRIC = ("eigenpairs/s at residual <= 1e-10 (mixed path: complex64 band LU/solves with FP64 residual refinement, "
          "tall Rayleigh-Ritz and band products as bf16 digit products on the tensor cores (FP64-class), "
          "float-float small products, FP64 inertia and eigensolver refinement; plain FP64 and mixed with "
          "float-float or FP64 Rayleigh-Ritz products reported alongside)")

# FP64 / FP32 ALU peaks from unit counts and clocks (152 SMs at 2070 MHz): FP32 = 152 x 128
# lanes x 2 flops x 2.07 GHz; FP64 = the part's 1.25 TFLOP/s figure.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25
# Float-float products: a complex multiply-add (8 algorithmic flops) costs 52 FP32-pipe
# instructions (4 real products x (2 for the exact product, 2 for the cross terms, 6 for the
# two-sum, 3 for the low word)); the FP32 pipes issue 152 x 128 x 2.07e9 instructions/s.
PEAK_FF_TFLOPS = 152 * 128 * 2.07e9 * 8 / 52 / 1e12
# Tensor-core tall products: 26 bf16 digit products per FP64-class product, so the usable peak is
# the measured sustained bf16 tensor rate (the GEMM runs inside a long step) divided by 26.
TC_DIGIT_PAIRS = 26


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback"


BF16_SUSTAINED_TFLOPS, BF16_PEAK_SOURCE = _measured_peaks()
PEAK_TC_TFLOPS = BF16_SUSTAINED_TFLOPS / TC_DIGIT_PAIRS
GROUP_BOUND = {"factor": ("alu", PEAK_FP32_TFLOPS, "fp32 from unit counts and clocks"),
               "solve": ("alu", PEAK_FP32_TFLOPS, "fp32 from unit counts and clocks"),
               "accum": ("hbm", None, None),
               "gemm": ("tensor", PEAK_TC_TFLOPS, "bf16 tensor cores (sustained, %s) / %d digit products per "
                        "FP64-class product" % (BF16_PEAK_SOURCE, TC_DIGIT_PAIRS)),
               "small": ("alu", PEAK_FP64_TFLOPS, "fp64 (part's figure)"),
               "bandmm": ("tensor", PEAK_TC_TFLOPS, "bf16 tensor cores (sustained, %s) / %d digit products per "
                          "FP64-class product" % (BF16_PEAK_SOURCE, TC_DIGIT_PAIRS)),
               "inertia": ("alu", PEAK_FP64_TFLOPS, "fp64 (part's figure)"),
               "eig": ("alu", PEAK_FP32_TFLOPS, "fp32 from unit counts and clocks")}


def boundary_indices():
    return [int(round(i * NEV / NSLICE)) for i in range(NSLICE + 1)]


def m0_rule(m):
    return max(int(math.ceil(1.3 * m - 1e-12)), m + 10)


def make_sequence(nmat):
    """B_0 .. B_{nmat-1} (host, complex128 bands)."""
    bands = [synth.random_band(N, BW, SEED, True, off_sigma=0.1)]
    for k in range(1, nmat):
        bands.append(bands[-1] + EPS * synth.perturbation(N, BW, SEED + k, True))
        bands[-1][:, 0] = bands[-1][:, 0].real
    return bands


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        med = float(np.median(sm)) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- GPU arm
class Sequence:
    """Runs the SCF sequence through pdeshep_band_slice on device-resident inputs."""

    def __init__(self, pk, torch, dev, nmat):
        self.pk, self.torch, self.dev = pk, torch, dev
        self.host = make_sequence(nmat)
        self.bands = [torch.from_numpy(a).to(dev) for a in self.host]
        self.bnorm = []
        for bd in self.bands:   # ||B_k||_2 of each input matrix (input property, computed before timing)
            lo, hi = pk.bisect(bd, [0, N - 1], rtol=1e-8, fanout=16)
            self.bnorm.append(max(abs(lo[0]), abs(hi[0]), abs(lo[1]), abs(hi[1])))
        ks = boundary_indices()
        # step 0 slicing: gap midpoints from GPU bisection on inertia
        idx = sorted(set([k for k in ks[1:]] + [k - 1 for k in ks[1:]] + [0]))
        lo, hi = pk.bisect(self.bands[0], idx, rtol=1e-12, fanout=8)
        lam = {k: 0.5 * (lo[i] + hi[i]) for i, k in enumerate(idx)}
        spacing = (lam[ks[1]] - lam[0]) / ks[1]
        self.bounds0 = [lam[0] - 2 * spacing] + [0.5 * (lam[k - 1] + lam[k]) for k in ks[1:]]
        counts = [ks[i + 1] - ks[i] for i in range(NSLICE)]
        self.m0 = np.array([m0_rule(c) for c in counts], dtype=np.int32)
        self.M = int(self.m0.sum())
        g = synth.rng(SEED + 999)
        x0 = (g.normal(size=(self.M, N)) + 1j * g.normal(size=(self.M, N))) / np.sqrt(2.0)
        self.x0 = torch.from_numpy(x0).to(dev)
        self.opts = dict(ne=NE, tol=TOL, ellipse_ratio=RHO, max_iter=40, autotune=1, rr_arith=pk.RR_TENSOR)
        self.ws = {}

    def next_bounds(self, res, bounds):
        """Boundaries for the next matrix from this step's eigenvalues (gap midpoints, Section 3.1)."""
        ev = res.evals.cpu().numpy()
        vals, off = [], 0
        above = []
        for i in range(NSLICE):
            k = int(res.nfound[i])
            vals.append(ev[off:off + k])
            rest = ev[off + k: off + self.m0[i]]
            above.append(rest[rest >= bounds[i + 1]])
            off += self.m0[i]
        lam = np.sort(np.concatenate(vals))
        nb = [bounds[0]]
        cum = 0
        ks = boundary_indices()
        for i in range(1, NSLICE):
            k = ks[i]
            nb.append(0.5 * (lam[k - 1] + lam[k]) if k < lam.size else bounds[i])
        nxt = np.min(above[-1]) if above[-1].size else bounds[-1] + 1e-4
        nb.append(0.5 * (lam[-1] + nxt) if lam.size == NEV else bounds[-1])
        return nb

    def workspace(self, precision, rr_arith=None):
        """Workspace for the given arithmetic (its size depends on both choices)."""
        rr = self.opts["rr_arith"] if rr_arith is None else rr_arith
        key = (precision, rr)
        if key not in self.ws:
            o = self.pk.default_opts(precision=precision, rr_arith=rr)
            nbytes = self.pk.workspace_size(N, BW, True, self.m0, NE, o)
            self.ws[key] = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.dev)
        return self.ws[key]

    def step(self, k, x0, bounds, precision, **extra):
        kw = dict(self.opts)
        kw.update(extra)
        return self.pk.band_slice(self.bands[k], bounds, self.m0, x0,
                                  workspace=self.workspace(precision, kw["rr_arith"]), bnorm=self.bnorm[k],
                                  precision=precision, raise_on_error=False, **kw)


def good_pairs(res, m0):
    return int(sum(int(res.nfound[i]) for i in range(len(m0)) if res.nfound[i] == res.counts[i]))


def reduce_over_ranks(dist, torch, dev, t_s, pairs):
    """Whole-job numbers of the replicas: the slowest rank's time and the pairs of all ranks
    (every rank runs its own copy of the workload; no collective inside the timed region)."""
    if not dist:
        return t_s, pairs
    t = torch.tensor([t_s], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    pt = torch.tensor([float(pairs)], device=dev, dtype=torch.float64)
    dist.all_reduce(pt, op=dist.ReduceOp.SUM)
    return float(t.item()), int(pt.item())


def run_gpu(args):
    import torch
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build as cb

    cb.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    W, K = args.warmup, args.steps
    seq = Sequence(pk, torch, dev, W + K + 1)
    stream = torch.cuda.current_stream()

    # warm-up: step 0 from random vectors, then warm-started steps
    x0, bounds = seq.x0, seq.bounds0
    for k in range(W):
        r = seq.step(k, x0, bounds, pk.MIXED)
        assert r.status == 0, ("warm-up step failed", k, r.status, r.counts, r.nfound)
        bounds = seq.next_bounds(r, bounds)
        x0 = r.evecs
    inputs = []   # (k, x0, bounds) of the timed steps, replayed by the FP64 and e2e legs
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = pk.kernel_launches()
    torch.cuda.synchronize()
    e0.record(stream)
    pairs = 0
    kg_ms = {g: 0.0 for g in pk.KERNEL_GROUPS}
    kg_fl = {g: 0.0 for g in pk.KERNEL_GROUPS}
    kg_n = {g: 0 for g in pk.KERNEL_GROUPS}
    iters, statuses, sweeps, eig_rep = [], [], [], []
    tuned_choice = {}
    for k in range(W, W + K):
        inputs.append((k, x0, bounds))
        r = seq.step(k, x0, bounds, pk.MIXED)
        statuses.append(r.status)
        pairs += good_pairs(r, seq.m0)
        iters.append(r.stats["iterations"])
        cluster_ctas = r.stats["cluster_ctas"]
        sweeps.append((r.stats["rr_calls"], r.stats["jacobi_sweeps32"], r.stats["jacobi_sweeps64"]))
        eig_rep.append({key: r.stats[key] for key in ("eig_refine_steps", "eig_clusters", "eig_max_cluster",
                                                    "eig_fallback_unconverged", "eig_fallback_wide")})
        tuned_choice = {"rhs_chunk": r.stats["rhs_chunk_used"], "gram_splits": r.stats["gram_splits_used"]}
        for g in pk.KERNEL_GROUPS:
            kg_ms[g] += r.stats["kg_ms"][g]
            kg_fl[g] += r.stats["kg_flops"][g]
            kg_n[g] += r.stats["kg_launches"][g]
        bounds = seq.next_bounds(r, bounds)
        x0 = r.evecs
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pk.kernel_launches() - l0
    clk = clocks.stop()
    t_s = e0.elapsed_time(e1) / 1e3
    t_s, pairs_all = reduce_over_ranks(dist, torch, dev, t_s, pairs)
    value = pairs_all / t_s

    # dominant kernel group and its roofline: the inertia counts run on a side stream under the
    # first filter pass (off the critical path), and the small eigensolver has no flop model
    # (Jacobi sweeps and refinement steps vary per block), so the roofline is reported for the
    # largest remaining group; every group's time is listed under kernel_groups.
    dom = max((g for g in kg_ms if g not in ("inertia", "eig")), key=lambda g: kg_ms[g])
    bound, peak, kind = GROUP_BOUND[dom]
    roof = None
    if kg_ms[dom] > 0:
        achieved = kg_fl[dom] / (kg_ms[dom] / 1e3) / 1e12
        roof = {"kernel_group": dom, "bound": bound, "achieved": round(achieved, 4), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None,
                "peak_kind": kind, "traffic": traffic_for(dom),
                "launches": kg_n[dom], "share_of_step": round(kg_ms[dom] / 1e3 / t_s, 4)}
    groups = {g: {"ms": round(kg_ms[g], 3), "launches": kg_n[g],
                  "tflops": round(kg_fl[g] / (kg_ms[g] / 1e3) / 1e12, 4) if kg_ms[g] > 0 else None}
              for g in pk.KERNEL_GROUPS}

    out = {"metric": METRIC,
           "value": round(value, 2), "unit": "eigenpairs/s", "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": round(t_s * 1e3 / K, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "c64+bf16x6+ff32x2+f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "b": BW, "slices": NSLICE, "ne": NE, "nev": NEV,
                      "m0": seq.m0.tolist(), "tol": TOL, "ellipse_ratio": RHO,
                      "l2": "inputs larger than L2 (factor set ~1.2 GB per step)",
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "iterations_per_step": iters, "status_per_step": statuses, "cluster_ctas": cluster_ctas,
           "rr_calls_sweeps32_sweeps64": sweeps,
           "eigensolver": eig_rep, "autotuned": tuned_choice,
           "kernel_groups": groups, "roofline": roof, "clocks": clk, "gpu_launches": int(launches)}

    if rank == 0 and not args.no_plain and args.plain_steps > 0:
        out["plain_fp64"] = plain_leg(pk, torch, seq, inputs[: args.plain_steps], stream)
        # mixed precision with the Rayleigh-Ritz products kept in FP64 arithmetic
        out["mixed_rr_floatfloat"] = plain_leg(pk, torch, seq, inputs[: args.plain_steps], stream,
                                               precision=pk.MIXED, dtype="c64+ff32x2+f64",
                                               rr_arith=pk.RR_FLOATFLOAT)
        out["mixed_rr_fp64"] = plain_leg(pk, torch, seq, inputs[: args.plain_steps], stream, precision=pk.MIXED,
                                         dtype="c64+f64", rr_arith=pk.RR_FP64)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(pk, torch, seq, inputs[: max(1, min(K, args.e2e_steps))], stream)
    if rank == 0 and not args.no_proposal:
        out["slice_proposal"] = proposal_leg(pk, torch, dev)
    if rank == 0:
        out["partition_report"] = partition_report(pk, r, seq)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(seq.host, seq.bounds0, seq.m0, seq.bnorm[0])
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def plain_leg(pk, torch, seq, inputs, stream, precision=None, dtype="c128+f64", **extra):
    """The same steps timed with another arithmetic (plain FP64 by default)."""
    precision = pk.FP64 if precision is None else precision
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    seq.workspace(precision, extra.get("rr_arith"))
    seq.step(*inputs[0], precision, **extra)     # untimed: tunes this arithmetic's choices
    torch.cuda.synchronize()
    e0.record(stream)
    pairs, iters = 0, []
    for k, x0, bounds in inputs:
        r = seq.step(k, x0, bounds, precision, **extra)
        pairs += good_pairs(r, seq.m0)
        iters.append(r.stats["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    return {"value": round(pairs / t, 2), "unit": "eigenpairs/s", "steps": len(inputs),
            "ms_per_step": round(t * 1e3 / len(inputs), 3), "iterations_per_step": iters,
            "dtype": dtype}


def partition_report(pk, res, seq):
    """The paper's re-slicing (Algorithm 3, simplified 1-D k-means) against the equal-count
    re-slicing the sequence uses, on the eigenvalues of the last timed step (host work only):
    counts per slice, the distance from the inner boundaries to the nearest eigenvalue in units
    of the median spacing, sweeps and host time."""
    try:
        ev = res.evals.cpu().numpy()
        vals, off = [], 0
        for i in range(NSLICE):
            k = int(res.nfound[i])
            vals.append(ev[off:off + k])
            off += int(seq.m0[i])
        lam = np.sort(np.concatenate(vals))
        spacing = float(np.median(np.diff(lam)))
        b0, bK = float(lam[0] - spacing), float(lam[-1] + spacing)
        out = {"eigenvalues": int(lam.size), "slices": NSLICE}
        for name, method in (("equal_counts", pk.PART_EQUAL_COUNT), ("kmeans", pk.PART_KMEANS)):
            t0 = time.perf_counter()
            b, c, sweeps = pk.partition(lam, NSLICE, b0, bK, method=method)
            us = (time.perf_counter() - t0) * 1e6
            gaps = [float(np.min(np.abs(lam - x))) / spacing for x in b[1:-1]]
            out[name] = {"counts_min": int(c.min()), "counts_max": int(c.max()),
                         "min_gap_spacings": round(min(gaps), 3), "median_gap_spacings": round(float(np.median(gaps)), 3),
                         "sweeps": sweeps, "host_us": round(us, 1)}
        return out
    except Exception as e:  # a report only: never let it break the bench line
        return {"error": repr(e)}


def proposal_leg(pk, torch, dev):
    """Learned slice proposal at the proposer's configuration (complex mixture bands, n = 16384,
    b = 64, 64 equal-count slices), reported beside the FEAST metric.  The network is trained here
    on 128 smaller spectra of the same generator and bandwidth (n = 1024, b = 64; the features are
    scale-free in n), labels by inertia bisection to 1e-4 relative, 1500 Adam steps; then held-out
    bands are sliced with the network and with equal widths (the no-network baseline); counts are
    exact in both."""
    from paper_2012_00506_gb300 import slicer

    def family(seed, n, b):
        g = np.random.default_rng(seed)
        k = int(g.integers(1, 7))
        return synth.mixture_band(n, b, seed, is_complex=True, ncomp=k, comp_sigma=float(g.uniform(0.01, 0.2)),
                                  off_sigma=float(g.uniform(0.005, 0.03)), means=g.uniform(-1.0, 1.0, size=k),
                                  weights=g.dirichlet(np.ones(k)))

    t0 = time.perf_counter()
    train = [torch.from_numpy(family(synth.config_seed(4) + s, 1024, 64)).to(dev) for s in range(128)]
    params, losses, _ = slicer.train(train, steps=1500, batch=64, lr=1e-3, seed=0, log_every=1499, label_rtol=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    res = {"mlp": [], "none": []}
    n, nsl = 16384, 64
    tgt = np.floor(n * np.arange(nsl + 1) / nsl + 0.5).astype(int)
    for s in range(3):
        band = torch.from_numpy(family(synth.config_seed(4) + 10000 + s, n, 64)).to(dev)
        for name, p in (("mlp", params), ("none", None)):
            slicer.propose_slices(band, p, nslices=nsl, count_tol=16)          # warm
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            pr = slicer.propose_slices(band, p, nslices=nsl, count_tol=16)
            t = time.perf_counter() - t1
            res[name].append((t, pr.inertia_evals, pr.used_fallback,
                              float(np.mean(np.abs(pr.proposed_counts - tgt)[1:-1])), int(pr.counts.sum())))
    out = {"config": "complex mixture bands n=16384 b=64, 64 slices, count tolerance 16", "train_seconds":
           round(t_train, 2), "train_loss": [round(l, 6) for _, l in losses]}
    for name in ("mlp", "none"):
        r = np.array([x[:4] for x in res[name]])
        out[name] = {"ms": round(1e3 * float(np.mean(r[:, 0])), 2), "inertia_evals": float(np.mean(r[:, 1])),
                     "boundaries_fixed": float(np.mean(r[:, 2])), "proposal_count_error": round(float(np.mean(r[:, 3])), 1)}
    return out


def e2e_leg(pk, torch, seq, inputs, stream):
    """Same metric through the C ABI with host buffers: pinned host band and start vectors copied in,
    eigenvalues and eigenvectors copied out, every step inside the timed region."""
    hb = [torch.from_numpy(seq.host[k]).pin_memory() for k, _, _ in inputs]
    hx = [x0.cpu().pin_memory() for _, x0, _ in inputs]
    dband = torch.empty_like(seq.bands[0])
    dx = torch.empty_like(inputs[0][1])
    ev_h = torch.empty(seq.M, dtype=torch.float64).pin_memory()
    vec_h = torch.empty((seq.M, N), dtype=torch.complex128).pin_memory()
    h2d = hb[0].numel() * 16 + hx[0].numel() * 16
    d2h = ev_h.numel() * 8 + vec_h.numel() * 16
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    pairs = 0
    for i, (k, _, bounds) in enumerate(inputs):
        dband.copy_(hb[i], non_blocking=True)
        dx.copy_(hx[i], non_blocking=True)
        r = seq.pk.band_slice(dband, bounds, seq.m0, dx, workspace=seq.workspace(pk.MIXED), bnorm=seq.bnorm[k],
                              precision=pk.MIXED, raise_on_error=False, **seq.opts)
        ev_h.copy_(r.evals, non_blocking=True)
        vec_h.copy_(r.evecs, non_blocking=True)
        pairs += good_pairs(r, seq.m0)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    return {"value": round(pairs / t, 2), "unit": "eigenpairs/s", "steps": len(inputs),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def traffic_for(group):
    """DRAM bytes per launch of the group's main kernel from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(group)
    if not ent or ent.get("workload") != WORKLOAD_KEY or ent.get("source_hash") != source_hash(group):
        return None
    return ent.get("dram_bytes_per_launch")


WORKLOAD_KEY = "c2"
GROUP_SOURCES = {"solve": "band_lu.cu", "factor": "band_lu.cu", "gemm": "tcgemm.cu", "small": "dense.cu",
                 "bandmm": "tcgemm.cu", "accum": "feast.cu", "inertia": "inertia.cu", "eig": "dense.cu"}


def source_hash(group):
    import hashlib
    p = os.path.join(ROOT, "paper_2012_00506_gb300", "csrc", GROUP_SOURCES.get(group, "feast.cu"))
    try:
        return hashlib.sha1(open(p, "rb").read()).hexdigest()[:12]
    except OSError:
        return None


# ----------------------------------------------------------------------------- CPU oracle leg
ORACLE_SAMPLE = ("one FEAST iteration (8 nodes: band LU, normal and adjoint solves for m0 right-hand sides, "
                 "CholQR2, Rayleigh-Ritz) of slice 0 of the first matrix of the sequence; eigenpairs/s = "
                 "slice count / iteration time, an upper bound on the oracle's throughput (it needs several "
                 "iterations to converge)")


def cpu_baseline(host_bands, bounds, m0, bnorm):
    import oracle
    oracle.build()
    ab = host_bands[0]
    cnt = boundary_indices()[1] - boundary_indices()[0]
    x0 = synth.random_subspace(N, int(m0[0]), SEED + 5, True)
    t0 = time.perf_counter()
    oracle.feast_slice(ab, bounds[0], bounds[1], x0, ne=NE, rho=RHO, tol=TOL, bnorm=bnorm, max_iter=1, count=cnt)
    t = time.perf_counter() - t0
    return {"value": round(cnt / t, 4), "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
            "sample": ORACLE_SAMPLE, "seconds": round(t, 2)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    host = make_sequence(1)
    ab = host[0]
    ks = boundary_indices()
    # slice boundaries from the oracle's own bisection on inertia (tolerance 1e-9)
    lam = {}
    for k in sorted(set([0] + ks[1:2] + [ks[1] - 1])):
        lo, hi = oracle.eig_by_bisection(ab, k, 1e-9)
        lam[k] = 0.5 * (lo + hi)
    spacing = (lam[ks[1]] - lam[0]) / ks[1]
    b0, b1 = lam[0] - 2 * spacing, 0.5 * (lam[ks[1] - 1] + lam[ks[1]])
    bnorm = 1.0
    lo, hi = oracle.gershgorin(ab)
    cnt = ks[1]
    m0 = m0_rule(cnt)
    for _ in range(args.warmup):
        x = synth.random_subspace(256, 8, 1, True)
        oracle.feast_slice(synth.random_band(256, 4, 1, True), -0.1, 0.1, x, max_iter=1, bnorm=1.0)
    times = []
    for s in range(args.steps):
        x0 = synth.random_subspace(N, m0, SEED + 100 + s, True)
        t0 = time.perf_counter()
        oracle.feast_slice(ab, b0, b1, x0, ne=NE, rho=RHO, tol=TOL, bnorm=max(abs(lo), abs(hi)), max_iter=1,
                           count=cnt)
        times.append(time.perf_counter() - t0)
    t = float(np.sum(times))
    value = cnt * len(times) / t
    out = {"impl": "reference", "metric": METRIC,
           "value": round(value, 4), "unit": "eigenpairs/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t * 1e3 / len(times), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "b": BW, "slices": NSLICE, "ne": NE},
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": ORACLE_SAMPLE, "value": round(value, 4)},
           "e2e": {"value": round(value, 4), "unit": "eigenpairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def profile_case(args):
    """A reduced instance of the bench workload for ncu captures: the first matrix of the
    sequence, the first `--profile-slices` slices of its partition (same n, b, m0, Ne),
    random start vectors, two band_slice calls (the second with resident tuning choices)."""
    import torch
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build as cb

    cb.build()
    dev = torch.device("cuda:0")
    ab = make_sequence(1)[0]
    band = torch.from_numpy(ab).to(dev)
    ks = boundary_indices()[: args.profile_slices + 1]
    idx = sorted(set([k for k in ks[1:]] + [k - 1 for k in ks[1:]] + [0]))
    lo, hi = pk.bisect(band, idx, rtol=1e-12, fanout=8)
    lam = {k: 0.5 * (lo[i] + hi[i]) for i, k in enumerate(idx)}
    spacing = (lam[ks[1]] - lam[0]) / ks[1]
    bounds = [lam[0] - 2 * spacing] + [0.5 * (lam[k - 1] + lam[k]) for k in ks[1:]]
    m0 = [m0_rule(ks[i + 1] - ks[i]) for i in range(args.profile_slices)]
    g = synth.rng(SEED + 999)
    x0 = torch.from_numpy((g.normal(size=(sum(m0), N)) + 1j * g.normal(size=(sum(m0), N))) / np.sqrt(2.0)).to(dev)
    lo2, hi2 = pk.bisect(band, [0, N - 1], rtol=1e-8, fanout=16)
    bn = max(abs(lo2[0]), abs(hi2[0]), abs(lo2[1]), abs(hi2[1]))
    for rep in range(2):
        r = pk.band_slice(band, bounds, m0, x0, bnorm=bn, precision=pk.MIXED, ne=NE, tol=TOL, ellipse_ratio=RHO,
                          max_iter=40, autotune=1, raise_on_error=False)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": WORKLOAD_KEY, "slices": args.profile_slices, "m0": m0, "status": r.status,
                      "nfound": [int(v) for v in r.nfound], "counts": [int(v) for v in r.counts]}))
    if r.status != 0 or list(r.nfound) != list(r.counts):
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-proposal", action="store_true", help="skip the slice-proposal report")
    ap.add_argument("--profile-case", action="store_true",
                    help="run a reduced instance of the workload (for ncu captures) instead of the bench")
    ap.add_argument("--profile-slices", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 1:
        args.warmup = 1
    if args.profile_case:
        profile_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
