#!/usr/bin/env python3
"""Benchmark: eigenpairs/s at residual <= 1e-10 for banded FEAST spectrum slicing.

Headline workload (the largest single-GPU configuration): 20-step SCF-like
sequence of complex Hermitian bands, n = 65536, semi-bandwidth b = 128,
B_0 with a clustered spectrum (diagonal from a mixture of 4 Gaussians,
sigma = 0.05; off-diagonals N(0, 0.02^2)), B_{k+1} = B_k + 1e-3 E_k (E_k a
random Hermitian band, entries N(0,1)); 128 slices over the lowest 30 % of the
spectrum (19661 eigenpairs), proposed for B_0 by the learned slice proposer
(exact inertia counts, multisection fall-back) and re-sliced for every later
matrix at gap midpoints of the previous eigenvalues; Ne = 16 Gauss-Legendre
nodes per slice on an ellipse (ratio 0.3); m0 = max(ceil(1.3 m_i), m_i + 10);
the first matrix starts from library-drawn random vectors, every later one from
the previous matrix's eigenvectors.

One timed step = one pdeshep_band_slice call on the next group of 16 slices of
the current matrix (8 steps per matrix): exact inertia counts, 256 complex64
shifted band factorizations kept resident (104 GB, under the 150 GB factor
cap) and their solves with FP64 residual refinement, CholQR and Rayleigh-Ritz
with FP64-class products, until every slice of the group has its exact count
of eigenpairs at residual <= 1e-10.  Inputs are resident in HBM when timing
starts and far exceed L2.  ||B_k||_2 of each matrix (the residual's
normalisation) is an input property computed before timing; its cost is
reported.

Also reported: the same sequence on the second configuration (n = 8192,
b = 64, 8 slices over the lowest 20 %, Ne = 8, one matrix per step) with plain
FP64 and the other Rayleigh-Ritz arithmetics beside it; plain FP64 on a sample
of the headline workload; end-to-end variants through the C ABI with host
buffers; the dominant kernel group's achieved throughput against its measured
roofline; SM clocks sampled during the timed region; the FP32-class error of
the unrefined path; the slice proposer; and the CPU oracle on a bounded sample
over the host cores (--impl reference times only that).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
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

TOL, RHO, EPS = 1e-10, 0.3, 1e-3


class Config:
    def __init__(self, key, n, b, nslices, group, ne, frac, gen, cap, slicing, seed, workload):
        self.key, self.n, self.b, self.nslices, self.group, self.ne = key, n, b, nslices, group, ne
        self.frac, self.gen, self.cap, self.slicing, self.seed, self.workload = frac, gen, cap, slicing, seed, workload
        self.nev = int(round(frac * n))
        self.groups = nslices // group

    def targets(self):
        """Equal-count boundary indices k * nev / nslices."""
        return [int(round(i * self.nev / self.nslices)) for i in range(self.nslices + 1)]


C5 = Config("c5", 65536, 128, 128, 16, 16, 0.3, "mixture", 150 << 30, "mlp", synth.config_seed(5),
            "SCF sequence of complex Hermitian bands n=65536 b=128 (clustered B_0, B_k+1 = B_k + 1e-3 E_k), "
            "128 learned-proposal slices over the lowest 30% (19661 eigenpairs), Ne=16, m0=max(1.3m, m+10), warm "
            "start; one step = one call on 16 slices (8 steps per matrix), factors resident under a 150 GB cap")
C2 = Config("c2", 8192, 64, 8, 8, 8, 0.2, "random", 0, "bisect", synth.config_seed(2),
            "SCF sequence of complex Hermitian bands n=8192 b=64 (B_k+1 = B_k + 1e-3 E_k), 8 slices over the "
            "lowest 20% (1638 eigenpairs), Ne=8, m0=max(1.3m, m+10), warm start; one step = one matrix")
CONFIGS = {"c5": C5, "c2": C2}

METRIC = ("eigenpairs/s at residual <= 1e-10 (mixed path: complex64 band LU and solves with FP64 residual "
          "refinement, the solve tiles of the first four filter passes as bf16x6 products on the tensor cores "
          "(FP32-class), tall Rayleigh-Ritz and band products as bf16 digit products on the tensor cores "
          "(FP64-class), float-float small products, FP64 inertia and eigensolver refinement; plain FP64 reported "
          "alongside)")
DTYPE = "c64+bf16x6+ff32x2+f64"

# Tensor-core tall products: 26 bf16 digit products per FP64-class product, so the usable peak is
# the measured sustained bf16 tensor rate (the GEMM runs inside a long step) divided by 26.
TC_DIGIT_PAIRS = 26


def _measured_bf16():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "of measured"
    except (OSError, KeyError, ValueError):
        return 1700.0, "of fallback"


BF16_SUSTAINED_TFLOPS, BF16_PEAK_SOURCE = _measured_bf16()
PEAK_TC_TFLOPS = BF16_SUSTAINED_TFLOPS / TC_DIGIT_PAIRS


def group_bounds(peaks):
    """(bound, peak TFLOP/s, what the peak is) per kernel group; the ALU peaks are measured on this
    GPU by pdeshep_alu_peak at the start of the run."""
    fp32, fp64 = peaks["fp32_tflops"], peaks["fp64_tflops"]
    # float-float: a complex multiply-add (8 algorithmic flops) costs 52 FP32-pipe instructions
    ff = fp32 / 2 * 8 / 52
    tc = ("tensor", PEAK_TC_TFLOPS, "bf16 tensor cores (sustained, %s) / %d digit products per FP64-class "
          "product" % (BF16_PEAK_SOURCE, TC_DIGIT_PAIRS))
    return {"factor": ("alu", fp32, "fp32 FMA, measured"), "solve": ("alu", fp32, "fp32 FMA, measured"),
            "accum": ("alu", fp64, "fp64 FMA, measured"), "gemm": tc, "bandmm": tc,
            "small": ("alu", fp64, "fp64 FMA, measured"), "inertia": ("alu", fp64, "fp64 FMA, measured"),
            "eig": ("alu", fp32, "fp32 FMA, measured (flops: FP32 Jacobi rotations only)"),
            "_ff": ff}


def m0_rule(m):
    return max(int(math.ceil(1.3 * m - 1e-12)), m + 10)


def make_matrix(cfg, k, prev=None):
    """B_k of the sequence (host, complex128 lower band)."""
    if k == 0:
        if cfg.gen == "mixture":
            return synth.mixture_band(cfg.n, cfg.b, cfg.seed, is_complex=True, off_sigma=0.02)
        return synth.random_band(cfg.n, cfg.b, cfg.seed, True, off_sigma=0.1)
    a = prev + EPS * synth.perturbation(cfg.n, cfg.b, cfg.seed + k, True)
    a[:, 0] = a[:, 0].real
    return a


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


# ----------------------------------------------------------------------------- the sequence
class Sequence:
    """Runs a configuration's SCF sequence through pdeshep_band_slice, one slice group per step,
    on device-resident inputs."""

    def __init__(self, pk, torch, dev, cfg, nsteps, proposer=None):
        self.pk, self.torch, self.dev, self.cfg = pk, torch, dev, cfg
        self.nmat = nsteps // cfg.groups + 2
        self.host = [make_matrix(cfg, 0)]
        for k in range(1, self.nmat):
            self.host.append(make_matrix(cfg, k, self.host[-1]))
        self.bands = [torch.from_numpy(a).to(dev) for a in self.host]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.bnorm = [self._bnorm(bd) for bd in self.bands]
        self.bnorm_ms = (time.perf_counter() - t0) * 1e3 / len(self.bands)
        ks = cfg.targets()
        self.m0 = np.array([m0_rule(ks[i + 1] - ks[i]) for i in range(cfg.nslices)], dtype=np.int32)
        self.col = np.concatenate([[0], np.cumsum(self.m0)]).astype(np.int64)
        self.proposal = None
        self.bounds0 = self._first_bounds(proposer)
        self.opts = dict(ne=cfg.ne, tol=TOL, ellipse_ratio=RHO, max_iter=40, autotune=1, rr_arith=pk.RR_TENSOR,
                         hbm_cap_bytes=cfg.cap)
        self.ws = {}

    def _bnorm(self, band):
        # to 1e-6 relative: the residual test at 1e-10 moves by at most 1e-6 of itself
        lo, hi = self.pk.bisect(band, [0, self.cfg.n - 1], rtol=1e-6, fanout=16)
        return max(abs(lo[0]), abs(hi[0]), abs(lo[1]), abs(hi[1]))

    def _first_bounds(self, proposer):
        cfg, pk = self.cfg, self.pk
        ks = cfg.targets()
        band = self.bands[0]
        lo0, hi0 = pk.bisect(band, [0], rtol=1e-12, fanout=8)
        lam0 = 0.5 * (lo0[0] + hi0[0])
        if cfg.slicing == "mlp":
            from paper_2012_00506_gb300 import slicer
            self.torch.cuda.synchronize()
            t0 = time.perf_counter()
            pr = slicer.propose_slices(band, proposer, nslices=cfg.nslices, frac=(0.0, cfg.frac), count_tol=16)
            self.torch.cuda.synchronize()
            tg = np.array(ks)
            self.proposal = {"ms": round((time.perf_counter() - t0) * 1e3, 1), "inertia_evals": pr.inertia_evals,
                             "boundaries_fixed": pr.used_fallback,
                             "proposal_count_error": round(float(np.mean(np.abs(pr.proposed_counts - tg)[1:-1])), 1),
                             "final_count_error_max": int(np.max(np.abs(np.cumsum(np.concatenate([[0], pr.counts]))
                                                                         - tg)))}
            b = np.array(pr.bounds, dtype=np.float64)
            spacing = (b[1] - lam0) / max(1, int(pr.counts[0]))
            b[0] = lam0 - 2 * spacing            # tight lower end (the proposal's sits below Gershgorin)
            return b.tolist()
        idx = sorted(set([k for k in ks[1:]] + [k - 1 for k in ks[1:]]))
        lo, hi = pk.bisect(band, idx, rtol=1e-12, fanout=8)
        lam = {k: 0.5 * (lo[i] + hi[i]) for i, k in enumerate(idx)}
        spacing = (lam[ks[1]] - lam0) / ks[1]
        return [lam0 - 2 * spacing] + [0.5 * (lam[k - 1] + lam[k]) for k in ks[1:]]

    def next_bounds(self, results, bounds):
        """Boundaries for the next matrix from this matrix's eigenvalues (equal counts at gap
        midpoints, Section 3.1).  results: the slice groups' results in order."""
        cfg = self.cfg
        vals, above = [], None
        for g, r in enumerate(results):
            ev = r.evals.cpu().numpy()
            for j in range(cfg.group):
                i = g * cfg.group + j
                off = int(self.col[i] - self.col[g * cfg.group])
                k = int(r.nfound[j])
                vals.append(ev[off:off + k])
                if i == cfg.nslices - 1:
                    rest = ev[off + k: off + int(self.m0[i])]
                    above = rest[rest >= bounds[i + 1]]
        lam = np.sort(np.concatenate(vals))
        ks = cfg.targets()
        nb = [bounds[0]]
        for i in range(1, cfg.nslices):
            k = ks[i]
            nb.append(0.5 * (lam[k - 1] + lam[k]) if k < lam.size else bounds[i])
        nxt = np.min(above) if above is not None and above.size else bounds[-1] + 1e-4
        nb.append(0.5 * (lam[-1] + nxt) if lam.size == cfg.nev else bounds[-1])
        return nb

    def group_m0(self, g):
        return self.m0[g * self.cfg.group:(g + 1) * self.cfg.group]

    def workspace(self, precision, rr_arith=None, nsl=None):
        rr = self.opts["rr_arith"] if rr_arith is None else rr_arith
        nsl = self.cfg.group if nsl is None else nsl
        key = (precision, rr, nsl)
        if key not in self.ws:
            o = self.pk.default_opts(precision=precision, rr_arith=rr, hbm_cap_bytes=self.cfg.cap)
            gs = self.cfg.group
            nbytes = max(self.pk.workspace_size(self.cfg.n, self.cfg.b, True, self.m0[g * gs:g * gs + nsl],
                                                self.cfg.ne, o) for g in range(self.cfg.groups))
            self.ws[key] = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.dev)
        return self.ws[key]

    def call(self, k, g, x0, bounds, precision, band=None, nsl=None, **extra):
        """One slice group (the first nsl slices of group g) of matrix k."""
        cfg = self.cfg
        kw = dict(self.opts)
        kw.update(extra)
        nsl = cfg.group if nsl is None else nsl
        s0 = g * cfg.group
        return self.pk.band_slice(self.bands[k] if band is None else band, bounds[s0:s0 + nsl + 1],
                                  self.m0[s0:s0 + nsl], x0, workspace=self.workspace(precision, kw["rr_arith"], nsl),
                                  bnorm=self.bnorm[k], precision=precision, raise_on_error=False,
                                  seed=cfg.seed + 1000 * k + g, **kw)


def good_pairs(res):
    return int(sum(int(res.nfound[i]) for i in range(len(res.nfound)) if res.nfound[i] == res.counts[i]))


class Walker:
    """Steps through the (matrix, group) sequence: start vectors and boundaries of each step."""

    def __init__(self, seq):
        self.seq = seq
        self.k, self.g = 0, 0
        self.bounds = seq.bounds0
        self.prev = None          # evecs of the previous matrix, per group
        self.cur = []             # results of the current matrix
        self.cur_x0 = []

    def inputs(self):
        x0 = None if self.prev is None else self.prev[self.g]
        return self.k, self.g, x0, self.bounds

    def advance(self, r):
        self.cur.append(r)
        self.g += 1
        if self.g == self.seq.cfg.groups:
            self.bounds = self.seq.next_bounds(self.cur, self.bounds)
            self.prev = [c.evecs for c in self.cur]
            self.cur = []
            self.k += 1
            self.g = 0


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


def eig_flops(m0_list, cplx, sweeps32):
    """Algorithmic flops of the FP32 Jacobi sweeps: per rotation the 2x2 unitary is applied to two
    rows, two columns and two eigenvector columns (m entries each, 2 outputs of 2 complex products
    + 1 addition = 28 flops per entry pair, 6 real flops for real data), m(m-1)/2 rotations per
    sweep."""
    per = 84 if cplx else 18
    return sum(per * m * m * (m - 1) / 2.0 for m in m0_list) * sweeps32


def run_sequence(pk, torch, seq, W, K, stream, clocks=None, dist=None, dev=None):
    """W untimed steps, then K timed steps; returns the measurement and the inputs of the timed steps."""
    walk = Walker(seq)
    for _ in range(W):
        k, g, x0, bounds = walk.inputs()
        r = seq.call(k, g, x0, bounds, pk.MIXED)
        assert r.status == 0, ("warm-up step failed", seq.cfg.key, k, g, r.status, r.counts, r.nfound)
        walk.advance(r)
    inputs = []
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    if clocks:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = pk.kernel_launches()
    torch.cuda.synchronize()
    e0.record(stream)
    pairs = 0
    kg_ms = {gname: 0.0 for gname in pk.KERNEL_GROUPS}
    kg_fl = {gname: 0.0 for gname in pk.KERNEL_GROUPS}
    kg_n = {gname: 0 for gname in pk.KERNEL_GROUPS}
    iters, statuses, eig_rep, tuned, step_ms, warm = [], [], [], {}, [], []
    for _ in range(K):
        k, g, x0, bounds = walk.inputs()
        inputs.append((k, g, x0, bounds))
        r = seq.call(k, g, x0, bounds, pk.MIXED)
        statuses.append(r.status)
        pairs += good_pairs(r)
        iters.append(r.stats["iterations"])
        step_ms.append(round(r.stats["ms_total"], 1))
        warm.append(x0 is not None)
        eig_rep.append((r.stats["rr_calls"], r.stats["jacobi_sweeps32"], r.stats["eig_refine_steps"],
                        r.stats["eig_fallback_unconverged"] + r.stats["eig_fallback_wide"]))
        tuned = {"rhs_chunk": r.stats["rhs_chunk_used"], "rhs_chunk_early": r.stats["rhs_chunk_early"],
                 "gram_splits": r.stats["gram_splits_used"]}
        for gname in pk.KERNEL_GROUPS:
            kg_ms[gname] += r.stats["kg_ms"][gname]
            kg_fl[gname] += r.stats["kg_flops"][gname]
            kg_n[gname] += r.stats["kg_launches"][gname]
        kg_fl["eig"] += eig_flops(seq.group_m0(g), True, r.stats["jacobi_sweeps32"])
        walk.advance(r)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = pk.kernel_launches() - l0
    clk = clocks.stop() if clocks else None
    t_s = e0.elapsed_time(e1) / 1e3
    t_s, pairs = reduce_over_ranks(dist, torch, dev, t_s, pairs)
    return dict(t_s=t_s, pairs=pairs, kg_ms=kg_ms, kg_fl=kg_fl, kg_n=kg_n, iters=iters, statuses=statuses,
                eig=eig_rep, tuned=tuned, launches=int(launches), clocks=clk, last=r, step_ms=step_ms,
                warm=warm), inputs


def solve_bound(bounds_tbl, tuned):
    """The solve group's roofline: the tensor-core solve (bf16x6 products, FP32-class) when the
    autotuner chose it for the early passes, else the FP32 FMA pipe."""
    tb = dict(bounds_tbl)
    if tuned.get("rhs_chunk_early") == 256 or tuned.get("rhs_chunk") == 256:
        tb["solve"] = ("tensor", BF16_SUSTAINED_TFLOPS / 6,
                       "bf16 tensor cores (sustained, %s) / 6 bf16 products per FP32-class product (bf16x6); "
                       "the group also holds the round-to-nearest passes after the fourth on the FP32 pipe"
                       % BF16_PEAK_SOURCE)
    return tb


def roofline(meas, bounds_tbl, traffic_key):
    kg_ms, kg_fl, kg_n, t_s = meas["kg_ms"], meas["kg_fl"], meas["kg_n"], meas["t_s"]
    bounds_tbl = solve_bound(bounds_tbl, meas["tuned"])
    # the inertia counts run on a side stream beside the first filter pass (off the critical path)
    dom = max((gname for gname in kg_ms if gname != "inertia"), key=lambda gname: kg_ms[gname])
    bound, peak, kind = bounds_tbl[dom]
    roof = None
    if kg_ms[dom] > 0:
        achieved = kg_fl[dom] / (kg_ms[dom] / 1e3) / 1e12
        roof = {"kernel_group": dom, "bound": bound, "achieved": round(achieved, 4), "peak": round(peak, 3),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4) if peak else None,
                "peak_kind": kind, "traffic": traffic_for(dom, traffic_key),
                "launches": kg_n[dom], "share_of_step": round(kg_ms[dom] / 1e3 / t_s, 4)}
    groups = {}
    for gname in kg_ms:
        tf = kg_fl[gname] / (kg_ms[gname] / 1e3) / 1e12 if kg_ms[gname] > 0 and kg_fl[gname] > 0 else None
        b_, p_, _ = bounds_tbl[gname]
        groups[gname] = {"ms": round(kg_ms[gname], 3), "launches": kg_n[gname],
                         "tflops": round(tf, 4) if tf else None,
                         "frac": round(tf / p_, 4) if tf and p_ else None}
    return roof, groups


def run_gpu(args):
    import torch
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build as cb

    cb.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle's pool starts before any GPU work (a process forked after it would hang)
    pool = None
    if rank == 0 and not args.no_cpu_baseline:
        pool = mp.get_context("spawn").Pool(oracle_cores())
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    W, K = args.warmup, args.steps
    stream = torch.cuda.current_stream()
    peaks = {"fp32_tflops": round(pk.alu_peak(False, 4096, device=dev), 2),
             "fp64_tflops": round(pk.alu_peak(True, 1024, device=dev), 3),
             "bf16_tflops_sustained": BF16_SUSTAINED_TFLOPS, "bf16_source": BF16_PEAK_SOURCE}
    btab = group_bounds(peaks)
    cfg = CONFIGS[args.workload]

    proposer, prop_report = None, None
    if cfg.slicing == "mlp" or (rank == 0 and not args.no_proposal):
        proposer, prop_report = train_proposer(pk, torch, dev, args)
    seq = Sequence(pk, torch, dev, cfg, W + K, proposer)
    clocks = ClockSampler(local)
    meas, inputs = run_sequence(pk, torch, seq, W, K, stream, clocks, dist, dev)
    value = meas["pairs"] / meas["t_s"]
    roof, groups = roofline(meas, btab, cfg.key)
    out = {"metric": METRIC,
           "value": round(value, 2), "unit": "eigenpairs/s", "n_gpus": world, "steps": K, "warmup": W,
           "ms_per_step": round(meas["t_s"] * 1e3 / K, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE, "data": "synthetic",
           "config": {"workload": cfg.workload, "n": cfg.n, "b": cfg.b, "slices": cfg.nslices,
                      "slices_per_step": cfg.group, "ne": cfg.ne, "nev": cfg.nev, "tol": TOL, "ellipse_ratio": RHO,
                      "m0_range": [int(seq.m0.min()), int(seq.m0.max())], "factor_cap_gb": cfg.cap >> 30,
                      "l2": "inputs larger than L2 (factors of one step exceed 1 GB)",
                      "bnorm": "||B_k||_2 by bisection on inertia before timing (%.0f ms per matrix)" % seq.bnorm_ms,
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "iterations_per_step": meas["iters"], "call_ms_per_step": meas["step_ms"],
           "warm_start_per_step": meas["warm"], "status_per_step": meas["statuses"],
           "eigensolver_rr_sweeps32_refine_fallback": meas["eig"], "autotuned": meas["tuned"],
           "kernel_groups": groups, "roofline": roof, "peaks": peaks, "clocks": meas["clocks"],
           "gpu_launches": meas["launches"]}
    if seq.proposal:
        out["slice_proposal_first_matrix"] = seq.proposal
    if rank == 0 and not args.no_plain:
        if cfg.key == "c2":
            n2 = max(1, min(len(inputs), args.plain_steps))
            out["plain_fp64"] = replay(pk, torch, seq, inputs[:n2], stream, pk.FP64, "c128+f64")
        else:
            out["plain_fp64"] = plain_sample(pk, torch, seq, inputs[0], stream, args.plain_slices)
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e_leg(pk, torch, seq, inputs[: max(1, min(K, args.e2e_steps))], stream)
    bounds0 = seq.bounds0
    seq.ws.clear()
    del seq, inputs, meas
    torch.cuda.empty_cache()
    if rank == 0 and args.workload != "c2" and not args.no_second:
        out["c2"] = second_config(pk, torch, dev, args, btab, stream)
    if rank == 0 and prop_report:
        out["slice_proposal"] = prop_report
    if rank == 0 and pool is not None:
        ks = cfg.targets()
        out["cpu_baseline"] = cpu_baseline(pool, cfg, bounds0, [m0_rule(ks[1] - ks[0])], args)
        pool.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


def second_config(pk, torch, dev, args, btab, stream):
    """The n = 8192 sequence (one matrix per step) with plain FP64, float-float and FP64 Rayleigh-Ritz
    products, CUDA-graph replay and the unrefined FP32-class path beside it."""
    cfg = C2
    W, K = max(3, min(args.warmup, 5)), max(2, min(args.steps, 20))
    seq = Sequence(pk, torch, dev, cfg, W + K)
    meas, inputs = run_sequence(pk, torch, seq, W, K, stream)
    roof, groups = roofline(meas, btab, cfg.key)
    out = {"workload": cfg.workload, "value": round(meas["pairs"] / meas["t_s"], 2), "unit": "eigenpairs/s",
           "steps": K, "warmup": W, "ms_per_step": round(meas["t_s"] * 1e3 / K, 3), "dtype": DTYPE,
           "iterations_per_step": meas["iters"], "kernel_groups": groups, "roofline": roof,
           "gpu_launches": meas["launches"]}
    n2 = max(1, min(len(inputs), args.plain_steps))
    out["plain_fp64"] = replay(pk, torch, seq, inputs[:n2], stream, pk.FP64, "c128+f64")
    out["mixed_rr_floatfloat"] = replay(pk, torch, seq, inputs[:n2], stream, pk.MIXED, "c64+ff32x2+f64",
                                       rr_arith=pk.RR_FLOATFLOAT)
    out["mixed_rr_fp64"] = replay(pk, torch, seq, inputs[:n2], stream, pk.MIXED, "c64+f64", rr_arith=pk.RR_FP64)
    out["graphs"] = graph_leg(pk, torch, seq, inputs[:n2])
    out["fp32_class_error"] = fp32_class_error(pk, torch, seq, inputs[0], meas["last"] if K == 1 else None)
    if not args.no_e2e:
        out["e2e"] = e2e_leg(pk, torch, seq, inputs[: max(1, min(K, args.e2e_steps))], stream)
    return out


def replay(pk, torch, seq, inputs, stream, precision, dtype, **extra):
    """The same steps timed with another arithmetic."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    seq.call(*inputs[0], precision, **extra)     # untimed: tunes this arithmetic's choices
    torch.cuda.synchronize()
    e0.record(stream)
    pairs, iters = 0, []
    for k, g, x0, bounds in inputs:
        r = seq.call(k, g, x0, bounds, precision, **extra)
        pairs += good_pairs(r)
        iters.append(r.stats["iterations"])
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    return {"value": round(pairs / t, 2), "unit": "eigenpairs/s", "steps": len(inputs),
            "ms_per_step": round(t * 1e3 / len(inputs), 3), "iterations_per_step": iters, "dtype": dtype}


def plain_sample(pk, torch, seq, inp, stream, nsl):
    """Plain FP64 against mixed on the same sample of the workload: the first `nsl` slices of the
    first timed step (a full step in FP64 would take minutes)."""
    k, g, x0, bounds = inp
    cols = int(seq.col[g * seq.cfg.group + nsl] - seq.col[g * seq.cfg.group])
    xs = None if x0 is None else x0[:cols].contiguous()
    out = {"sample": "slices %d-%d of matrix %d (first timed step), same start vectors" %
           (g * seq.cfg.group, g * seq.cfg.group + nsl - 1, k)}
    for name, prec, dt in (("mixed", pk.MIXED, DTYPE), ("fp64", pk.FP64, "c128+f64")):
        seq.call(k, g, xs, bounds, prec, nsl=nsl, max_iter=1)            # untimed: tuning, workspace
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = seq.call(k, g, xs, bounds, prec, nsl=nsl)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out[name] = {"value": round(good_pairs(r) / t, 2), "unit": "eigenpairs/s", "seconds": round(t, 3),
                     "iterations": r.stats["iterations"], "dtype": dt, "status": r.status}
    out["value"] = out["fp64"]["value"]
    out["unit"] = "eigenpairs/s"
    out["mixed_over_fp64"] = round(out["mixed"]["value"] / max(out["fp64"]["value"], 1e-9), 2)
    return out


def graph_leg(pk, torch, seq, inputs):
    """The same steps on a side stream with and without CUDA-graph replay of the filter passes."""
    s = torch.cuda.Stream()
    res = {}
    with torch.cuda.stream(s):
        for graphs in (0, 1):
            seq.call(*inputs[0], pk.MIXED, graphs=graphs, stream=s)
            s.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            pairs, gl = 0, 0
            for k, g, x0, bounds in inputs:
                r = seq.call(k, g, x0, bounds, pk.MIXED, graphs=graphs, stream=s)
                pairs += good_pairs(r)
                gl += r.stats["graph_launches"]
            e1.record(s)
            s.synchronize()
            t = e0.elapsed_time(e1) / 1e3
            res["graphs_on" if graphs else "graphs_off"] = {"value": round(pairs / t, 2),
                                                            "ms_per_step": round(t * 1e3 / len(inputs), 3),
                                                            "graph_launches": gl}
    return res


def fp32_class_error(pk, torch, seq, inp, _ref=None):
    """The unrefined complex64 filter (PDESHEP_REFINE_NONE, the FP32-class path) against the refined
    result of the same step, after the FP32-class path has run until its residuals stall (tolerance
    1e-6).  Every eigenpair the FP32-class path finds is matched against all refined eigenpairs of the
    step (a pair at a slice boundary may be found by the neighbouring slice): per slice the largest
    distance to the nearest refined eigenvalue relative to ||B||_2, and the sine of the largest
    principal angle between its eigenvectors and the span of all refined eigenvectors."""
    k, g, x0, bounds = inp
    ref = seq.call(k, g, x0, bounds, pk.MIXED)
    r32 = seq.call(k, g, x0, bounds, pk.MIXED, refine_policy=0, tol=1e-6, max_iter=12)
    bn = seq.bnorm[k]
    ref_l, ref_v = [], []
    for i in range(len(ref.nfound)):
        off, m = ref.offset(i), int(ref.nfound[i])
        ref_l.append(ref.evals[off:off + m].cpu().numpy())
        ref_v.append(ref.evecs[off:off + m].cpu().numpy())
    La = np.concatenate(ref_l)
    Xa = np.concatenate(ref_v).T
    Qa, _ = np.linalg.qr(Xa)
    dl, sa, counts = [], [], []
    for i in range(len(r32.nfound)):
        off, m = r32.offset(i), int(r32.nfound[i])
        counts.append([int(ref.nfound[i]), m])
        if m == 0:
            continue
        b = r32.evals[off:off + m].cpu().numpy()
        dl.append(float(np.max(np.min(np.abs(b[:, None] - La[None, :]), axis=1)) / bn))
        Xb = r32.evecs[off:off + m].cpu().numpy().T
        P = Xb - Qa @ (Qa.conj().T @ Xb)
        sa.append(float(np.linalg.norm(P, 2)))
    return {"max_abs_dlambda_over_bnorm": max(dl) if dl else None, "per_slice_dlambda": [float("%.3g" % v) for v in dl],
            "max_sin_angle": max(sa) if sa else None, "per_slice_sin_angle": [float("%.3g" % v) for v in sa],
            "found_refined_vs_fp32": counts,
            "fp32_path_max_residual": r32.stats["max_residual"], "fp32_path_iterations": r32.stats["iterations"]}


def e2e_leg(pk, torch, seq, inputs, stream):
    """Same metric through the C ABI with host buffers: pinned host band and start vectors copied in,
    eigenvalues and eigenvectors copied out, every step inside the timed region.  The copies run on
    a second stream (double-buffered device inputs and host outputs), so step i's results come back
    and step i+1's inputs go in while the GPU computes; the region ends when the last results are on
    the host.  (Falls back to copies on the compute stream if the overlapped run fails.)"""
    try:
        return _e2e_run(pk, torch, seq, inputs, stream, overlap=True)
    except Exception as e:  # noqa: BLE001 - report the sequential measurement instead
        out = _e2e_run(pk, torch, seq, inputs, stream, overlap=False)
        out["overlap_error"] = str(e)[:200]
        return out


def _e2e_run(pk, torch, seq, inputs, stream, overlap):
    cfg = seq.cfg
    gcols = [int(seq.col[(g + 1) * cfg.group] - seq.col[g * cfg.group]) for g in range(cfg.groups)]
    cols = max(gcols)
    nb = 2 if overlap else 1
    hb = {k: torch.from_numpy(seq.host[k]).pin_memory() for k, _, _, _ in inputs}
    hx = [x0.cpu().pin_memory() if x0 is not None else None for _, _, x0, _ in inputs]
    dband = [torch.empty_like(seq.bands[0]) for _ in range(nb)]
    dx = [torch.empty((cols, cfg.n), dtype=torch.complex128, device=seq.dev) for _ in range(nb)]
    ev_h = [torch.empty(cols, dtype=torch.float64).pin_memory() for _ in range(nb)]
    vec_h = [torch.empty((cols, cfg.n), dtype=torch.complex128).pin_memory() for _ in range(nb)]
    cs = torch.cuda.Stream() if overlap else stream
    c0 = gcols[inputs[0][1]]
    h2d = hb[inputs[0][0]].numel() * 16 + (c0 * cfg.n * 16 if hx[0] is not None else 0)
    d2h = c0 * 8 + c0 * cfg.n * 16
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def upload(i):  # step i's inputs into buffer i % nb, on the copy stream
        k, g, _, _ = inputs[i]
        j = i % nb
        with torch.cuda.stream(cs):
            dband[j].copy_(hb[k], non_blocking=True)
            if hx[i] is not None:
                dx[j][:gcols[g]].copy_(hx[i], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
        return ev

    torch.cuda.synchronize()
    e0.record(stream)
    pairs = 0
    keep = []
    up = upload(0)
    done_out = [None] * nb  # event: buffer j's previous results are on the host
    for i, (k, g, x0i, bounds) in enumerate(inputs):
        j = i % nb
        cg = gcols[g]
        stream.wait_event(up)
        if i + 1 < len(inputs) and overlap:
            if done_out[(i + 1) % nb] is not None:
                cs.wait_event(done_out[(i + 1) % nb])  # (inputs of i+1 reuse buffer (i+1) % nb)
            up_next = upload(i + 1)
        x0 = dx[j][:cg] if hx[i] is not None else None
        r = seq.call(k, g, x0, bounds, pk.MIXED, band=dband[j])
        pairs += good_pairs(r)
        fin = torch.cuda.Event()
        fin.record(stream)
        cs.wait_event(fin)
        with torch.cuda.stream(cs):
            ev_h[j][:cg].copy_(r.evals, non_blocking=True)
            vec_h[j][:cg].copy_(r.evecs, non_blocking=True)
            d = torch.cuda.Event()
            d.record(cs)
        done_out[j] = d
        keep.append(r)  # the device results stay alive until their copies have run
        if i + 1 < len(inputs):
            up = up_next if overlap else upload(i + 1)
    stream.wait_stream(cs)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    return {"value": round(pairs / t, 2), "unit": "eigenpairs/s", "steps": len(inputs),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "copies": "overlapped on a second stream" if overlap else "on the compute stream"}


def train_proposer(pk, torch, dev, args):
    """The learned slice proposer: trained here on 128 smaller spectra of the mixture family (n =
    1024; half at b = 64, half at b = 128; labels by the library's inertia bisection to 1e-4
    relative; 1500 Adam steps), then evaluated on held-out complex mixture bands (n = 16384, b = 64,
    64 equal-count slices) against equal widths (the no-network baseline); counts are exact in both."""
    from paper_2012_00506_gb300 import slicer

    def family(seed, n, b):
        g = np.random.default_rng(seed)
        k = int(g.integers(1, 7))
        return synth.mixture_band(n, b, seed, is_complex=True, ncomp=k, comp_sigma=float(g.uniform(0.01, 0.2)),
                                  off_sigma=float(g.uniform(0.005, 0.03)), means=g.uniform(-1.0, 1.0, size=k),
                                  weights=g.dirichlet(np.ones(k)))

    t0 = time.perf_counter()
    train = [torch.from_numpy(family(synth.config_seed(4) + s, 1024, 64 if s % 2 else 128)).to(dev)
             for s in range(128)]
    params, losses, _ = slicer.train(train, steps=1500, batch=64, lr=1e-3, seed=0, log_every=1499, label_rtol=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if args.no_proposal:
        return params, None
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
                              float(np.mean(np.abs(pr.proposed_counts - tgt)[1:-1]))))
    out = {"config": "complex mixture bands n=16384 b=64, 64 slices, count tolerance 16; network trained on "
                     "128 bands n=1024 (b=64 and b=128)", "train_seconds": round(t_train, 2),
           "train_loss": [round(l, 6) for _, l in losses]}
    for name in ("mlp", "none"):
        r = np.array(res[name])
        out[name] = {"ms": round(1e3 * float(np.mean(r[:, 0])), 2), "inertia_evals": float(np.mean(r[:, 1])),
                     "boundaries_fixed": float(np.mean(r[:, 2])), "proposal_count_error": round(float(np.mean(r[:, 3])), 1)}
    return params, out


def traffic_for(group, key):
    """DRAM bytes per launch of the group's main kernel from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        data = json.load(open(path))
    except (OSError, ValueError):
        return None
    ent = data.get(key, {}).get(group) if isinstance(data.get(key), dict) else None
    if not ent or ent.get("source_hash") != source_hash(group):
        return None
    return ent.get("dram_bytes_per_launch")


GROUP_SOURCES = {"solve": ("band_lu.cu", "solve_tc.cu", "solve_tm.cu"), "factor": "band_lu.cu", "gemm": "tcgemm.cu", "small": "dense.cu",
                 "bandmm": "tcgemm.cu", "accum": "feast.cu", "inertia": "inertia.cu", "eig": "dense.cu"}


def source_hash(group):
    import hashlib
    files = GROUP_SOURCES.get(group, "feast.cu")
    files = (files,) if isinstance(files, str) else files
    h = hashlib.sha1()
    try:
        for f in files:
            h.update(open(os.path.join(ROOT, "paper_2012_00506_gb300", "csrc", f), "rb").read())
    except OSError:
        return None
    return h.hexdigest()[:12]


# ----------------------------------------------------------------------------- CPU oracle leg
def oracle_cores():
    return max(1, min(16, os.cpu_count() or 1))


REF_COLS = 16


def _oracle_unit(job):
    """One (slice, node) unit of the oracle's filter in a worker process: band LU of z_j I - B and
    the normal and adjoint solves of `cols` start vectors; returns (t_lu, t_solve)."""
    cfg_key, bounds, j, ne, cols, seed = job
    sys.path.insert(0, ROOT)
    import oracle
    cfg = CONFIGS[cfg_key]
    ab = make_matrix(cfg, 0)
    z, _ = oracle.contour_rule(ne, bounds[0], bounds[1], RHO)
    Y = synth.random_subspace(cfg.n, cols, seed, True)
    t0 = time.perf_counter()
    F, ipiv, info = oracle.band_lu(ab, z[j])
    t1 = time.perf_counter()
    oracle.band_solve(F, ipiv, cfg.b, Y, 0)
    oracle.band_solve(F, ipiv, cfg.b, Y, 1)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def oracle_filter_sample(pool, cfg, bounds, m0, units):
    """The oracle's filter of one FEAST iteration of slice 0 spread over the pool's processes (one
    quadrature node per process, the paper's level-L2 parallelism), the solves timed on REF_COLS of
    the m0 start vectors and scaled to m0; eigenpairs/s = the slice's count / the iteration's filter
    time on the pool.  Rayleigh-Ritz and later iterations are left out, so it bounds the oracle's
    throughput from above."""
    cnt = cfg.targets()[1] - cfg.targets()[0]
    jobs = [(cfg.key, (bounds[0], bounds[1]), j % cfg.ne, cfg.ne, REF_COLS, 77 + j) for j in range(units)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_unit, jobs)
    wall = time.perf_counter() - t0
    t_unit = float(np.median([a + b * m0[0] / REF_COLS for a, b in res]))
    cores = units
    t_iter = t_unit * math.ceil(cfg.ne / cores)
    return cnt / t_iter, wall, cores


def oracle_sample_text(cfg):
    return ("filter of one FEAST iteration of slice 0 of the first matrix (%d quadrature nodes, one per host "
            "process: band LU of z_j I - B, n=%d b=%d, and normal and adjoint solves timed on %d of the m0 "
            "start vectors, scaled to m0); eigenpairs/s = slice count / filter time; Rayleigh-Ritz and "
            "later iterations excluded (an upper bound on the oracle)" % (cfg.ne, cfg.n, cfg.b, REF_COLS))


def cpu_baseline(pool, cfg, bounds, m0, args):
    v, wall, cores = oracle_filter_sample(pool, cfg, bounds, m0, cores_units(pool, cfg))
    return {"value": round(v, 4), "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
            "sample": oracle_sample_text(cfg), "seconds": round(wall, 2)}


def cores_units(pool, cfg):
    """(slice, node) units of the sample: one per process, at most the slice's Ne nodes."""
    return max(1, min(pool._processes, cfg.ne))


def ref_bounds(cfg):
    """Slice 0 of an equal-width partition of the oracle's Gershgorin interval into nev / count pieces:
    the reference arm only times the filter's factorizations and solves, whose cost does not depend
    on where the slice lies (the eigenpairs/s use slice 0's target count)."""
    import oracle
    ab = make_matrix(cfg, 0)
    lo, hi = oracle.gershgorin(ab)
    ks = cfg.targets()
    w = (hi - lo) * (ks[1] - ks[0]) / cfg.n
    return [lo, lo + w]


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    cfg = CONFIGS[args.workload]
    pool = mp.get_context("spawn").Pool(oracle_cores())
    bounds = ref_bounds(cfg)
    ks = cfg.targets()
    m0 = [m0_rule(ks[1] - ks[0])]
    units = cores_units(pool, cfg)
    for _ in range(args.warmup):
        pool.map(_oracle_warm, range(pool._processes))
    vals, walls = [], []
    for _ in range(args.steps):
        v, wall, cores = oracle_filter_sample(pool, cfg, bounds, m0, units)
        vals.append(v)
        walls.append(wall)
    pool.close()
    value = float(len(vals) / np.sum([1.0 / v for v in vals]))      # pairs per total extrapolated time
    out = {"impl": "reference", "metric": METRIC,
           "value": round(value, 4), "unit": "eigenpairs/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(walls)), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg.workload, "n": cfg.n, "b": cfg.b, "slices": cfg.nslices, "ne": cfg.ne},
           "cpu_baseline": {"kind": "oracle", "cores": units, "sample": oracle_sample_text(cfg),
                            "value": round(value, 4)},
           "e2e": {"value": round(value, 4), "unit": "eigenpairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def _oracle_warm(_):
    sys.path.insert(0, ROOT)
    import oracle
    oracle.build()
    ab = synth.random_band(256, 4, 1, True)
    F, ipiv, _ = oracle.band_lu(ab, 0.1 + 0.05j)
    oracle.band_solve(F, ipiv, 4, synth.random_subspace(256, 8, 1, True), 0)
    return 0


def profile_case(args):
    """A reduced instance of a workload for ncu captures: the first matrix, the first
    `--profile-slices` slices of its partition (same n, b, m0, Ne), library-drawn start vectors, two
    band_slice calls (the second with resident tuning choices)."""
    import torch
    import paper_2012_00506_gb300 as pk
    from paper_2012_00506_gb300 import build as cb

    cb.build()
    dev = torch.device("cuda:0")
    cfg = CONFIGS[args.workload]
    ab = make_matrix(cfg, 0)
    band = torch.from_numpy(ab).to(dev)
    ks = cfg.targets()[: args.profile_slices + 1]
    idx = sorted(set([k for k in ks[1:]] + [k - 1 for k in ks[1:]] + [0]))
    lo, hi = pk.bisect(band, idx, rtol=1e-12, fanout=8)
    lam = {k: 0.5 * (lo[i] + hi[i]) for i, k in enumerate(idx)}
    spacing = (lam[ks[1]] - lam[0]) / ks[1]
    bounds = [lam[0] - 2 * spacing] + [0.5 * (lam[k - 1] + lam[k]) for k in ks[1:]]
    m0 = [m0_rule(ks[i + 1] - ks[i]) for i in range(args.profile_slices)]
    lo2, hi2 = pk.bisect(band, [0, cfg.n - 1], rtol=1e-8, fanout=16)
    bn = max(abs(lo2[0]), abs(hi2[0]), abs(lo2[1]), abs(hi2[1]))
    for rep in range(2):
        r = pk.band_slice(band, bounds, m0, None, bnorm=bn, precision=pk.MIXED, ne=cfg.ne, tol=TOL,
                          ellipse_ratio=RHO, max_iter=40, autotune=1, raise_on_error=False, seed=cfg.seed)
        torch.cuda.synchronize()
    print(json.dumps({"profile_case": cfg.key, "slices": args.profile_slices, "m0": m0, "status": r.status,
                      "nfound": [int(v) for v in r.nfound], "counts": [int(v) for v in r.counts],
                      "iterations": r.stats["iterations"]}))
    if r.status != 0 or list(r.nfound) != list(r.counts):
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(CONFIGS), default="c5")
    ap.add_argument("--plain-steps", type=int, default=2)
    ap.add_argument("--plain-slices", type=int, default=2, help="slices in the plain FP64 sample of the headline")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-second", action="store_true", help="skip the n=8192 configuration beside the headline")
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
