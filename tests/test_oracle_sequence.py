"""A short SCF-like sequence through the oracle's FEAST (Algorithm 1, CPU) with the paper's
re-slicing between steps (Section 3.1): every step partitions the previous step's converged
eigenvalues (equal counts or the simplified k-means of Algorithm 3), takes the exact counts by
inertia, sizes m0 by the rule of Section 3.2, and starts every slice from the previous
eigenvectors chosen by the restart plan (the nearest ones when the slice grew).  Gauss,
trapezoid and Zolotarev rules.  Every slice must converge with its exact count; the iteration counts (a
property of the algorithm, not of the hardware) are printed."""
import numpy as np
import pytest

import oracle
import synth
from oracle import partition_oracle as po
from oracle import rules_oracle as ro


def _sequence(method, rule_kind, n=800, b=8, nev=160, K=8, steps=4, ne=8, seed=5, outer="dense"):
    B = synth.random_band(n, b, seed, True, off_sigma=0.1)
    g = np.random.default_rng(seed + 1)
    totals, maxima = [], []
    vals = vecs = lam = None
    dense_ev = np.linalg.eigvalsh(synth.band_to_dense(B))
    for step in range(steps):
        ref = dense_ev[:nev] if step == 0 else lam
        if outer == "alg4" and step > 0:
            # Algorithm 4 on the current matrix from the previous eigenvalues (Section 3.2)
            b0, bK, _, _, ok = po.outer_bounds(B, lam, 0, nev)
            assert ok
        else:
            spacing = float(np.median(np.diff(ref)))
            b0 = float(ref[0] - 2 * spacing)
            bK = float(0.5 * (dense_ev[nev - 1] + dense_ev[nev]))   # previous matrix: excludes eigenvalue nev
        if method == "equal":
            bounds, _ = po.equal_count_slices(ref, K, b0, bK)
        else:
            bounds, _, _ = po.kmeans_slices(ref, K, b0, bK)
        counts = [oracle.inertia(B, bounds[i + 1]) - oracle.inertia(B, bounds[i]) for i in range(len(bounds) - 1)]
        m0 = [oracle.m0_rule(c) for c in counts]
        plan = [[-1] * m for m in m0] if vals is None else po.restart_plan(vals, bounds, m0, mode=1)
        bn = float(np.max(np.abs(dense_ev)))
        its, new_vals, new_vecs = [], [], []
        for i in range(len(bounds) - 1):
            Y = np.empty((n, m0[i]), dtype=np.complex128)
            for q, src in enumerate(plan[i]):
                Y[:, q] = vecs[:, src] if src >= 0 else g.standard_normal(n) + 1j * g.standard_normal(n)
            if rule_kind == "trapezoid":
                rule = ro.trapezoid_rule(ne, bounds[i], bounds[i + 1], 0.3)
            elif rule_kind == "zolotarev":
                rule = ro.zolotarev_rule(ne, bounds[i], bounds[i + 1], 0.2)[:2]
            else:
                rule = None
            o = oracle.feast_slice(B, bounds[i], bounds[i + 1], Y, ne=ne, rho=0.3, tol=1e-10, bnorm=bn,
                                   max_iter=40, count=counts[i], rule=rule)
            assert o["status"] == 0 and o["nfound"] == counts[i]
            its.append(o["iters"])
            k = o["nfound"]
            new_vals.append(o["evals"][:k])            # converged pairs only: distinct eigenvectors
            new_vecs.append(o["evecs"][:, :k])
        totals.append(int(sum(its)))
        maxima.append(int(max(its)))
        vals = np.concatenate(new_vals)
        vecs = np.concatenate(new_vecs, axis=1)
        lam = np.sort(vals)
        dense_ev = np.linalg.eigvalsh(synth.band_to_dense(B))
        B = B + 1e-3 * synth.perturbation(n, b, seed + 100 + step, True)
    return totals, maxima


@pytest.mark.slow
@pytest.mark.parametrize("method,rule,outer", [("equal", "gauss", "dense"), ("kmeans", "gauss", "dense"),
                                               ("kmeans", "trapezoid", "dense"), ("kmeans", "zolotarev", "dense"),
                                               ("equal", "zolotarev", "dense"), ("kmeans", "gauss", "alg4")])
def test_sequence_with_reslicing(method, rule, outer):
    """outer = "alg4": the outer bounds of every warm step come from Algorithm 4 on the current
    matrix instead of the previous matrix's dense spectrum (the loop of the paper's Algorithm 2)."""
    totals, maxima = _sequence(method, rule, outer=outer)
    print(f"\n{method:6s} {rule:9s} {outer:5s} slice iterations per step {totals}, slowest slice per step {maxima}")
    assert all(m <= 6 for m in maxima[1:])            # warm-started steps converge in a few iterations
