"""Spectrum partitioning from earlier eigenvalues -- TEST INFRASTRUCTURE (oracle).

Only ``tests/`` may import this module; the library never does.  Plain Python
loops over the sorted eigenvalues, following the paper's steps in order:

* ``kmeans_slices``       the simplified one-dimensional k-means of Algorithm 3
                          (Section 3.1): start from equal counts, then move every
                          boundary to the gap that follows the midpoint of the two
                          neighbouring group centroids (centroid = mean of a group's
                          extreme points) until no boundary moves; groups that
                          become empty are merged away (K may shrink).
* ``equal_count_slices``  "Approach-1" of Section 3.1: the starting partition of
                          Algorithm 3 (equal counts, boundaries at gap midpoints).
* ``equal_width_slices``  "Approach-2" of Section 3.1: K equal pieces of [b0, bK].
* ``restart_plan``        start vectors after a re-slicing (Section 3.1: previous
                          vectors interlaced with random ones when a slice grows,
                          some removed when it shrinks).
* ``outer_bounds``        the bound search of Algorithm 4 (Section 3.2) and its
                          lower-bound counterpart described in the text: step away
                          from the previous extreme wanted eigenvalues by
                          max(|alpha d|, m_hat delta) until the inertia count of the
                          current band encloses every wanted eigenvalue.

Readings (the paper is ambiguous there):
* groups are defined by value, G_i = {d : b_{i-1} <= d < b_i}, so that a group and
  the slice [b_{i-1}, b_i) of the FEAST call count the same eigenvalues (ties never
  straddle a boundary);
* Algorithm 3 updates the boundaries one after another within a sweep (a boundary
  moved in the sweep changes the next group's centroid), and the (n mod K) groups
  of the starting partition with one extra point are the first ones;
* Algorithm 4's stopping test is printed as n_- <= nev but the text asks for "more
  than nev eigenvalues less than b_K": the search stops once n_-(b_K) >= i0 + nev
  (all wanted eigenvalues below b_K); the lower bound stops once n_-(b_0) <= i0;
  the step uses |alpha d| (the paper takes alpha = +-1e-3 to make it positive).
"""
from __future__ import annotations

import numpy as np


def _counts(d, bounds):
    """Number of points in each [b_{i-1}, b_i) (Section 3.2: counts per slice)."""
    out = []
    for i in range(1, len(bounds)):
        out.append(sum(1 for x in d if bounds[i - 1] <= x < bounds[i]))
    return out


def _dedup(bounds):
    """Remove repeated boundaries (empty groups), keeping the order (Algorithm 3, last step)."""
    out = [bounds[0]]
    for b in bounds[1:]:
        if b != out[-1]:
            out.append(b)
    return out


def equal_count_slices(d, K, b0, bK):
    """Approach-1 / steps 1-2 of Algorithm 3: K groups of floor(n/K) or floor(n/K)+1 points
    (the first n mod K groups one more), boundary b_i between G_i and G_{i+1} at the midpoint of
    G_i's largest and G_{i+1}'s smallest point; b0 and bK enclose the points."""
    d = [float(x) for x in d]
    n = len(d)
    q, r = divmod(n, K)
    bounds = [float(b0)]
    end = 0
    for i in range(1, K):
        end += q + (1 if i <= r else 0)
        if end <= 0:
            bounds.append(float(b0))
        elif end >= n:
            bounds.append(float(bK))
        else:
            bounds.append(0.5 * (d[end - 1] + d[end]))
    bounds.append(float(bK))
    bounds = _dedup(bounds)
    return bounds, _counts(d, bounds)


def equal_width_slices(d, K, b0, bK):
    """Approach-2 of Section 3.1: [b0, bK] cut into K pieces of equal width."""
    bounds = [b0 + (bK - b0) * i / K for i in range(K)] + [float(bK)]
    bounds = _dedup([float(b) for b in bounds])
    return bounds, _counts([float(x) for x in d], bounds)


def kmeans_slices(d, K, b0, bK, max_sweeps=1000):
    """Algorithm 3: returns (bounds, counts, sweeps).  ``sweeps`` counts the passes over the
    boundaries, the last of which moved none (or max_sweeps if that cap stopped it)."""
    d = [float(x) for x in d]
    n = len(d)
    bounds, _ = equal_count_slices(d, K, b0, bK)
    sweeps = 0
    while sweeps < max_sweeps:
        sweeps += 1
        old = list(bounds)
        for i in range(1, len(bounds) - 1):
            lo, mid, hi = bounds[i - 1], bounds[i], bounds[i + 1]
            left = [x for x in d if lo <= x < mid]
            right = [x for x in d if mid <= x < hi]
            if not left or not right:
                continue
            c_left = 0.5 * (left[0] + left[-1])      # centroid: mean of the extreme points
            c_right = 0.5 * (right[0] + right[-1])
            t = 0.5 * (c_left + c_right)
            # first point beyond t; the point before it is the last of the left group
            ell = next(k for k in range(n) if d[k] > t)
            bounds[i] = 0.5 * (d[ell] + d[ell - 1])
        bounds = _dedup(bounds)
        if bounds == old:
            break
    return bounds, _counts(d, bounds), sweeps


def outer_bounds(ab, d_prev, i0, nev, alpha=1e-3, m_hat=6, max_it=64, inertia=None):
    """Algorithm 4 (upper bound) and the lower-bound search described beside it.

    d_prev: sorted eigenvalues of the previous matrix of the sequence, covering indices
    i0 .. i0+nev-1 (and one neighbour on each side when they exist).  Returns
    (b0, bK, it_lo, it_hi, ok): n_-(b0) <= i0 and n_-(bK) >= i0 + nev for the band ``ab``
    when ok; ok is False when a search stopped at max_it with its count still short of the
    target (the bounds then do not enclose the wanted eigenvalues)."""
    if inertia is None:
        from oracle import inertia as _inertia
        inertia = _inertia
    d = [float(x) for x in d_prev]
    du = d[i0 + nev - 1]
    delta = du - d[i0 + nev - 2] if nev >= 2 else 0.0
    step = max(abs(alpha * du), m_hat * delta)
    if not step > 0.0:
        step = 2.0 ** -40 * max(1.0, abs(du))
    bK = du + step
    it_hi = 1
    hi_ok = inertia(ab, bK) >= i0 + nev
    while not hi_ok and it_hi < max_it:
        bK = bK + step
        it_hi += 1
        hi_ok = inertia(ab, bK) >= i0 + nev
    dl = d[i0]
    delta2 = d[i0 + 1] - dl if i0 + 1 < len(d) else 0.0
    step2 = max(abs(alpha * dl), m_hat * delta2)
    if not step2 > 0.0:
        step2 = 2.0 ** -40 * max(1.0, abs(dl))
    b0 = dl - step2
    it_lo = 1
    lo_ok = inertia(ab, b0) <= i0
    while not lo_ok and it_lo < max_it:
        b0 = b0 - step2
        it_lo += 1
        lo_ok = inertia(ab, b0) <= i0
    return b0, bK, it_lo, it_hi, bool(hi_ok and lo_ok)


def kmeans_objective(d, bounds):
    """J of eq. (11) with the paper's centroids (mean of each group's extreme points)."""
    J = 0.0
    for i in range(1, len(bounds)):
        g = [x for x in d if bounds[i - 1] <= x < bounds[i]]
        if g:
            c = 0.5 * (g[0] + g[-1])
            J += sum((x - c) ** 2 for x in g)
    return J


def min_boundary_gap(d, bounds):
    """Smallest distance from an inner boundary to its nearest point (how deep a boundary cuts
    into a cluster; objective 1 of Section 3.1 wants it large)."""
    d = np.asarray(d, dtype=float)
    return float(min(np.min(np.abs(d - b)) for b in bounds[1:-1])) if len(bounds) > 2 else float("inf")


def restart_plan(prev_vals, bounds, m0_new, mode=0):
    """Start vectors for the next matrix of a sequence when the slices change (Section 3.1:
    when a slice's count grows, the previous vectors are interlaced with random ones; when it
    shrinks, some are removed).  ``prev_vals[c]`` is the Ritz value of previous column c.
    For new slice i (block of m0_new[i] columns): the previous columns whose values lie in
    [b_i, b_{i+1}) -- the m0_new[i] nearest to the slice centre if there are more -- in
    ascending value (ties by column); then, with mode 1, the nearest columns outside the slice
    (by distance to the interval; ties by value, then column); the rest -1 (a random vector).
    The columns offered should be the previous converged pairs (distinct eigenvectors).
    Returns one list per slice."""
    v = [float(x) for x in prev_vals]
    out = []
    for i in range(len(bounds) - 1):
        lo, hi = bounds[i], bounds[i + 1]
        c = 0.5 * (lo + hi)
        m = int(m0_new[i])
        inside = [k for k in range(len(v)) if lo <= v[k] < hi]
        if len(inside) > m:
            inside = sorted(inside, key=lambda k: (abs(v[k] - c), k))[:m]
        inside = sorted(inside, key=lambda k: (v[k], k))
        pick = list(inside)
        if mode == 1 and len(pick) < m:
            outside = [k for k in range(len(v)) if not (lo <= v[k] < hi)]
            dist = lambda k: (lo - v[k]) if v[k] < lo else (v[k] - hi)
            outside = sorted(outside, key=lambda k: (dist(k), v[k], k))
            pick += outside[: m - len(pick)]
        pick += [-1] * (m - len(pick))
        out.append(pick)
    return out
