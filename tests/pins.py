"""Independent checks that pin the oracle to the mathematics of the paper.

Nothing here calls the oracle or the CUDA library: these are separate,
deliberately naive restatements (brute force, textbook formulas, optimality
certificates) used by the tests to check both.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np


def R_pairs_py(u) -> float:
    """Eq. (1): R(u) = 1/(d-1) sum_{i>j} |u_i - u_j| (pure Python, O(d^2))."""
    d = len(u)
    if d < 2:
        return 0.0
    acc = 0.0
    for i in range(d):
        for j in range(i):
            acc += abs(u[i] - u[j])
    return acc / (d - 1)


def hyperplane(w, pi) -> float:
    """Eq. hyperplane: h_pi(w) = 1/(d-1) sum_i (2i - d - 1) w_{pi_i}, pi 1-based order."""
    d = len(w)
    return sum((2 * (i + 1) - d - 1) * w[pi[i]] for i in range(d)) / (d - 1)


def ordered_partitions(items):
    """All ordered set partitions (sequences of non-empty disjoint blocks)."""
    items = list(items)
    if not items:
        yield []
        return
    n = len(items)
    for r in range(1, n + 1):
        for first in itertools.combinations(items, r):
            rest = [x for x in items if x not in first]
            for tail in ordered_partitions(rest):
                yield [list(first)] + tail


def brute_force_prox(w, lam):
    """argmin_u 1/2||u - w||^2 + lam R(u) by enumeration of ordered partitions.

    On the face where u is constant on blocks B_1 < B_2 < ... (block i taking
    sorted positions s_i+1 .. s_i+|B_i|), R is linear (Eq. r_alt restricted to
    the active hyperplane), so the face minimiser is
        v_i = mean_{B_i}(w) + lam * mean_{k in positions(B_i)} (d + 1 - 2k)/(d - 1).
    The prox lies in the relative interior of its own face, so it is one of
    these candidates; every candidate is a feasible point, so the candidate
    with the smallest true objective (R evaluated by Eq. (1)) is the prox.
    Returns (u, objective).  Exponential: d <= 7 only.
    """
    w = [float(v) for v in w]
    d = len(w)
    if d == 1:
        return np.array(w), 0.0
    best_u, best_f = None, None
    for blocks in ordered_partitions(range(d)):
        u = [0.0] * d
        pos = 0
        for blk in blocks:
            n = len(blk)
            ks = range(pos + 1, pos + n + 1)
            shift = sum((d + 1 - 2 * k) / (d - 1) for k in ks) / n
            v = sum(w[i] for i in blk) / n + lam * shift
            for i in blk:
                u[i] = v
            pos += n
        f = 0.5 * sum((u[i] - w[i]) ** 2 for i in range(d)) + lam * R_pairs_py(u)
        if best_f is None or f < best_f:
            best_u, best_f = u, f
    return np.array(best_u), best_f


def isotonic_minmax(y):
    """Isotonic regression (Eq. iso_regr) by the min-max formula
    x_k = max_{i<=k} min_{j>=k} avg(y_{i..j})  (textbook; O(d^3), d <= ~300)."""
    y = np.asarray(y, dtype=np.float64)
    d = y.shape[0]
    P = np.concatenate([[0.0], np.cumsum(y)])
    out = np.empty(d)
    for k in range(d):
        i = np.arange(0, k + 1)[:, None]
        j = np.arange(k, d)[None, :]
        avg = (P[j + 1] - P[i]) / (j - i + 1)
        out[k] = avg.min(axis=1).max()
    return out


def shift_coefficients(d):
    """(d + 1 - 2k)/(d - 1), k = 1..d (Alg. 2's velocity divided by lambda)."""
    k = np.arange(1, d + 1, dtype=np.float64)
    return (d + 1 - 2 * k) / (d - 1)


def certificate_residual(w, u, lam) -> float:
    """How far (w - u)/lam is from the subdifferential dR(u) (Eq. subdiff_R).

    dR(u) = conv{grad h_pi : pi sorts u}.  For u whose level sets are the
    clusters (ordered by value, cluster C on sorted positions a..b), the
    convex hull is the product over clusters of permutahedra: g restricted to
    C must be majorised by the coefficients {(2k - d - 1)/(d - 1): k = a..b}
    (Rado): sorted descending, every prefix sum of g_C is <= the prefix sum of
    the coefficients, with equality for the full sum.  Returns the largest
    violation (0 means u = prox_{lam R}(w) by Eq. prox_opt); requires lam > 0.
    """
    w = np.asarray(w, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    d = w.shape[0]
    if d < 2:
        return float(np.abs(u - w).max()) if d else 0.0
    g = (w - u) / lam
    order = np.argsort(u, kind="stable")
    us = u[order]
    coef = -shift_coefficients(d)  # (2k - d - 1)/(d - 1) ascending in k
    worst = 0.0
    a = 0
    while a < d:
        b = a
        while b + 1 < d and us[b + 1] == us[a]:
            b += 1
        gc = np.sort(g[order[a:b + 1]])[::-1]
        cc = np.sort(coef[a:b + 1])[::-1]
        pg = np.cumsum(gc)
        pc = np.cumsum(cc)
        worst = max(worst, float((pg - pc).max()), abs(float(pg[-1] - pc[-1])))
        a = b + 1
    return worst


def collapse_threshold(x_sorted) -> float:
    """Smallest lambda for which prox collapses everything into one cluster.

    By Prop. 4.1 particle 1 collides with particle d iff d attains
    min_j avg(y_{1:j}) (ties pool), i.e. avg(x_{1:j}) + lam (d - j)/(d - 1) >=
    mean(x) for all j < d, since sum_{k<=j} (d + 1 - 2k)/(d - 1) = j (d - j)/(d - 1).
    Hence lam_max = max_{1<=j<d} (d - 1)(mean(x) - avg(x_{1:j}))/(d - j).
    """
    x = np.asarray(x_sorted, dtype=np.float64)
    d = x.shape[0]
    if d < 2:
        return 0.0
    j = np.arange(1, d)
    pre = np.cumsum(x)[:-1] / j
    return float(((d - 1) * (x.mean() - pre) / (d - j)).max())


def prop41_extremes(x_sorted, lam):
    """Prop. 4.1 and its mirror: min out = min_j avg(y_{1:j}), max out = max_j avg(y_{j:d})."""
    x = np.asarray(x_sorted, dtype=np.float64)
    d = x.shape[0]
    y = x + lam * shift_coefficients(d)
    pre = np.cumsum(y) / np.arange(1, d + 1)
    suf = np.cumsum(y[::-1]) / np.arange(1, d + 1)
    return float(pre.min()), float(suf.max())


def exact_prox_fraction(w, lam):
    """Exact rational PAV on y (Fractions) for tiny inputs: the values and the
    partition with no rounding at all (w and lam are converted exactly)."""
    d = len(w)
    if d == 0:
        return [], []
    if d == 1:
        return [Fraction(w[0])], [0]
    order = sorted(range(d), key=lambda i: (w[i], i))
    lamf = Fraction(lam)
    y = [Fraction(w[order[k]]) + lamf * Fraction(d + 1 - 2 * (k + 1), d - 1) for k in range(d)]
    blocks = []  # (sum, count)
    for v in y:
        blocks.append([v, 1])
        while len(blocks) >= 2 and blocks[-2][0] / blocks[-2][1] >= blocks[-1][0] / blocks[-1][1]:
            s, c = blocks.pop()
            blocks[-1][0] += s
            blocks[-1][1] += c
    out = [None] * d
    ids = [0] * d
    k = 0
    for r, (s, c) in enumerate(blocks):
        for _ in range(c):
            out[order[k]] = s / c
            ids[order[k]] = r
            k += 1
    return out, ids
