"""Comparison of the CUDA path with the oracle (used by the -m gpu tests).

Partition: the cluster ids must equal the oracle's element by element; a
boundary where the two partitions differ is excused only if the
neighbour-collision slack there (Cor. D.5, computed by the oracle in long
double) is within 1e-12 * (max|w| + lambda) of zero, i.e. the two adjacent
block means tie to that precision.  Values: |gpu - oracle| <= tol *
(max|w| + lambda), with tol = 1e-12 for FP64 and 1e-5 for FP32 storage.
"""
from __future__ import annotations

import numpy as np

import oracle

TIE_TOL = 1e-12


def boundaries(ids_sorted):
    return set(np.nonzero(ids_sorted[1:] != ids_sorted[:-1])[0].tolist())


def compare_segment(w, lam, out_gpu, ids_gpu, nc_gpu, tol, ref=None):
    """Returns a dict of diagnostics; raises AssertionError on a parity failure."""
    w = np.asarray(w)
    d = w.shape[0]
    if ref is None:
        ref = oracle.prox(w, lam, return_perm=True)
    out_ref, ids_ref, nc_ref, perm, xs = ref
    scale = (float(np.abs(w).max()) if d else 0.0) + lam
    diag = {"d": d, "lam": lam, "clusters": nc_ref}
    if d == 0:
        return diag
    ids_gpu = np.asarray(ids_gpu)
    excused = 0
    if not np.array_equal(ids_gpu, ids_ref):
        bg = boundaries(ids_gpu[perm])
        br = boundaries(ids_ref[perm])
        diff = sorted(bg ^ br)
        assert len(diff) <= 64, f"partition differs at {len(diff)} boundaries (first {diff[:8]})"
        for k in diff:
            s = oracle.neighbour_slack(xs, lam, k)
            assert abs(s) <= TIE_TOL * scale, f"partition differs at sorted boundary {k}: slack {s:.3e}"
        excused = len(diff)
        # ids must still be a valid ranked partition consistent with the value order
        g = ids_gpu[perm]
        assert g[0] == 0 and np.all(np.diff(g) >= 0) and np.all(np.diff(g) <= 1)
    else:
        assert int(nc_gpu) == nc_ref
    diag["excused"] = excused
    err = float(np.abs(np.asarray(out_gpu, dtype=np.float64) - out_ref).max())
    diag["max_abs_err"] = err
    diag["rel_err"] = err / scale if scale > 0 else err
    assert err <= tol * scale, f"max |gpu - oracle| = {err:.3e} > {tol:.0e} * {scale:.3e}"
    return diag


def integer_pav(Y):
    """PAV of integers y in sorted order, pooling while mean(below) >= mean(top)
    (Sec. 4.1: ties pool); means compared by exact cross-multiplication.
    Returns the block starts, sums and counts."""
    starts, sums, cnts = [], [], []
    for k, yk in enumerate(Y.tolist()):
        starts.append(k)
        sums.append(yk)
        cnts.append(1)
        while len(sums) >= 2 and sums[-2] * cnts[-1] >= sums[-1] * cnts[-2]:
            s, c = sums.pop(), cnts.pop()
            starts.pop()
            sums[-1] += s
            cnts[-1] += c
    return np.array(starts, np.int64), sums, cnts


def lattice_expected(n, d):
    """Exact prox partition of a tie lattice (inputs.tie_lattice) from its integer
    indices n: 2 (y_k - base) / u = 2 n_k + d + 1 - 2k.  Returns the cluster id
    of every element (input order), the cluster mean of those integers for every
    element (value = base + mean * u / 2) and the cluster count."""
    perm = np.argsort(n, kind="stable")
    Y = 2 * n[perm] + (d + 1) - 2 * np.arange(1, d + 1, dtype=np.int64)
    starts, sums, cnts = integer_pav(Y)
    ids = np.empty(d, np.int32)
    ids[perm] = np.repeat(np.arange(len(starts), dtype=np.int32), cnts)
    means = np.empty(d, np.float64)
    means[perm] = np.repeat(np.array([s / c for s, c in zip(sums, cnts)]), cnts)
    return ids, means, len(starts)
