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
