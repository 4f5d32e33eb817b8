"""FP64 CPU oracle for prox_{lambda R} (arXiv 2311.03096).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never
imports this package and shares no code with it.

The C core (``ws_oracle.c``) is the plain definition written out: stable sort,
the shift of Alg. 2, pool-adjacent-violators with pooling on ``>=``
(Sec. 4.1), scatter back.  This module adds numpy marshalling plus the
independent checks that pin it (``oracle.pins``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ws_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libws_oracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile ws_oracle.c into a shared library next to it (plain gcc, -O2)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.ws_oracle_prox.argtypes = [_f64p, ctypes.c_int64, ctypes.c_double, _f64p, _i32p, _i64p,
                                           _f64p, _i64p]
            lib.ws_oracle_prox.restype = ctypes.c_int
            lib.ws_oracle_prox_l1.argtypes = [_f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, _f64p, _i32p, _i64p]
            lib.ws_oracle_prox_l1.restype = ctypes.c_int
            lib.ws_oracle_prox_batched.argtypes = [_f64p, _i64p, ctypes.c_int64, _f64p, _f64p, _i32p, _i64p]
            lib.ws_oracle_prox_batched.restype = ctypes.c_int
            lib.ws_oracle_backward.argtypes = [_f64p, _i32p, _i64p, ctypes.c_int64, ctypes.c_int64, _f64p]
            lib.ws_oracle_backward.restype = ctypes.c_int
            lib.ws_oracle_R_pairs.argtypes = [_f64p, ctypes.c_int64]
            lib.ws_oracle_R_pairs.restype = ctypes.c_double
            lib.ws_oracle_R_sorted.argtypes = [_f64p, ctypes.c_int64]
            lib.ws_oracle_R_sorted.restype = ctypes.c_double
            lib.ws_oracle_neighbour_slack.argtypes = [_f64p, ctypes.c_int64, ctypes.c_double, ctypes.c_int64]
            lib.ws_oracle_neighbour_slack.restype = ctypes.c_double
            lib.ws_oracle_sort.argtypes = [_f64p, ctypes.c_int64, _i64p, _f64p]
            lib.ws_oracle_sort.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


class OracleError(RuntimeError):
    pass


_ERRORS = {1: "invalid argument", 2: "non-finite input", 4: "out of memory"}


def _check(rc):
    if rc != 0:
        raise OracleError(_ERRORS.get(rc, f"error {rc}"))


def prox(w, lam: float, *, return_perm: bool = False):
    """prox_{lam R}(w) in FP64.  Returns (out, ids, n_clusters[, perm, x_sorted]).

    ``w`` may be float32 or float64; float32 values are widened exactly.
    """
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    d = w.shape[0]
    out = np.empty(d, np.float64)
    ids = np.empty(d, np.int32)
    nc = ctypes.c_int64(0)
    perm = np.empty(d, np.int64) if return_perm else None
    xs = np.empty(d, np.float64) if return_perm else None
    _check(_load().ws_oracle_prox(_p(w, _f64p), d, float(lam), _p(out, _f64p), _p(ids, _i32p),
                                  _p(perm, _i64p), _p(xs, _f64p), ctypes.byref(nc)))
    if return_perm:
        return out, ids, int(nc.value), perm, xs
    return out, ids, int(nc.value)


def prox_l1(w, alpha: float, beta: float, rho: float = 0.0, v_scale: float = 1.0):
    """Weight sharing + l1 with rewinding (Alg. 2) in FP64.  Returns (out, ids, n_clusters)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    d = w.shape[0]
    out = np.empty(d, np.float64)
    ids = np.empty(d, np.int32)
    nc = np.zeros(1, np.int64)
    _check(_load().ws_oracle_prox_l1(_p(w, _f64p), d, float(alpha), float(beta), float(rho), float(v_scale),
                                     _p(out, _f64p), _p(ids, _i32p), _p(nc, _i64p)))
    return out, ids, int(nc[0])


def prox_batched(values, offsets, lambdas):
    """Per-segment prox.  Returns (out, ids, n_clusters_per_segment)."""
    w = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64))
    n_seg = off.shape[0] - 1
    out = np.empty_like(w)
    ids = np.empty(w.shape[0], np.int32)
    nc = np.empty(max(n_seg, 1), np.int64)
    _check(_load().ws_oracle_prox_batched(_p(w, _f64p), _p(off, _i64p), n_seg, _p(lam, _f64p),
                                          _p(out, _f64p), _p(ids, _i32p), _p(nc, _i64p)))
    return out, ids, nc[:n_seg]


def backward(grad_out, ids, offsets=None):
    """grad_in[i] = mean of grad_out over the cluster (segment, id) of i."""
    g = np.ascontiguousarray(np.asarray(grad_out, dtype=np.float64))
    idv = np.ascontiguousarray(np.asarray(ids, dtype=np.int32))
    off = None if offsets is None else np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n_seg = 1 if off is None else off.shape[0] - 1
    gin = np.empty_like(g)
    _check(_load().ws_oracle_backward(_p(g, _f64p), _p(idv, _i32p), _p(off, _i64p), n_seg, g.shape[0],
                                      _p(gin, _f64p)))
    return gin


def dlambda(grad_out, ids, offsets=None):
    """Gradient of <grad_out, prox_{lam_s R}(w)> with respect to each segment's lam_s,
    the partition held fixed: a cluster on sorted positions k = a..b (1-based) moves
    with its mean velocity, d out / d lam = mean of (d + 1 - 2k)/(d - 1) over the
    cluster = (d + 1 - a - b)/(d - 1) (Sec. 3 particle model; 0 when d <= 1).
    Cluster r of a segment occupies the positions after clusters 0..r-1, so a and b
    follow from the cluster sizes.  Returns one float64 per segment."""
    g = np.asarray(grad_out, dtype=np.float64)
    idv = np.asarray(ids, dtype=np.int64)
    off = np.array([0, g.shape[0]], np.int64) if offsets is None else np.asarray(offsets, dtype=np.int64)
    res = np.zeros(off.shape[0] - 1)
    for s in range(off.shape[0] - 1):
        a0, b0 = off[s], off[s + 1]
        d = int(b0 - a0)
        if d <= 1:
            continue
        r = idv[a0:b0]
        size = np.bincount(r)
        start = np.concatenate([[0], np.cumsum(size)[:-1]])       # 0-based first position
        first, last = start + 1, start + size                      # 1-based a, b
        dl = (d + 1 - first - last) / (d - 1)
        res[s] = float(np.sum(g[a0:b0] * dl[r]))
    return res


def imminent_collisions_v2(w, lam: float, max_rounds: int | None = None):
    """The paper's Imminent Collisions algorithm, version 2 (the appendix's
    Algorithm "Imminent collisions algorithm (v2)"; Sec. 4.1 for IC), in FP64
    numpy, kept here to count its rounds.

    Particles are the sorted weights x_k with velocity v_k = lam (d + 1 - 2k)/(d - 1)
    and mass 1.  One round marks a new block wherever the destination y = x + v
    strictly increases from one particle to the next, so every maximal run of
    non-increasing y collides at once (a prefix sum numbers the blocks; positions
    and velocities are mass-weighted means).  Rounds repeat until one changes
    nothing; that last round is counted, as in the algorithm's repeat-until.

    Returns (out, ids, n_clusters, rounds, converged); out/ids are in input order
    (ids rank the blocks from the left).  With max_rounds the loop stops early and
    converged is False if the last round still merged."""
    perm, xs = sort(w)
    d = xs.shape[0]
    if d == 0:
        return np.empty(0), np.empty(0, np.int32), 0, 0, True
    k = np.arange(1, d + 1, dtype=np.float64)
    v = lam * (d + 1 - 2 * k) / (d - 1) if d > 1 else np.zeros(1)
    x = xs.copy()
    m = np.ones(d)
    starts = np.arange(d)          # first sorted position of every block
    rounds, converged = 0, False
    while max_rounds is None or rounds < max_rounds:
        n = x.shape[0]
        y = x + v
        c = np.zeros(n, np.int64)
        c[1:] = y[:-1] < y[1:]
        i = np.cumsum(c)
        rounds += 1
        if i[-1] + 1 == n:
            converged = True
            break
        mn = np.bincount(i, weights=m)
        x = np.bincount(i, weights=x * m) / mn
        v = np.bincount(i, weights=v * m) / mn
        m = mn
        starts = starts[np.concatenate([[True], c[1:] != 0])]
    sizes = np.diff(np.concatenate([starts, [d]]))
    ids_sorted = np.repeat(np.arange(starts.shape[0], dtype=np.int32), sizes)
    vals_sorted = np.repeat(x + v, sizes)
    ids = np.empty(d, np.int32)
    out = np.empty(d, np.float64)
    ids[perm] = ids_sorted
    out[perm] = vals_sorted
    return out, ids, int(starts.shape[0]), rounds, converged


def ws_measure(w) -> float:
    """Weight-sharing measure of the CIFAR10 experiment: #distinct nonzero weights /
    #nonzero weights (0 when every weight is zero); -0.0 counts as zero."""
    w = np.asarray(w, dtype=np.float64)
    nz = w[w != 0]
    return float(np.unique(nz).shape[0]) / float(nz.shape[0]) if nz.shape[0] else 0.0


def R_pairs(w) -> float:
    """R(w) from Eq. (1), O(d^2)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    return float(_load().ws_oracle_R_pairs(_p(w, _f64p), w.shape[0]))


def R_sorted(w) -> float:
    """R(w) from the sorted prefix-sum form of App. B, O(d log d)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    return float(_load().ws_oracle_R_sorted(_p(w, _f64p), w.shape[0]))


def neighbour_slack(x_sorted, lam: float, k0: int) -> float:
    """Cor. D.5 slack at the boundary between sorted positions k0 and k0+1 (0-based)."""
    xs = np.ascontiguousarray(np.asarray(x_sorted, dtype=np.float64))
    return float(_load().ws_oracle_neighbour_slack(_p(xs, _f64p), xs.shape[0], float(lam), int(k0)))


def sort(w):
    """Stable sort by IEEE total order.  Returns (perm, x_sorted)."""
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    d = w.shape[0]
    perm = np.empty(d, np.int64)
    xs = np.empty(d, np.float64)
    _check(_load().ws_oracle_sort(_p(w, _f64p), d, _p(perm, _i64p), _p(xs, _f64p)))
    return perm, xs
