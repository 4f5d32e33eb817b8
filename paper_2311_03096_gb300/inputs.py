"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws numbers.  Both
the CUDA path's tests/benchmark and the oracle-based checks use it, so the two
sides always see bit-identical inputs.  Every generator takes an explicit seed
and uses numpy's PCG64, so values are reproducible on any machine.

Workloads (sizes as used by the tests and the benchmark):
  * ``normal``      w_i ~ N(0, 1), drawn in FP64 then rounded to the dtype.
  * ``duplicates``  10% of positions overwritten by exact copies of other
                    randomly chosen positions (exercises ties).
  * ``cascade``     the worst case of Sec. 4.1 realised in sorted-x space: the
                    left half is all zeros and the right half grows by h or 2h
                    per step (h = 2^-20) with lambda = (15/16) h (d - 1)/2, so the
                    left block absorbs the right half one particle per round.
  * ``mirror``      pairs of exact duplicates, 3h or 4h apart, with
                    lambda = 0.75 h (d - 1)/2: d/2 independent two-particle merges.
  * ``tie_lattice`` values on a lattice of one unit with lambda set so the
                    shift drops one unit per position: dense exact ties.
  * ``mlp``         Kaiming-uniform weights of an MLP 3072-4096-4096-10 split
                    into per-row segments, whole-layer segments and extra
                    segments with log-uniform lengths (batched workload).
  * ``images``      CIFAR10-shaped batches (32x32x3, pixels U[0,1]) under one
                    fixed seeded pixel permutation, labels uniform over 10.
"""
from __future__ import annotations

import numpy as np

H_CASCADE = 2.0 ** -20


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def normal(d: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    """w_i ~ N(0,1) i.i.d., drawn in FP64 and rounded to ``dtype``."""
    return _rng(seed).standard_normal(d).astype(dtype)


def with_duplicates(w: np.ndarray, frac: float = 0.1, seed: int = 1) -> np.ndarray:
    """Overwrite ``frac`` of the positions with exact copies of other positions."""
    w = np.array(w, copy=True)
    d = w.shape[0]
    if d < 2:
        return w
    rng = _rng(seed)
    m = int(round(frac * d))
    dst = rng.choice(d, size=m, replace=False)
    src = rng.integers(0, d, size=m)
    w[dst] = w[src]
    return w


def normal_with_duplicates(d: int, seed: int = 0, dtype=np.float32) -> np.ndarray:
    return with_duplicates(normal(d, seed, dtype), 0.1, seed + 7919)


def cascade(d: int, seed: int = 0, shuffle: bool = False):
    """Adversarial cascade (worst case of Sec. 4.1).  Returns (w float32, lam).

    x_k = 0 for k <= d/2; for k > d/2, x_k = h * n_k with n_k = n_{k-1} + g_k,
    g_k = 1 + Bernoulli(0.1), n_{d/2} = 0.  All values are exact in FP32
    (n_k < 2^24 for d <= 2^24).  lam = (15/16) h (d - 1)/2.
    """
    rng = _rng(seed)
    half = d // 2
    g = 1 + (rng.random(d - half) < 0.1).astype(np.int64)
    n = np.cumsum(g)
    x = np.zeros(d, np.float64)
    x[half:] = H_CASCADE * n
    w = x.astype(np.float32)
    if shuffle:
        w = w[rng.permutation(d)]
    lam = (15.0 / 16.0) * H_CASCADE * (d - 1) / 2.0
    return w, lam


def mirror(d: int, seed: int = 0, shuffle: bool = False):
    """d/2 pairs of exact duplicates, pair gaps of 3h or 4h; lam = 0.75 h (d - 1)/2."""
    assert d % 2 == 0
    rng = _rng(seed)
    gaps = 3 + (rng.random(d // 2) < 0.5).astype(np.int64)
    levels = np.cumsum(gaps) - gaps[0]
    x = np.repeat(levels.astype(np.float64) * H_CASCADE, 2)
    w = x.astype(np.float32)
    if shuffle:
        w = w[rng.permutation(d)]
    lam = 0.75 * H_CASCADE * (d - 1) / 2.0
    return w, lam


def tie_lattice(d: int, seed: int = 0, dtype=np.float32, binade: bool = True, shuffle: bool = True):
    """Values on a lattice of one unit u = 2^-(p-1) (p = 24 for float, 53 for
    double): w = base + n u with n a random walk of steps 0 to 3 (base = 1,
    one binade, or base = 0, spanning binades), and lam = (d - 1) u / 2, so the
    shift drops by exactly one unit per sorted position.  Every sum the prox
    compares is then an integer multiple of u / 2, and steps of one unit are
    exact ties of adjacent block means.  Returns (w, lam, n) with n the integer
    lattice index of every w (same order)."""
    p = 24 if np.dtype(dtype) == np.float32 else 53
    rng = _rng(seed)
    n = np.cumsum(rng.integers(0, 4, d)).astype(np.int64)
    if shuffle:
        n = n[rng.permutation(d)]
    base = 1.0 if binade else 0.0
    w = (base + n.astype(np.float64) * 2.0 ** -(p - 1)).astype(dtype)
    lam = (d - 1) * 2.0 ** -p
    return w, lam, n


MLP_SIZES = (3072, 4096, 4096, 10)


def mlp_weights(seed: int = 0, sizes=MLP_SIZES):
    """Kaiming-uniform (a=0) weights: U(-sqrt(6/fan_in), +sqrt(6/fan_in)), float32."""
    rng = _rng(seed)
    mats = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        bound = np.sqrt(6.0 / fan_in)
        mats.append(rng.uniform(-bound, bound, size=(fan_out, fan_in)).astype(np.float32))
    return mats


def log_uniform_lengths(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = _rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).astype(np.int64)


def batched_segments(seed: int = 0, rows: bool = True, layers: bool = True, extra: int = 4096,
                     extra_lo: int = 16, extra_hi: int = 2 ** 20, sizes=MLP_SIZES):
    """The batched workload.  Returns (values float32, offsets int64, lambdas float64, kinds).

    Segments: every output-neuron row of each layer (rows), every whole layer
    (layers), then ``extra`` segments of N(0, 1) values with lengths
    log-uniform in [extra_lo, extra_hi].  lambda_s ~ LogUniform[1e-3, 1].
    ``kinds`` labels each segment ("row", "layer", "extra").
    """
    mats = mlp_weights(seed, sizes)
    parts, kinds = [], []
    if rows:
        for m in mats:
            for r in range(m.shape[0]):
                parts.append(m[r])
                kinds.append("row")
    if layers:
        for m in mats:
            parts.append(m.reshape(-1))
            kinds.append("layer")
    if extra:
        lens = log_uniform_lengths(extra, extra_lo, extra_hi, seed + 101)
        rng = _rng(seed + 202)
        for n in lens:
            parts.append(rng.standard_normal(int(n)).astype(np.float32))
            kinds.append("extra")
    lengths = np.array([p.shape[0] for p in parts], np.int64)
    offsets = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    values = np.concatenate(parts) if parts else np.zeros(0, np.float32)
    lam = np.exp(_rng(seed + 303).uniform(np.log(1e-3), np.log(1.0), size=len(parts)))
    return values, offsets, lam.astype(np.float64), kinds


def images(batch: int = 256, seed: int = 0, perm_seed: int = 12345):
    """CIFAR10-shaped synthetic batch: x (batch, 3072) float32 in U[0,1] under one
    fixed seeded pixel permutation, labels int64 uniform over 10 classes."""
    perm = _rng(perm_seed).permutation(3072)
    rng = _rng(seed)
    x = rng.random((batch, 3072)).astype(np.float32)[:, perm]
    y = rng.integers(0, 10, size=batch).astype(np.int64)
    return x, y
