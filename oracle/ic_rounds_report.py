"""Round counts of the paper's Imminent Collisions v2 (oracle.imminent_collisions_v2)
on the benchmark's inputs and on training-like weights.

Test infrastructure (runs the oracle on the CPU only).  It measures how many
IC v2 rounds -- each a full pass over the remaining blocks -- a round-based GPU
path would need, against which the hull path's fixed log-depth is compared:

  * the benchmark vector, N(0, 1) + 10 % exact duplicates (seed 0), at d = 2^22
    and 2^24, lambda in {1e-2, 1, 1e2};
  * the adversarial cascade (Sec. 4.1's worst case), d = 2^16;
  * the MLP 3072-4096-4096-10 rows during proximal SGD (lr 0.1, alpha 1e-3,
    lambda = lr alpha per row, batch 256 of synthetic 32x32x3 images): the
    weights just before each prox, on a seeded sample of 512 rows, steps 1-5.

Usage: python -m oracle.ic_rounds_report   (prints one JSON object)
"""
from __future__ import annotations

import json
import time

import numpy as np

import oracle
from paper_2311_03096_gb300 import inputs


def rounds(w, lam):
    _, _, nc, r, conv = oracle.imminent_collisions_v2(w, lam)
    return {"rounds": r, "clusters": nc, "converged": conv}


def training_rows(steps=5, sample=512, lr=0.1, alpha=1e-3, seed=0):
    import torch
    mats = [torch.from_numpy(m.astype(np.float32)) for m in inputs.mlp_weights(seed)]
    biases = [torch.zeros(m.shape[0]) for m in mats]
    x_np, y_np = inputs.images(batch=256, seed=seed)
    x, y = torch.from_numpy(x_np), torch.from_numpy(y_np).long()
    rows = [(l, r) for l, m in enumerate(mats) for r in range(m.shape[0])]
    pick = np.random.default_rng(seed + 1).choice(len(rows), sample, replace=False)
    lam = lr * alpha
    per_step = []
    for _ in range(steps):
        ps = [m.clone().requires_grad_(True) for m in mats]
        h = x
        for l, (wm, b) in enumerate(zip(ps, biases)):
            h = torch.nn.functional.linear(h, wm, b)
            if l + 1 < len(ps):
                h = torch.relu(h)
        loss = torch.nn.functional.cross_entropy(h, y)
        grads = torch.autograd.grad(loss, ps)
        mats = [(m - lr * g).detach() for m, g in zip(mats, grads)]
        rs = [oracle.imminent_collisions_v2(mats[rows[i][0]][rows[i][1]].numpy(), lam)[3] for i in pick]
        per_step.append({"loss": float(loss.detach()), "rounds_max": int(max(rs)), "rounds_mean": float(np.mean(rs))})
        # the prox of every row (oracle), as in the training step
        for l, m in enumerate(mats):
            a = m.numpy().astype(np.float64)
            off = np.arange(a.shape[0] + 1, dtype=np.int64) * a.shape[1]
            out, _, _ = oracle.prox_batched(a.reshape(-1), off, np.full(a.shape[0], lam))
            mats[l] = torch.from_numpy(out.reshape(a.shape).astype(np.float32))
    return {"lambda": lam, "rows_sampled": sample, "steps": per_step}


def main():
    t0 = time.time()
    rep = {"benchmark_vector": {}, "cascade": {}, "training_rows": None}
    for d in (1 << 22, 1 << 24):
        w = inputs.normal_with_duplicates(d, seed=0)
        rep["benchmark_vector"][f"d=2^{d.bit_length() - 1}"] = {f"lam={lam:g}": rounds(w, lam) for lam in (1e-2, 1.0, 1e2)}
    w, lam = inputs.cascade(1 << 16, seed=1, shuffle=True)
    rep["cascade"]["d=2^16"] = rounds(w, lam)
    rep["training_rows"] = training_rows()
    rep["seconds"] = round(time.time() - t0, 1)
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
