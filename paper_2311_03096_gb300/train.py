"""Proximal SGD on the MLP 3072 -> 4096 -> 4096 -> 10: the training step the
prox is used in (Sec. 5: an SGD step on the loss, then the proximal map of
lr * alpha * R applied to every output-neuron row of every weight matrix).

All rows of all layers live in one flat float32 buffer, so the prox of every
row is one ws_prox_batched call (one segment per row, one lambda per row).
The MLP forward/backward itself is plain PyTorch; only the prox runs through
the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import inputs, ws


class ProxMLP:
    def __init__(self, sizes=inputs.MLP_SIZES, seed: int = 0, lr: float = 0.1, alpha: float = 1e-3,
                 prec: str = "fp32comp", device="cuda", warm: bool = False):
        self.sizes = tuple(sizes)
        self.lr, self.alpha, self.prec = lr, alpha, prec
        self.warm = warm   # start every row's prox from the previous step's clusters (same result)
        mats = inputs.mlp_weights(seed, sizes)
        self.shapes = [m.shape for m in mats]
        numel = [m.size for m in mats]
        self.flat = torch.from_numpy(np.concatenate([m.reshape(-1) for m in mats])).to(device)
        self.flat_out = torch.empty_like(self.flat)
        self.bounds = np.concatenate([[0], np.cumsum(numel)]).astype(np.int64)
        # one segment per output-neuron row, rows of layer l back to back
        offs = [np.arange(r, dtype=np.int64) * c + self.bounds[l] for l, (r, c) in enumerate(self.shapes)]
        self.offsets = np.concatenate(offs + [np.array([self.bounds[-1]], np.int64)])
        self.plan = ws.Plan(self.offsets, torch.float32)
        n_rows = self.offsets.shape[0] - 1
        self.lams = torch.full((n_rows,), lr * alpha, dtype=torch.float64, device=device)
        self.ids = torch.zeros(self.flat.shape[0], dtype=torch.int32, device=device)
        self.n_clusters = torch.zeros(n_rows, dtype=torch.int64, device=device)
        self.biases = [torch.zeros(r, device=device) for r, _ in self.shapes]

    def weights(self, flat=None):
        flat = self.flat if flat is None else flat
        return [flat[self.bounds[l]:self.bounds[l + 1]].view(*s) for l, s in enumerate(self.shapes)]

    def loss(self, x, y, flat=None):
        h = x
        ws_ = self.weights(flat)
        for l, (w, b) in enumerate(zip(ws_, self.biases)):
            h = torch.nn.functional.linear(h, w, b)
            if l + 1 < len(ws_):
                h = torch.relu(h)
        return torch.nn.functional.cross_entropy(h, y)

    def sgd(self, x, y):
        """Loss, gradient and the SGD update of the weights (no prox)."""
        flat = self.flat.detach().requires_grad_(True)
        loss = self.loss(x, y, flat)
        (g,) = torch.autograd.grad(loss, flat)
        with torch.no_grad():
            self.flat.sub_(self.lr * g)
        return loss.detach()

    def prox(self, stream=None):
        """prox_{lr alpha R} of every row, from self.flat into self.flat_out; then swap."""
        self.plan.forward(self.flat, self.lams, self.prec, out=self.flat_out, id_out=self.ids,
                          n_clusters=self.n_clusters, stream=stream, ids_prev=self.ids if self.warm else None)
        self.flat, self.flat_out = self.flat_out, self.flat

    def step(self, x, y):
        loss = self.sgd(x, y)
        self.prox()
        return loss
