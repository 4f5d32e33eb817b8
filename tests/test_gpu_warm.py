"""Warm start across steps (the paper's Future Work: start from a candidate
weight-sharing and edit it into the exact one), through ws_prox_batched_warm.

The candidate (runs of equal earlier cluster ids along the sorted order) only
decides which points the Imminent Collisions rounds start from; every point
that can be a hull vertex is kept, so the outputs must be bit-identical to the
cold call whatever the earlier ids are: the previous step's, stale ones,
garbage, all zeros, or the output buffer itself (aliasing).  And the proximal
training step with the warm start must match the oracle at every step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2311_03096_gb300 import inputs  # noqa: E402
from parity import compare_segment  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    from paper_2311_03096_gb300 import ws as _ws
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _ws


@pytest.fixture()
def ctx(ws):
    c = ws.Context.get(0)
    c.set_small_max(-1)
    c.set_ic_cap(-1)
    c.status()
    yield c
    c.set_ic_cap(-1)


def _same(a, b):
    return all(torch.equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("lam_mode", ["logu", "large"])
@pytest.mark.parametrize("dt", [torch.float32, torch.float64])
def test_warm_equals_cold_for_any_candidate(ws, ctx, lam_mode, dt):
    vals, off, lam, kinds = inputs.batched_segments(seed=7, layers=False, extra=0)
    if lam_mode == "large":
        lam = np.full_like(lam, 0.1)   # clusters of hundreds of weights
    np_dt = np.float32 if dt == torch.float32 else np.float64
    prec = "fp32comp" if dt == torch.float32 else "fp64"
    plan = ws.Plan(off, dt, ctx=ctx)
    lt = torch.from_numpy(lam).cuda()
    v1 = torch.from_numpy(vals.astype(np_dt)).cuda()
    out1, ids1, _ = plan.forward(v1, lt, prec)
    # the next step's input: the prox output moved by a small gradient step
    g = torch.from_numpy(inputs.normal(v1.shape[0], seed=8, dtype=np_dt)).cuda()
    v2 = out1 - 1e-3 * float(v1.std()) * g
    cold = [t.clone() for t in plan.forward(v2, lt, prec)]
    n = v2.shape[0]
    rng = np.random.default_rng(9)
    candidates = {
        "previous step": ids1.clone(),
        "exact": cold[1].clone(),
        "zeros": torch.zeros(n, dtype=torch.int32, device="cuda"),
        "garbage": torch.from_numpy(rng.integers(-2 ** 31, 2 ** 31 - 1, n, dtype=np.int64).astype(np.int32)).cuda(),
        "singletons": torch.arange(n, dtype=torch.int32, device="cuda"),
    }
    for name, prev in candidates.items():
        warm = plan.forward(v2, lt, prec, ids_prev=prev)
        ctx.check(what=f"warm {name}")
        assert _same(cold, warm), name
    # aliasing: the earlier ids are read from the output buffer itself
    buf = ids1.clone()
    warm = plan.forward(v2, lt, prec, id_out=buf, ids_prev=buf)
    ctx.check(what="warm aliased")
    assert _same(cold, warm)
    # and against the oracle on a sample of rows
    w_np = v2.cpu().numpy()
    o_np, i_np, nc_np = (t.cpu().numpy() for t in warm)
    tol = 1e-5 if dt == torch.float32 else 1e-12
    for s in rng.choice(off.shape[0] - 1, 12, replace=False):
        a, b = off[s], off[s + 1]
        compare_segment(w_np[a:b], float(lam[s]), o_np[a:b], i_np[a:b], int(nc_np[s]), tol)


def test_warm_with_round_cap_and_fallback(ws, ctx):
    # a cap of 1 round sends every segment whose candidate is not already
    # the answer to the tree of merges; the outputs still must not change
    vals, off, lam, kinds = inputs.batched_segments(seed=11, layers=False, extra=0)
    plan = ws.Plan(off, torch.float32, ctx=ctx)
    lt = torch.from_numpy(np.full_like(lam, 3e-2)).cuda()
    v = torch.from_numpy(vals).cuda()
    cold = [t.clone() for t in plan.forward(v, lt)]
    prev = torch.zeros(v.shape[0], dtype=torch.int32, device="cuda")
    for cap in (1, 2, 0):
        ctx.set_ic_cap(cap)
        warm = plan.forward(v, lt, ids_prev=prev)
        ctx.check(what=f"warm cap {cap}")
        assert _same(cold, warm), cap


def test_proximal_training_warm_start(ws, ctx):
    from paper_2311_03096_gb300.train import ProxMLP

    cold = ProxMLP(seed=0)
    warm = ProxMLP(seed=0, warm=True)
    x_np, y_np = inputs.images(batch=256, seed=0)
    x, y = torch.from_numpy(x_np).cuda(), torch.from_numpy(y_np).cuda()
    rng = np.random.default_rng(13)
    lam = warm.lr * warm.alpha
    for step in range(5):
        cold.sgd(x, y)
        warm.sgd(x, y)
        before = warm.flat.cpu().numpy()
        cold.prox()
        warm.prox()
        ctx.check(what="warm train prox")
        assert torch.equal(cold.flat, warm.flat), step
        assert torch.equal(cold.ids, warm.ids), step
        after = warm.flat.cpu().numpy()
        ids = warm.ids.cpu().numpy()
        for r in rng.choice(warm.offsets.shape[0] - 1, 8, replace=False):
            a, b = warm.offsets[r], warm.offsets[r + 1]
            compare_segment(before[a:b], lam, after[a:b], ids[a:b], int(warm.n_clusters[r].item()), 1e-5)


def test_warm_requires_ids(ws, ctx):
    plan = ws.Plan(np.array([0, 100], np.int64), torch.float32, ctx=ctx)
    v = torch.zeros(100, device="cuda")
    lt = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        plan.forward(v, lt, ids_prev=torch.zeros(99, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        plan.forward(v, lt, ids_prev=torch.zeros(100, dtype=torch.int64, device="cuda"))
