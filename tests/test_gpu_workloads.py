"""GPU parity at the benchmark workloads' full sizes (through the C ABI, in the
launch configuration bench.py times), against the FP64 oracle.

  - single vector, d = 2^24 and 2^26 FP32 N(0,1) + 10% duplicates (seed 0,
    the bench's vector), lambda in {1e-2, 1, 1e2}, FP32-comp and FP64
    arithmetic: every output compared with the oracle;
  - adversarial cascade (sorted and shuffled) and mirror at d = 2^24;
  - the batched MLP layout (8202 rows, 3 whole layers, 4096 log-uniform
    extra segments, ~3.9e8 elements): every segment computed on the GPU,
    all layers plus a seeded sample of rows and extras compared with the
    oracle segment by segment; the same call captured in a CUDA graph and
    replayed on new values;
  - the proximal training step on the MLP (SGD then prox of every row), and
    the cluster-averaging backward of WSProx against central finite
    differences (eps = 1e-6, FP64, d = 64 segments).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
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
    c.set_spin_limit(0)
    c.status()
    yield c


@pytest.mark.parametrize("d", [2 ** 24, 2 ** 26])
def test_single_vector_full_size(ws, ctx, d):
    w_np = inputs.normal_with_duplicates(d, seed=0, dtype=np.float32)
    w = torch.from_numpy(w_np).cuda()
    out = torch.empty_like(w)
    nc = torch.zeros(1, dtype=torch.int64, device="cuda")
    for lam in (1e-2, 1.0, 1e2):
        ref = oracle.prox(w_np, lam, return_perm=True)
        for prec in ("fp32comp", "fp64"):
            o, i, n = ws.prox(w, lam, prec, ctx=ctx, out=out, n_clusters=nc)
            ctx.check(what="prox")
            compare_segment(w_np, lam, o.cpu().numpy(), i.cpu().numpy(), int(n.item()), 1e-5, ref=ref)
        del ref


@pytest.mark.parametrize("shuffle", [False, True])
def test_cascade_2e24(ws, ctx, shuffle):
    d = 2 ** 24
    w_np, lam = inputs.cascade(d, seed=1, shuffle=shuffle)
    w = torch.from_numpy(w_np).cuda()
    out, ids, nc = ws.prox(w, lam, "fp32comp", ctx=ctx)
    ctx.check(what="prox")
    assert int(nc.item()) == 1
    compare_segment(w_np, lam, out.cpu().numpy(), ids.cpu().numpy(), int(nc.item()), 1e-5)


def test_mirror_2e24(ws, ctx):
    d = 2 ** 24
    w_np, lam = inputs.mirror(d, seed=2, shuffle=True)
    w = torch.from_numpy(w_np).cuda()
    out, ids, nc = ws.prox(w, lam, "fp32comp", ctx=ctx)
    ctx.check(what="prox")
    assert int(nc.item()) == d // 2
    compare_segment(w_np, lam, out.cpu().numpy(), ids.cpu().numpy(), int(nc.item()), 1e-5)


@pytest.fixture(scope="module")
def mlp_batch():
    return inputs.batched_segments(seed=0)


def _sample_segments(kinds, lens, seed=7, n_rows=48, n_extra=32):
    kinds = np.asarray(kinds)
    rng = np.random.default_rng(seed)
    layers = np.nonzero(kinds == "layer")[0]
    rows = np.nonzero(kinds == "row")[0]
    extra = np.nonzero(kinds == "extra")[0]
    pick = list(layers) + list(rng.choice(rows, n_rows, replace=False)) + list(rng.choice(extra, n_extra, replace=False))
    pick += [extra[np.argmax(lens[extra])], extra[np.argmin(lens[extra])]]
    return sorted(set(int(s) for s in pick))


def test_batched_mlp_full(ws, ctx, mlp_batch):
    vals, off, lam, kinds = mlp_batch
    assert off[-1] > 3.0e8
    plan = ws.Plan(off, torch.float32)
    v = torch.from_numpy(vals).cuda()
    lt = torch.from_numpy(lam).cuda()
    sample = _sample_segments(kinds, np.diff(off))
    refs = {s: oracle.prox(vals[off[s]:off[s + 1]], float(lam[s]), return_perm=True) for s in sample}
    for prec in ("fp32comp", "fp64"):
        out, ids, nc = plan.forward(v, lt, prec)
        ctx.check(what="batched")
        out_h, ids_h, nc_h = out.cpu().numpy(), ids.cpu().numpy(), nc.cpu().numpy()
        # every segment: ids are ranked clusters 0..nc-1 and out is constant on each
        assert np.all(nc_h[np.diff(off) > 0] >= 1)
        for s in sample:
            a, b = off[s], off[s + 1]
            compare_segment(vals[a:b], float(lam[s]), out_h[a:b], ids_h[a:b], nc_h[s], 1e-5, ref=refs[s])
        del out, ids, nc


def test_batched_graph_replay(ws, ctx):
    vals, off, lam, kinds = inputs.batched_segments(seed=3, layers=True, extra=256)
    plan = ws.Plan(off, torch.float32)
    v = torch.from_numpy(vals).cuda()
    lt = torch.from_numpy(lam).cuda()
    out = torch.empty_like(v)
    ids = torch.empty(v.shape[0], dtype=torch.int32, device="cuda")
    nc = torch.zeros(len(lam), dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forward(v, lt, "fp32comp", out=out, id_out=ids, n_clusters=nc)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.forward(v, lt, "fp32comp", out=out, id_out=ids, n_clusters=nc)
    for seed in (11, 12):
        new = inputs.normal(v.shape[0], seed=seed, dtype=np.float32)
        v.copy_(torch.from_numpy(new))
        out.zero_()
        ids.fill_(-1)
        g.replay()
        torch.cuda.synchronize()
        ctx.check(what="graph replay")
        e_out, e_ids, e_nc = plan.forward(v, lt, "fp32comp")
        ctx.check(what="eager")
        assert torch.equal(out, e_out) and torch.equal(ids, e_ids) and torch.equal(nc, e_nc)
        for s in (0, len(lam) - 1, int(np.argmax(np.diff(off)))):
            a, b = off[s], off[s + 1]
            compare_segment(new[a:b], float(lam[s]), out[a:b].cpu().numpy(), ids[a:b].cpu().numpy(),
                            int(nc[s].item()), 1e-5)


def test_training_step_rows_are_prox(ws, ctx):
    from paper_2311_03096_gb300.train import ProxMLP

    m = ProxMLP(seed=0)
    x_np, y_np = inputs.images(batch=256, seed=0)
    x, y = torch.from_numpy(x_np).cuda(), torch.from_numpy(y_np).cuda()
    loss0 = float(m.loss(x, y).item())
    for _ in range(2):
        m.sgd(x, y)
        before = m.flat.cpu().numpy()
        m.prox()
        ctx.check(what="train prox")
        after = m.flat.cpu().numpy()
        rng = np.random.default_rng(5)
        rows = rng.choice(m.offsets.shape[0] - 1, 24, replace=False)
        lam = m.lr * m.alpha
        for r in rows:
            a, b = m.offsets[r], m.offsets[r + 1]
            compare_segment(before[a:b], lam, after[a:b], m.ids[a:b].cpu().numpy(), int(m.n_clusters[r].item()),
                            1e-5)
    assert np.isfinite(loss0) and np.isfinite(float(m.loss(x, y).item()))


def test_wsprox_backward_central_fd(ws, ctx):
    rng = np.random.default_rng(4)
    rows, d, lam, eps = 6, 64, 0.05, 1e-6
    w0 = rng.standard_normal((rows, d))
    gout = torch.from_numpy(rng.standard_normal((rows, d))).cuda()
    w = torch.from_numpy(w0).cuda().requires_grad_(True)
    out = ws.WSProx.apply(w, lam, "fp64")
    (out * gout).sum().backward()
    grad = w.grad.cpu().numpy()
    # the cluster-averaging Jacobian also matches the oracle's
    ids = ws.prox(torch.from_numpy(w0[0]).cuda(), lam, "fp64")[1].cpu().numpy()
    np.testing.assert_allclose(grad[0], oracle.backward(gout[0].cpu().numpy(), ids), atol=1e-12)

    def f(wn):
        with torch.no_grad():
            o = ws.WSProx.apply(torch.from_numpy(wn).cuda(), lam, "fp64")
            return float((o * gout).sum().item())

    checked = 0
    base_ids = [oracle.prox(w0[r], lam)[1] for r in range(rows)]
    for r in range(rows):
        for i in range(d):
            wp, wm = w0.copy(), w0.copy()
            wp[r, i] += eps
            wm[r, i] -= eps
            # central differences are only the derivative where the partition is locally constant
            if not (np.array_equal(oracle.prox(wp[r], lam)[1], base_ids[r])
                    and np.array_equal(oracle.prox(wm[r], lam)[1], base_ids[r])):
                continue
            fd = (f(wp) - f(wm)) / (2 * eps)
            assert abs(fd - grad[r, i]) <= 1e-6 * (1 + abs(grad[r, i])), (r, i, fd, grad[r, i])
            checked += 1
    assert checked >= 0.95 * rows * d
