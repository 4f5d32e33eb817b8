"""GPU R(w) and weight-sharing measure (ws_R) against the oracle: R by the
appendix "Computing R" formula in FP64 (and the O(d^2) definition on small
inputs), the measure by its definition (#distinct nonzero / #nonzero)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2311_03096_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}


@pytest.fixture(scope="module")
def ws():
    from paper_2311_03096_gb300 import ws as _ws
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return _ws


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("d", [0, 1, 2, 300, 5000, 70001, 2 ** 20 + 7])
def test_R_and_measure(ws, dt, d):
    ctx = ws.Context.get(0)
    w_np = inputs.normal_with_duplicates(d, seed=d + 1, dtype=NP[dt]) if d else np.zeros(0, NP[dt])
    if d > 4:
        w_np[:3] = 0.0
        w_np[3] = -0.0
    w = torch.from_numpy(w_np).cuda()
    r, m = ws.R(w, ctx=ctx)
    ctx.check(what="ws_R")
    ref = oracle.R_sorted(w_np) if d > 1 else 0.0
    assert abs(float(r.item()) - ref) <= 1e-10 * max(1.0, abs(ref))
    if 1 < d <= 300:
        assert abs(float(r.item()) - oracle.R_pairs(w_np)) <= 1e-10 * max(1.0, abs(ref))
    assert float(m.item()) == oracle.ws_measure(w_np)


def test_measure_of_prox_output(ws):
    ctx = ws.Context.get(0)
    w_np = inputs.normal_with_duplicates(100000, seed=5, dtype=np.float32)
    w = torch.from_numpy(w_np).cuda()
    out, ids, nc = ws.prox_l1(w, 0.5, 0.2, 0.0, 1.0, "fp64", ctx=ctx)
    r, m = ws.R(out, ctx=ctx)
    ctx.check(what="ws_R")
    o = out.cpu().numpy()
    assert float(m.item()) == oracle.ws_measure(o)
    assert abs(float(r.item()) - oracle.R_sorted(o)) <= 1e-10 * max(1.0, oracle.R_sorted(o))


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_dlambda_single(ws, dt):
    ctx = ws.Context.get(0)
    for d in (1, 2, 300, 4096, 70001, 2 ** 20 + 3):
        w_np = inputs.normal_with_duplicates(d, seed=d + 9, dtype=NP[dt])
        g_np = inputs.normal(d, seed=d + 10, dtype=NP[dt])
        w, g = torch.from_numpy(w_np).cuda(), torch.from_numpy(g_np).cuda()
        for lam in (0.01, 1.0):
            out, ids, _ = ws.prox(w, lam, "fp64", ctx=ctx)
            got = float(ws.prox_dlambda(g, ids, ctx=ctx).item())
            ctx.check(what="dlambda")
            ref = oracle.dlambda(g_np, ids.cpu().numpy())[0]
            assert abs(got - ref) <= 1e-9 * (1 + np.abs(g_np).sum() / max(d, 1)) * max(1.0, abs(ref)), (d, lam)


def test_dlambda_batched(ws):
    ctx = ws.Context.get(0)
    rng = np.random.default_rng(61)
    lens = rng.integers(0, 40000, 40)
    lens[:6] = [0, 1, 2, 4096, 4097, 9000]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = inputs.normal_with_duplicates(int(off[-1]), seed=62, dtype=np.float32)
    g_np = inputs.normal(int(off[-1]), seed=63, dtype=np.float32)
    lam = np.exp(rng.uniform(np.log(1e-3), np.log(3.0), len(lens)))
    plan = ws.Plan(off, torch.float32)
    out, ids, nc = plan.forward(torch.from_numpy(vals).cuda(), torch.from_numpy(lam).cuda(), "fp64")
    got = plan.dlambda(torch.from_numpy(g_np).cuda(), ids).cpu().numpy()
    ctx.check(what="dlambda batched")
    ref = oracle.dlambda(g_np, ids.cpu().numpy(), off)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-9)
