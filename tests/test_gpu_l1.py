"""GPU parity of weight sharing + l1 with rewinding (Alg. 2, Rewinding section)
through ws_prox_l1 / ws_prox_batched_l1, against the FP64 oracle.

Cluster ids must equal the oracle's.  Values must agree within the path's
tolerance, except for clusters whose zero-mask decision |x + v| < beta is a
near-tie (| |x + v| - beta | within the same tolerance): there either outcome
is accepted, because the two sides round x + v differently.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2311_03096_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}
TOL = {("f64", "fp64"): 1e-12, ("f64", "fp32comp"): 1e-5, ("f32", "fp64"): 1e-5, ("f32", "fp32comp"): 1e-5}


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


def check_l1(w, lam, beta, rho, vs, out, ids, tol):
    w = np.asarray(w, np.float64)
    ref, rid, nc = oracle.prox_l1(w, lam, beta, rho, vs)
    assert np.array_equal(np.asarray(ids), rid), "cluster ids differ from the oracle"
    scale = (float(np.abs(w).max()) if w.size else 0.0) + lam + beta
    out = np.asarray(out, np.float64)
    err = np.abs(out - ref)
    bad = err > tol * scale
    if bad.any():
        # accepted only where the oracle's zero-mask decision is a near-tie
        p, _, _ = oracle.prox(w, lam)
        near = np.abs(np.abs(p) - beta) <= 4 * tol * scale
        assert np.all(near[bad]), f"max err {err[bad & ~near].max():.3e} beyond {tol:.0e} * {scale:.3e}"
    return int(bad.sum())


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("d", [1, 2, 100, 4096, 70001, 2 ** 20])
def test_prox_l1_single(ws, ctx, dt, d):
    w_np = inputs.normal_with_duplicates(d, seed=d + 5, dtype=NP[dt])
    w = torch.from_numpy(w_np).cuda()
    for lam in (0.01, 1.0):
        for beta, rho, vs in ((0.0, 0.0, 1.0), (0.05, 0.0, 1.0), (0.5, 0.3, 1.0), (0.2, 1.0, 1.0), (0.1, 0.5, 0.1)):
            for prec in ("fp32comp", "fp64"):
                out, ids, nc = ws.prox_l1(w, lam, beta, rho, vs, prec, ctx=ctx)
                ctx.check(what="prox_l1")
                check_l1(w_np, lam, beta, rho, vs, out.cpu().numpy(), ids.cpu().numpy(), TOL[(dt, prec)])


def test_prox_l1_beta0_equals_prox(ws, ctx):
    w_np = inputs.normal_with_duplicates(50000, seed=3, dtype=np.float32)
    w = torch.from_numpy(w_np).cuda()
    a, ia, _ = ws.prox(w, 0.3, "fp64", ctx=ctx)
    b, ib, _ = ws.prox_l1(w, 0.3, 0.0, 0.0, 1.0, "fp64", ctx=ctx)
    ctx.check(what="prox_l1")
    assert torch.equal(ia, ib)
    assert torch.equal(a, b)


def test_prox_l1_batched(ws, ctx):
    rng = np.random.default_rng(17)
    lens = rng.integers(0, 30000, 30)
    lens[:5] = [0, 1, 2, 4096, 9000]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = inputs.normal_with_duplicates(int(off[-1]), seed=18, dtype=np.float32)
    lam = np.exp(rng.uniform(np.log(1e-3), np.log(3.0), len(lens)))
    plan = ws.Plan(off, torch.float32)
    v = torch.from_numpy(vals).cuda()
    lt = torch.from_numpy(lam).cuda()
    for beta, rho, vs in ((0.1, 0.0, 1.0), (0.3, 0.7, 0.5)):
        out, ids, nc = plan.forward_l1(v, lt, beta, rho, vs, "fp32comp")
        ctx.check(what="batched l1")
        out, ids = out.cpu().numpy(), ids.cpu().numpy()
        for s in range(len(lens)):
            a, b = off[s], off[s + 1]
            if b > a:
                check_l1(vals[a:b], lam[s], beta, rho, vs, out[a:b], ids[a:b], 1e-5)


def test_prox_l1_invalid(ws, ctx):
    w = torch.zeros(10, device="cuda")
    for beta, rho, vs in ((-0.1, 0.0, 1.0), (0.1, 1.5, 1.0), (0.1, -0.1, 1.0), (0.1, 0.0, -1.0),
                          (float("nan"), 0.0, 1.0)):
        with pytest.raises(ws.WSError):
            ws.prox_l1(w, 0.1, beta, rho, vs, ctx=ctx)
