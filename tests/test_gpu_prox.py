"""GPU parity tests: the CUDA path (through the C ABI) against the FP64 oracle.

Every input is seeded and synthetic (paper_2311_03096_gb300.inputs).  Sizes
are chosen so the oracle finishes in seconds while the GPU path still spans
several tiles and a ragged tail; the device-wide path is also forced onto
small inputs with ws_debug_set_small_max.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2311_03096_gb300 import inputs  # noqa: E402
from parity import compare_segment  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {("f64", "fp64"): 1e-12, ("f64", "fp32comp"): 1e-5, ("f32", "fp64"): 1e-5, ("f32", "fp32comp"): 1e-5}
NP = {"f32": np.float32, "f64": np.float64}
TT = {"f32": torch.float32, "f64": torch.float64}


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
    c.set_small_max(-1)
    c.set_spin_limit(0)


def run_one(ws, ctx, w_np, lam, dt, prec):
    w = torch.from_numpy(w_np).cuda()
    out, ids, nc = ws.prox(w, lam, prec)
    ctx.check(what="prox")
    return out.cpu().numpy(), ids.cpu().numpy(), int(nc.item())


# -- config: plain FP64 prox, d = 4096, lambda in {0, 0.1, 1, 1000} (single-CTA path)
@pytest.mark.parametrize("lam", [0.0, 0.1, 1.0, 1000.0])
@pytest.mark.parametrize("prec", ["fp64", "fp32comp"])
def test_d4096_fp64(ws, ctx, lam, prec):
    w_np = inputs.normal(4096, seed=0, dtype=np.float64)
    out, ids, nc = run_one(ws, ctx, w_np, lam, "f64", prec)
    compare_segment(w_np, lam, out, ids, nc, TOL[("f64", prec)])
    if lam == 0.0 and prec == "fp64":
        assert np.array_equal(out, w_np)   # identity, bit for bit
    if lam == 1000.0:
        assert nc == 1


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("d", [0, 1, 2, 3, 31, 32, 33, 255, 1000, 2047, 2048, 4095, 4096])
def test_small_sizes(ws, ctx, dt, d):
    w_np = inputs.normal_with_duplicates(d, seed=d + 17, dtype=NP[dt])
    for lam in (0.0, 0.05, 2.0):
        for prec in ("fp32comp", "fp64"):
            out, ids, nc = run_one(ws, ctx, w_np, lam, dt, prec)
            compare_segment(w_np, lam, out, ids, nc, TOL[(dt, prec)])


def test_ties_and_signed_zero(ws, ctx):
    w_np = np.array([0.0, -0.0, 1.0, 1.0, -1.0, 0.0, -0.0, 1.0], np.float32)
    for lam in (0.0, 0.01, 1.0):
        out, ids, nc = run_one(ws, ctx, w_np, lam, "f32", "fp64")
        compare_segment(w_np, lam, out, ids, nc, 1e-6)


@pytest.mark.parametrize("small_max", [0, 64, 1000])
@pytest.mark.parametrize("d", [2, 3, 100, 4096, 4097, 9000, 20000])
def test_device_wide_path_forced(ws, ctx, small_max, d):
    ctx.set_small_max(small_max)
    w_np = inputs.normal_with_duplicates(d, seed=d, dtype=np.float32)
    for lam in (0.0, 1e-3, 0.3, 50.0):
        out, ids, nc = run_one(ws, ctx, w_np, lam, "f32", "fp64")
        compare_segment(w_np, lam, out, ids, nc, 1e-5)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("d", [5000, 70000, 2 ** 20 + 3])
def test_device_wide_path(ws, ctx, dt, d):
    w_np = inputs.normal_with_duplicates(d, seed=d, dtype=NP[dt])
    for lam in (1e-2, 1.0, 1e2):
        ref = oracle.prox(w_np, lam, return_perm=True)
        for prec in ("fp32comp", "fp64"):
            out, ids, nc = run_one(ws, ctx, w_np, lam, dt, prec)
            compare_segment(w_np, lam, out, ids, nc, TOL[(dt, prec)], ref=ref)


@pytest.mark.parametrize("d", [2 ** 12, 2 ** 16, 2 ** 20])
@pytest.mark.parametrize("shuffle", [False, True])
def test_cascade(ws, ctx, d, shuffle):
    w_np, lam = inputs.cascade(d, seed=1, shuffle=shuffle)
    out, ids, nc = run_one(ws, ctx, w_np, lam, "f32", "fp64")
    compare_segment(w_np, lam, out, ids, nc, 1e-5)
    assert nc == 1


@pytest.mark.parametrize("d", [2 ** 12, 2 ** 16, 2 ** 20])
def test_mirror(ws, ctx, d):
    w_np, lam = inputs.mirror(d, seed=2, shuffle=True)
    out, ids, nc = run_one(ws, ctx, w_np, lam, "f32", "fp64")
    compare_segment(w_np, lam, out, ids, nc, 1e-5)
    assert nc == d // 2


def test_debug_sort_bit_exact(ws, ctx):
    ctx.set_small_max(0)
    for dt in ("f32", "f64"):
        for d in (3, 8192, 8193, 50000):
            w_np = inputs.normal_with_duplicates(d, seed=d, dtype=NP[dt])
            w_np[:5] = np.array([0.0, -0.0, 0.0, -0.0, 1.0], NP[dt])[: min(5, d)]
            plan = ws.Plan([0, d], TT[dt])
            w = torch.from_numpy(w_np).cuda()
            s = torch.zeros_like(w)
            plan.debug_sort(w, s)
            ctx.check(what="debug_sort")
            _, xs = oracle.sort(w_np)
            got = s.cpu().numpy()
            # bit-exact, including the sign of zeros
            assert np.array_equal(got.view(np.uint32 if dt == "f32" else np.uint64),
                                  xs.astype(NP[dt]).view(np.uint32 if dt == "f32" else np.uint64))


def _batched_case(seed, n_seg=40, maxlen=30000):
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, maxlen, n_seg)
    lens[:6] = [0, 1, 2, 4096, 4097, 8193]
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    vals = inputs.normal_with_duplicates(int(off[-1]), seed=seed, dtype=np.float32)
    lam = np.exp(rng.uniform(np.log(1e-3), np.log(10.0), n_seg))
    return vals, off, lam


@pytest.mark.parametrize("prec", ["fp32comp", "fp64"])
def test_batched(ws, ctx, prec):
    vals, off, lam = _batched_case(3)
    plan = ws.Plan(off, torch.float32)
    out, ids, nc = plan.forward(torch.from_numpy(vals).cuda(), torch.from_numpy(lam).cuda(), prec)
    ctx.check(what="batched")
    out, ids, nc = out.cpu().numpy(), ids.cpu().numpy(), nc.cpu().numpy()
    for s in range(len(lam)):
        a, b = off[s], off[s + 1]
        compare_segment(vals[a:b], lam[s], out[a:b], ids[a:b], nc[s], 1e-5)


@pytest.mark.parametrize("dt", ["f32", "f64"])
def test_backward_matches_oracle(ws, ctx, dt):
    vals, off, lam = _batched_case(4, n_seg=12)
    vals = vals.astype(NP[dt])
    plan = ws.Plan(off, TT[dt])
    out, ids, nc = plan.forward(torch.from_numpy(vals).cuda(), torch.from_numpy(lam).cuda(), "fp64")
    g = inputs.normal(vals.shape[0], seed=9, dtype=NP[dt])
    gin = plan.backward(torch.from_numpy(g).cuda(), ids)
    ctx.check(what="backward")
    ref = oracle.backward(g, ids.cpu().numpy(), off)
    tol = 1e-12 if dt == "f64" else 1e-5
    np.testing.assert_allclose(gin.cpu().numpy(), ref, atol=tol * (1 + np.abs(g).max()))


def test_nonfinite_reported(ws, ctx):
    for d in (100, 20000):
        w_np = inputs.normal(d, seed=1, dtype=np.float32)
        w_np[d // 2] = np.nan
        w = torch.from_numpy(w_np).cuda()
        ws.prox(w, 0.1)
        assert ctx.status() == ws.WS_ERR_NONFINITE
        w_np[d // 2] = np.inf
        ws.prox(torch.from_numpy(w_np).cuda(), 0.1)
        assert ctx.status() == ws.WS_ERR_NONFINITE
    # the context stays usable
    w_np = inputs.normal(1000, seed=2, dtype=np.float32)
    out, ids, nc = run_one(ws, ctx, w_np, 0.1, "f32", "fp64")
    compare_segment(w_np, 0.1, out, ids, nc, 1e-5)


def test_invalid_arguments(ws, ctx):
    w = torch.zeros(10, device="cuda")
    with pytest.raises(ws.WSError):
        ws.prox(w, -1.0)
    with pytest.raises(ws.WSError):
        ws.prox(w, float("nan"))
    with pytest.raises(ws.WSError):
        ws.Plan([1, 5])
    plan = ws.Plan([0, 5, 10])
    bad = torch.tensor([0.1, -0.5], dtype=torch.float64, device="cuda")
    plan.forward(w, bad)
    assert ctx.status() == ws.WS_ERR_INVALID


def test_spin_wait_gives_up(ws, ctx):
    """A look-back wait with a tiny bound gives up, reports WS_ERR_TIMEOUT and
    the kernel exits; the context stays usable."""
    ctx.set_spin_limit(1)
    w_np = inputs.normal(2 ** 22, seed=3, dtype=np.float32)
    w = torch.from_numpy(w_np).cuda()
    st = ws.WS_OK
    for _ in range(5):
        ws.prox(w, 0.5)
        st = ctx.status()
        if st == ws.WS_ERR_TIMEOUT:
            break
        assert st == ws.WS_OK
    assert st == ws.WS_ERR_TIMEOUT
    ctx.set_spin_limit(0)
    w_np = inputs.normal(20000, seed=4, dtype=np.float32)
    out, ids, nc = run_one(ws, ctx, w_np, 0.5, "f32", "fp64")
    compare_segment(w_np, 0.5, out, ids, nc, 1e-5)


def test_autotuned_plan_matches_default(ws, ctx):
    vals, off, lam = _batched_case(21, n_seg=60, maxlen=9000)
    v = torch.from_numpy(vals).cuda()
    lt = torch.from_numpy(lam).cuda()
    tuned = ws.Plan.autotuned(off, v, lt, "fp32comp", thresholds=[0, 1024, 4096], reps=2)
    ctx.check(what="autotune")
    assert tuned.threshold in (0, 1024, 4096) and len(tuned.times_ms) == 3 and min(tuned.times_ms) > 0
    assert tuned.ic_cap in (8, 16, 32, 64)   # the cap it chose (or the context's default, 32)
    a = ws.Plan(off, torch.float32).forward(v, lt, "fp32comp")
    b = tuned.forward(v, lt, "fp32comp")
    ctx.check(what="autotuned forward")
    # same exact partition whichever path a segment takes
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    assert float((a[0] - b[0]).abs().max()) <= 1e-5 * (1 + float(v.abs().max()) + float(lt.max()))


@pytest.mark.parametrize("path", ["one_cta", "device_wide"])
def test_degenerate_and_extreme_inputs(ws, ctx, path):
    """Constant vectors, sorted and reverse-sorted inputs, denormals and signed
    zeros, values spanning ~60 binades, and extreme lambdas, on both paths."""
    if path == "device_wide":
        ctx.set_small_max(0)
    rng = np.random.default_rng(77)
    d = 3000 if path == "one_cta" else 300001
    cases = []
    cases.append(("constant", np.full(d, 0.37, np.float32), (0.0, 1e-3, 10.0)))
    x = np.sort(rng.standard_normal(d)).astype(np.float32)
    cases.append(("sorted", x, (1e-2, 1.0)))
    cases.append(("reversed", x[::-1].copy(), (1e-2, 1.0)))
    den = rng.standard_normal(d).astype(np.float32)
    den[: d // 4] = (rng.integers(1, 1000, d // 4) * np.float32(1e-45)).astype(np.float32)   # denormals
    den[d // 4: d // 4 + 50] = -0.0
    cases.append(("denormals", den, (1e-30, 1e-3, 1.0)))
    wide = (rng.standard_normal(d) * 10.0 ** rng.uniform(-4, 4, d)).astype(np.float32)   # ~27 binades: 128-bit tiles
    cases.append(("wide_range", wide, (1e-3, 1e3)))
    small = rng.standard_normal(d).astype(np.float32)
    cases.append(("extreme_lambda", small, (1e-30, 1e6)))
    for name, w_np, lams in cases:
        for lam in lams:
            out, ids, nc = run_one(ws, ctx, w_np, lam, "f32", "fp64")
            compare_segment(w_np, lam, out, ids, nc, 1e-5)
            if name == "constant":
                assert nc == 1 and np.all(out == w_np[0])

    # beyond the exact domain (values spanning ~200 binades): bits below 2^-L of the
    # smallest values are dropped, so only the values and the structure of the
    # partition are checked (ids rank the clusters in value order)
    huge = (rng.standard_normal(d) * 10.0 ** rng.uniform(-30, 30, d)).astype(np.float32)
    for lam in (1e-3, 1e3):
        out, ids, nc = run_one(ws, ctx, huge, lam, "f32", "fp64")
        ref, _, _ = oracle.prox(huge, lam)
        scale = float(np.abs(huge).max()) + lam
        assert float(np.abs(out.astype(np.float64) - ref).max()) <= 1e-5 * scale
        order = np.argsort(huge, kind="stable")
        g = ids[order]
        assert g[0] == 0 and np.all(np.diff(g) >= 0) and np.all(np.diff(g) <= 1) and g[-1] == nc - 1


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("d", [37, 5001, 300001])
def test_one_signed_inputs_device_wide(ws, ctx, dt, d):
    """All-positive and all-negative vectors on the device-wide path at ragged
    sizes: lanes past a tile's end carry no element, and their placeholder
    value 0 lies outside the data range (before every cluster or after the
    last one); the device status must stay clean."""
    ctx.set_small_max(0)
    base = inputs.normal_with_duplicates(d, seed=d + 9, dtype=NP[dt])
    for shift in (6.0, -6.0):
        w_np = (base + NP[dt](shift)).astype(NP[dt])
        for lam in (1e-3, 0.5):
            out, ids, nc = run_one(ws, ctx, w_np, lam, dt, "fp64")
            compare_segment(w_np, lam, out, ids, nc, TOL[(dt, "fp64")])


@pytest.mark.parametrize("path", ["one_cta", "device_wide"])
def test_inexact_fixed_point_is_reported(ws, ctx, path):
    # values spanning more than 34 binades (FP32) are truncated in the fixed
    # point: ws_get_inexact says so; within the span it stays clear
    if path == "device_wide":
        ctx.set_small_max(0)
    ctx.inexact()   # (clear)
    w_np = inputs.normal(4000, seed=31, dtype=np.float32)
    w_np = np.where(np.abs(w_np) < 1e-3, np.float32(1e-3), w_np)   # about 12 binades
    out, ids, nc = run_one(ws, ctx, w_np, 1.0, "f32", "fp32comp")
    assert not ctx.inexact()
    wide = w_np.copy()
    wide[::7] *= np.float32(1e-30)   # now about 110 binades
    out, ids, nc = run_one(ws, ctx, wide, 1.0, "f32", "fp32comp")
    assert ctx.inexact()
    assert not ctx.inexact()   # cleared by the query
    # the outputs still meet the tolerance (values only: the partition is exact
    # for the truncated values)
    ref = oracle.prox(wide.astype(np.float64), 1.0)[0]
    assert np.abs(out.astype(np.float64) - ref).max() <= 1e-5 * (np.abs(wide).max() + 1.0)
    # FP64 segments of N(0,1) weights span more than 5 binades: reported
    run_one(ws, ctx, inputs.normal(4096, seed=32, dtype=np.float64), 0.1, "f64", "fp64")
    assert ctx.inexact()
