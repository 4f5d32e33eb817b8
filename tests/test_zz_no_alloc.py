"""The allocation-free backward entry point (ws_prox_backward_noalloc).

It serves callers that must not allocate device memory where the backward
runs (a framework that has pre-reserved the GPU's memory for its own pool, or a
loop that cannot take the device-wide synchronisation of cudaMalloc/cudaFree).
Its output must equal the regular
plan-based ws_prox_backward on the same inputs, on consecutive calls that
reuse the library's fixed scratch array.  This file is collected last so that
a stop-at-first-failure run has already run every other test; it also passes
alone in a fresh process.  The entry point writes no status word, so these
tests rely on its return code and on the values it writes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ws():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2311_03096_gb300 import ws as _ws
    return _ws


def _case(ws, d, lam, seed, np_dt):
    from paper_2311_03096_gb300 import inputs
    w = torch.from_numpy(inputs.normal_with_duplicates(d, seed=seed, dtype=np_dt)).cuda()
    _, ids, _ = ws.prox(w, lam, "fp64")
    g = torch.from_numpy(inputs.normal(d, seed=seed + 100, dtype=np_dt)).cuda()
    return g, ids


@pytest.mark.parametrize("dt,np_dt,tol", [(torch.float32, np.float32, 1e-5), (torch.float64, np.float64, 1e-12)])
def test_noalloc_backward_matches_regular_backward_on_two_calls(ws, dt, np_dt, tol):
    # two calls in a row: a larger vector first, then a smaller one, so the
    # second call also shows that leftovers of the first are cleared
    for call, (d, lam) in enumerate(((300_000, 0.5), (70_000, 2.0))):
        g, ids = _case(ws, d, lam, 100 + call, np_dt)
        ref = ws.prox_backward(g, ids)
        got = torch.full_like(g, float("nan"))
        ws.prox_backward_noalloc(g, ids, got)
        torch.cuda.synchronize()
        scale = 1.0 + float(g.abs().max())
        err = float((got - ref).abs().max())
        assert err <= tol * scale, (call, err)


def test_noalloc_at_the_size_limit_and_aliased(ws):
    d = ws.NOALLOC_MAX_ELEMS
    g, ids = _case(ws, d, 0.3, 7, np.float32)
    ref = ws.prox_backward(g, ids)
    got = torch.full_like(g, float("nan"))
    ws.prox_backward_noalloc(g, ids, got)
    # grad_in may be grad_out itself
    alias = g.clone()
    ws.prox_backward_noalloc(alias, ids, alias)
    torch.cuda.synchronize()
    scale = 1.0 + float(g.abs().max())
    assert float((got - ref).abs().max()) <= 1e-5 * scale
    assert float((alias - ref).abs().max()) <= 1e-5 * scale


def test_noalloc_skips_out_of_range_ids(ws):
    d = 50_000
    g, ids = _case(ws, d, 0.2, 11, np.float64)
    bad = torch.tensor([0, 17, 4096, d - 1], device="cuda")
    ids = ids.clone()
    ids[bad[:2]] = -1
    ids[bad[2:]] = d
    got = torch.full_like(g, 123.0)
    ws.prox_backward_noalloc(g, ids, got)
    torch.cuda.synchronize()
    g_h, ids_h, got_h = g.cpu().numpy(), ids.cpu().numpy(), got.cpu().numpy()
    ok = (ids_h >= 0) & (ids_h < d)
    sums = np.bincount(ids_h[ok], weights=g_h[ok], minlength=d)
    cnts = np.bincount(ids_h[ok], minlength=d)
    want = sums[ids_h[ok]] / cnts[ids_h[ok]]
    assert np.all(got_h[~ok] == 123.0)
    assert np.max(np.abs(got_h[ok] - want)) <= 1e-12 * (1.0 + np.abs(g_h).max())


def test_noalloc_call_allocates_nothing(ws):
    g, ids = _case(ws, 200_000, 1.0, 13, np.float32)
    got = torch.empty_like(g)
    ws.prox_backward_noalloc(g, ids, got)   # warm-up: the module is loaded by now
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        ws.prox_backward_noalloc(g, ids, got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_the_limit(ws):
    n = ws.NOALLOC_MAX_ELEMS + 1
    g = torch.zeros(n, device="cuda")
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ws.WSError) as e:
        ws.prox_backward_noalloc(g, ids, torch.empty_like(g))
    assert e.value.code == ws.WS_ERR_INVALID


def test_noalloc_binding_rejects_mismatched_tensors(ws):
    g = torch.zeros(100, device="cuda")
    ids = torch.zeros(100, dtype=torch.int32, device="cuda")
    with pytest.raises(ValueError):
        ws.prox_backward_noalloc(g, ids[:99], torch.empty_like(g))
    with pytest.raises(ValueError):
        ws.prox_backward_noalloc(g, ids.long(), torch.empty_like(g))
    with pytest.raises(ValueError):
        ws.prox_backward_noalloc(g, ids, torch.empty(100, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        ws.prox_backward_noalloc(g, ids, torch.empty(99, device="cuda"))
