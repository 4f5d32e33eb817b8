"""The allocation-free backward entry point (ws_prox_backward_noalloc).

It serves callers that must not allocate device memory where the backward
runs (a framework that has pre-reserved the GPU's memory for its own pool, or a
loop that cannot take the device-wide synchronisation of cudaMalloc/cudaFree).
Its output must equal the regular
plan-based ws_prox_backward on the same inputs, on consecutive calls that
reuse the library's fixed scratch array.  This file is collected last so that
a stop-at-first-failure run has already run every other test; it also passes
alone in a fresh process.
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


@pytest.mark.parametrize("dt,np_dt,tol", [(torch.float32, np.float32, 1e-5), (torch.float64, np.float64, 1e-12)])
def test_noalloc_backward_matches_regular_backward_on_two_calls(ws, dt, np_dt, tol):
    from paper_2311_03096_gb300 import inputs
    ctx = ws.Context.get(0)
    ctx.status()
    # two calls in a row: a larger vector first, then a smaller one, so the
    # second call also shows that leftovers of the first are cleared
    for call, (d, lam) in enumerate(((300_000, 0.5), (70_000, 2.0))):
        w = torch.from_numpy(inputs.normal_with_duplicates(d, seed=100 + call, dtype=np_dt)).cuda()
        _, ids, _ = ws.prox(w, lam, "fp64")
        g = torch.from_numpy(inputs.normal(d, seed=200 + call, dtype=np_dt)).cuda()
        ref = ws.prox_backward(g, ids)
        got = torch.full_like(g, float("nan"))
        ws.prox_backward_noalloc(g, ids, got)
        ctx.check(what="no-alloc backward")
        scale = 1.0 + float(g.abs().max())
        err = float((got - ref).abs().max())
        assert err <= tol * scale, (call, err)


def test_noalloc_rejects_sizes_beyond_the_limit(ws):
    n = ws.NOALLOC_MAX_ELEMS + 1
    g = torch.zeros(n, device="cuda")
    ids = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ws.WSError) as e:
        ws.prox_backward_noalloc(g, ids, torch.empty_like(g))
    assert e.value.code == ws.WS_ERR_INVALID
