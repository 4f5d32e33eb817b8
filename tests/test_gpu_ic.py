"""The in-tile Imminent Collisions rounds of the device-wide path (appendix
algorithm "Imminent collisions algorithm (v2)", Sec. 4) with their round cap
and the fallback to the tree of bridge merges.

Whatever the cap -- 0 (every tile takes the merges), 2 (tiles that need
more than one merging round fall back), the default -- the GPU partition and
values must equal the oracle's, on the benchmark vector, the adversarial
cascade and its mirror, and the exact-tie lattice.  The per-tile outcome counts say which path ran.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2311_03096_gb300 import inputs  # noqa: E402
from parity import compare_segment, lattice_expected  # noqa: E402

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
    c.set_small_max(-1)
    c.set_ic_cap(-1)


def _run(ws, ctx, w_np, lam, cap, prec="fp32comp"):
    ctx.set_ic_cap(cap)
    w = torch.from_numpy(w_np).cuda()
    out, ids, nc = ws.prox(w, lam, prec)
    ctx.check(what="prox")
    stats = ctx.hull_stats(w_np.shape[0], w.dtype)
    return out.cpu().numpy(), ids.cpu().numpy(), int(nc.item()), stats


@pytest.mark.parametrize("lam", [1e-2, 1.0, 1e2])
def test_ic_rounds_and_fallback_match_oracle(ws, ctx, lam):
    d = (1 << 20) + 777   # many tiles and a ragged last one
    w_np = inputs.normal_with_duplicates(d, seed=3, dtype=np.float32)
    ref = oracle.prox(w_np, lam, return_perm=True)
    seen = {}
    for cap in (0, 2, -1):
        out, ids, nc, st = _run(ws, ctx, w_np, lam, cap)
        compare_segment(w_np, lam, out, ids, nc, 1e-5, ref=ref)
        seen[cap] = st
    tiles = -(-d // 4096)
    assert seen[0]["capped"] + seen[0]["general"] == tiles          # no rounds at all
    assert sum(seen[-1]["rounds"][1:]) + seen[-1]["general"] + seen[-1]["capped"] == tiles
    if lam == 1e-2:   # ties pool in round 1, round 2 confirms: no tile reaches the cap
        assert seen[-1]["capped"] == 0
    if lam == 1.0:    # clusters of tens of elements: many tiles need more than two rounds
        assert seen[2]["capped"] > 0


@pytest.mark.parametrize("shuffle", [False, True])
def test_ic_on_the_cascade(ws, ctx, shuffle):
    # Inside one tile the cascade converges in a few rounds; its d/2 rounds
    # are a property of the whole segment, where the tiles' hulls are joined
    # (here: every tile is swallowed by the one final cluster).
    d = 1 << 18
    w_np, lam = inputs.cascade(d, seed=1, shuffle=shuffle)
    ref = oracle.prox(w_np, lam, return_perm=True)
    for cap in (0, 4, -1):
        out, ids, nc, st = _run(ws, ctx, w_np, lam, cap)
        compare_segment(w_np, lam, out, ids, nc, 1e-5, ref=ref)
        assert nc == 1


def test_ic_mirror(ws, ctx):
    d = 1 << 18
    w_np, lam = inputs.mirror(d, seed=2, shuffle=True)
    ref = oracle.prox(w_np, lam, return_perm=True)
    for cap in (0, -1):
        out, ids, nc, st = _run(ws, ctx, w_np, lam, cap)
        compare_segment(w_np, lam, out, ids, nc, 1e-5, ref=ref)
        assert nc == d // 2


@pytest.mark.parametrize("binade", [True, False])
def test_ic_tie_lattice_exact(ws, ctx, binade):
    d = (1 << 18) + 5
    w_np, lam, n_idx = inputs.tie_lattice(d, seed=4, dtype=np.float32, binade=binade)
    want_ids, _, want_nc = lattice_expected(n_idx, d)
    for cap in (0, 3, -1):
        out, ids, nc, st = _run(ws, ctx, w_np, lam, cap)
        assert nc == want_nc
        assert np.array_equal(ids, want_ids)
