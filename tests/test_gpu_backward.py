"""The backward (cluster-mean Jacobian, partition held fixed) on the device-wide
path at full size, and its exactness: the cluster sums are exact integers at
a per-segment scale, so the result is deterministic (bit-identical across
calls and across any order of the additions) and its error does not grow
with the cluster size -- one huge cluster (lambda = 1e2) included.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2311_03096_gb300 import inputs  # noqa: E402

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
    c.status()
    yield c
    c.set_small_max(-1)


@pytest.mark.parametrize("lam", [1e-2, 1e2])
@pytest.mark.parametrize("dt,np_dt,tol,d", [(torch.float32, np.float32, 1e-5, 1 << 24),
                                            (torch.float64, np.float64, 1e-12, 1 << 22)])
def test_large_backward_matches_oracle(ws, ctx, lam, dt, np_dt, tol, d):
    w = torch.from_numpy(inputs.normal_with_duplicates(d, seed=21, dtype=np_dt)).cuda()
    _, ids, nc = ws.prox(w, lam, "fp64")
    if lam == 1e2:
        assert int(nc.item()) == 1
    g_np = inputs.normal(d, seed=22, dtype=np_dt)
    g = torch.from_numpy(g_np).cuda()
    gin = ws.prox_backward(g, ids)
    ctx.check(what="backward")
    ref = oracle.backward(g_np, ids.cpu().numpy())
    err = float(np.abs(gin.cpu().numpy().astype(np.float64) - ref).max())
    assert err <= tol * (1.0 + float(np.abs(ref).max())), err


def test_backward_is_deterministic(ws, ctx):
    d = (1 << 22) + 123
    w = torch.from_numpy(inputs.normal_with_duplicates(d, seed=23, dtype=np.float32)).cuda()
    for lam in (1.0, 1e2):
        _, ids, _ = ws.prox(w, lam)
        g = torch.from_numpy(inputs.normal(d, seed=24, dtype=np.float32)).cuda()
        a = ws.prox_backward(g, ids).clone()
        b = ws.prox_backward(g, ids).clone()
        # the same values in another order within every cluster: same sums, same means
        perm = torch.argsort(ids.long() * (d + 1) + torch.randperm(d, device="cuda"))
        order = torch.argsort(ids.long(), stable=True)
        g2 = g.clone()
        g2[order] = g[perm]   # values permuted among positions of equal id
        c = ws.prox_backward(g2, ids)
        ctx.check(what="backward")
        assert torch.equal(a, b)
        assert torch.equal(a, c)


@pytest.mark.parametrize("small", [True, False])
def test_backward_cancellation_is_exact(ws, ctx, small):
    # one cluster per segment (lambda far above the collapse threshold); grad_out
    # holds +-2^40 pairs and a few ones: the mean is exactly (number of ones)/n
    n_seg, n = 8, 3000
    off = np.arange(n_seg + 1, dtype=np.int64) * n
    vals = inputs.normal(n_seg * n, seed=25, dtype=np.float32)
    if not small:
        ctx.set_small_max(0)
    plan = ws.Plan(off, torch.float32)
    lam = torch.full((n_seg,), 1e4, dtype=torch.float64, device="cuda")
    _, ids, nc = plan.forward(torch.from_numpy(vals).cuda(), lam)
    assert np.all(nc.cpu().numpy() == 1)
    g = np.zeros(n_seg * n, np.float32)
    rng = np.random.default_rng(26)
    for s in range(n_seg):
        idx = rng.permutation(n) + s * n
        g[idx[: n // 2 - 10: 2]] = 2.0 ** 40
        g[idx[1: n // 2 - 10: 2]] = -(2.0 ** 40)
        g[idx[n // 2: n // 2 + 3 + s]] = 1.0
    gin = plan.backward(torch.from_numpy(g).cuda(), ids).cpu().numpy()
    ctx.check(what="backward")
    for s in range(n_seg):
        want = np.float32(3 + s) / np.float32(n)   # one correctly rounded FP32 division
        assert np.all(gin[s * n:(s + 1) * n] == want), (s, gin[s * n], want)


@pytest.mark.parametrize("dt,np_dt", [(torch.float32, np.float32), (torch.float64, np.float64)])
def test_backward_exact_sums_scattered_clusters(ws, ctx, dt, np_dt):
    # ids chosen by hand (the backward holds any partition fixed): cluster c
    # holds every element i = c (mod 1000), so every tile mixes a thousand
    # clusters and the sums go through the bucketed pairs, with warps adding
    # neighbours of one cluster together.  grad_out: +-2^40 pairs in every
    # cluster and, where the cluster size is odd, one small integer c mod 7 in
    # place of the unpaired +2^40; each sum is exactly that integer.
    d, ncl = (1 << 22) + 77, 1000
    i = np.arange(d)
    c, k = i % ncl, i // ncl
    size = (d - np.arange(ncl) + ncl - 1) // ncl
    g = np.where(k % 2 == 0, 2.0 ** 40, -(2.0 ** 40)).astype(np_dt)
    last_odd = (k == size[c] - 1) & (size[c] % 2 == 1)
    g[last_odd] = (c[last_odd] % 7).astype(np_dt)
    ids = c.astype(np.int32)
    gin = ws.prox_backward(torch.from_numpy(g).cuda(), torch.from_numpy(ids).cuda()).cpu().numpy()
    ctx.check(what="backward")
    tot = np.where(size % 2 == 1, np.arange(ncl) % 7, 0)
    if dt == torch.float32:
        want = (tot.astype(np.float32) / size.astype(np.float32))[c]   # one correctly rounded division
        assert np.array_equal(gin, want)
    else:
        want = (tot / size)[c]
        assert np.all(np.abs(gin - want) <= 1e-12 * np.abs(want))
