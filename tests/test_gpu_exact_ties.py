"""Exact ties on the GPU path: inputs on a lattice of one unit u with lambda
chosen so that the shift of Sec. 3 drops by exactly one unit per sorted
position (inputs.tie_lattice).  Then 2 (y_k - base) / u = 2 n_k + d + 1 - 2k
is an integer for every k, and pool-adjacent-violators on those integers,
pooling on >= (Sec. 4.1, ties pool), gives the partition exactly -- no
rounding anywhere, so no boundary is excused here: the GPU's cluster ids must
equal it element by element.  Steps of one unit make adjacent block means tie
exactly, the boundary case of every hull test (including the chunk
thresholds of the tile kernel).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2311_03096_gb300 import inputs  # noqa: E402
from parity import lattice_expected as expected  # noqa: E402

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
    c.set_small_max(-1)


@pytest.mark.parametrize("dt", ["f32", "f64"])
@pytest.mark.parametrize("binade", [True, False])
@pytest.mark.parametrize("d", [37, 4096, 70001, 2 ** 20])
def test_lattice_ties_exact(ws, ctx, dt, binade, d):
    npdt = np.float32 if dt == "f32" else np.float64
    w_np, lam, n = inputs.tie_lattice(d, seed=d % 97 + 3, dtype=npdt, binade=binade)
    ids_ref, half_units, nc_ref = expected(n, d)
    p = 24 if dt == "f32" else 53
    base = 1.0 if binade else 0.0
    ref = base + half_units * 2.0 ** -p
    w = torch.from_numpy(w_np).cuda()
    for prec in ("fp32comp", "fp64"):
        out, ids, nc = ws.prox(w, lam, prec, ctx=ctx)
        ctx.check(what="prox")
        assert int(nc.item()) == nc_ref
        assert np.array_equal(ids.cpu().numpy(), ids_ref)
        tol = 1e-12 if (dt == "f64" and prec == "fp64") else 1e-5
        err = np.abs(out.cpu().numpy().astype(np.float64) - ref).max()
        assert err <= tol * (np.abs(w_np).max() + lam)
    # the same through the device-wide path at sizes the one-CTA kernel would take
    if d <= 4096:
        ctx.set_small_max(0)
        out, ids, nc = ws.prox(w, lam, "fp32comp", ctx=ctx)
        ctx.check(what="prox (device-wide)")
        ctx.set_small_max(-1)
        assert np.array_equal(ids.cpu().numpy(), ids_ref)


def test_lattice_ties_batched(ws, ctx):
    rng = np.random.default_rng(5)
    lens = rng.integers(0, 9000, 24)
    lens[:4] = [0, 1, 4096, 20000]
    vals, lams, ns = [], [], []
    for i, L in enumerate(lens):
        w_i, lam_i, n_i = inputs.tie_lattice(int(L), seed=100 + i, binade=bool(i % 2))
        vals.append(w_i); lams.append(lam_i if L > 1 else 0.5); ns.append(n_i)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    plan = ws.Plan(off, torch.float32)
    out, ids, nc = plan.forward(torch.from_numpy(np.concatenate(vals)).cuda(), torch.tensor(lams, dtype=torch.float64).cuda(), "fp32comp")
    ctx.check(what="batched")
    ids = ids.cpu().numpy()
    nc = nc.cpu().numpy()
    for i, L in enumerate(lens):
        if L < 2:
            continue
        ids_ref, _, nc_ref = expected(ns[i], int(L))
        assert nc[i] == nc_ref
        assert np.array_equal(ids[off[i]:off[i + 1]], ids_ref)
