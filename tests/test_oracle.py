"""Pins for the FP64 CPU oracle (no GPU).

The oracle (oracle/ws_oracle.c) is checked against things the paper and the
mathematics fix, none of which re-run the oracle's own algorithm:
brute-force minimisation over ordered partitions, the subgradient optimality
certificate (Eq. prox_opt + Eq. subdiff_R), the textbook min-max formula of
isotonic regression, printed worked examples, closed forms, Prop. 3.2 / 4.1,
Cor. D.5, and the worst-case generators of Sec. 4.1.
"""
import os

import numpy as np
import pytest

import oracle
import pins
from paper_2311_03096_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    kv = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            kv[k] = [float(t) for t in v]
    return kv


def test_kearsley_worked_example():
    kv = _read_kv("kearsley.txt")
    lam = kv["lambda"][0]
    w = np.array(kv["w"])
    # the fixture's y is w plus the shift of Alg. 2
    np.testing.assert_allclose(w + lam * pins.shift_coefficients(4), kv["y"], atol=1e-15)
    out, ids, nc = oracle.prox(w, lam)
    np.testing.assert_allclose(out, kv["out"], atol=1e-15)
    assert ids.tolist() == [int(t) for t in kv["ids"]]
    assert nc == 3


def test_hyperplanes_d3_example():
    rows, printed = [], []
    with open(os.path.join(GOLDEN, "hyperplanes_d3.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "set":
                printed.append(tuple(int(t) for t in parts[1:]))
            else:
                order = [int(t) - 1 for t in parts[0].split(",")]
                rows.append((order, [int(t) for t in parts[1:]]))
    rng = np.random.default_rng(3)
    for _ in range(50):
        w = rng.standard_normal(3)
        for order, c in rows:
            assert pins.hyperplane(w, order) == pytest.approx(float(np.dot(c, w)), abs=1e-14)
        r_eq1 = pins.R_pairs_py(list(w))
        assert oracle.R_pairs(w) == pytest.approx(r_eq1, abs=1e-14)
        assert max(float(np.dot(c, w)) for c in printed) == pytest.approx(r_eq1, abs=1e-14)
        # the maximising hyperplanes are exactly those of sorting permutations (Sec. 2)
        srt = list(np.argsort(w))
        best = max(rows, key=lambda oc: float(np.dot(oc[1], w)))
        assert best[0] == srt
    assert sorted(printed) == sorted(tuple(c) for _, c in rows)


@pytest.mark.parametrize("d", [2, 3, 5, 17, 200])
def test_R_sorted_form_matches_definition(d):
    rng = np.random.default_rng(d)
    w = rng.standard_normal(d)
    w[: d // 3] = w[0]  # ties
    ref = pins.R_pairs_py(list(w))
    assert oracle.R_pairs(w) == pytest.approx(ref, rel=1e-12, abs=1e-12)
    assert oracle.R_sorted(w) == pytest.approx(ref, rel=1e-12, abs=1e-12)


def _small_cases():
    rng = np.random.default_rng(11)
    cases = []
    for d in range(1, 7):
        for lam in (0.0, 0.05, 0.3, 1.0, 10.0):
            cases.append((rng.standard_normal(d), lam))
            w = np.round(rng.standard_normal(d), 1)  # frequent exact ties
            cases.append((w, lam))
    return cases


@pytest.mark.parametrize("w,lam", _small_cases())
def test_brute_force_small(w, lam):
    u_bf, _ = pins.brute_force_prox(list(w), lam)
    out, ids, nc = oracle.prox(w, lam)
    np.testing.assert_allclose(out, u_bf, atol=1e-10)
    # the partition: each cluster is a level set of the output; two clusters
    # may share a value only on a near-tie (real-valued equal means that
    # rounding separates), and the exact rational PAV of the same FP inputs
    # gives the same partition
    order = np.argsort(out, kind="stable")
    assert np.all(np.diff(ids[order]) >= 0)
    for c in range(nc):
        assert np.ptp(out[ids == c]) == 0.0
    _, exact_ids = pins.exact_prox_fraction(list(w), lam)
    assert ids.tolist() == exact_ids


def test_brute_force_d7():
    rng = np.random.default_rng(7)
    w = rng.standard_normal(7)
    for lam in (0.2, 1.5):
        u_bf, _ = pins.brute_force_prox(list(w), lam)
        out, _, _ = oracle.prox(w, lam)
        np.testing.assert_allclose(out, u_bf, atol=1e-10)


def test_d2_closed_form():
    rng = np.random.default_rng(2)
    for _ in range(200):
        w = rng.standard_normal(2) * 3
        lam = float(rng.uniform(0, 3))
        out, ids, nc = oracle.prox(w, lam)
        lo, hi = (0, 1) if w[0] <= w[1] else (1, 0)
        if w[hi] - w[lo] > 2 * lam:
            exp = np.empty(2)
            exp[lo], exp[hi] = w[lo] + lam, w[hi] - lam
            assert nc == 2
        else:
            exp = np.full(2, w.mean())
            assert nc == 1
        np.testing.assert_allclose(out, exp, atol=1e-14)


@pytest.mark.parametrize("d,lam", [(10, 0.1), (64, 0.5), (257, 0.02), (1000, 1.0), (1000, 0.001)])
def test_optimality_certificate(d, lam):
    rng = np.random.default_rng(d)
    w = np.round(rng.standard_normal(d), 2)
    out, _, _ = oracle.prox(w, lam)
    assert pins.certificate_residual(w, out, lam) < 1e-9
    # a perturbed output fails the certificate
    bad = out.copy()
    bad[rng.integers(d)] += 1e-3
    assert pins.certificate_residual(w, bad, lam) > 1e-6


def test_certificate_rejects_plausible_mistakes():
    """The pins catch the mistakes an implementation could plausibly make:
    the opposite sign of the shift, a 0-based range(d) and a dropped 1/(d-1)."""
    rng = np.random.default_rng(5)
    d, lam = 50, 0.4
    w = rng.standard_normal(d)
    out, _, _ = oracle.prox(w, lam)
    assert pins.certificate_residual(w, out, lam) < 1e-9
    x = np.sort(w)
    order = np.argsort(w, kind="stable")
    k = np.arange(1, d + 1)
    wrong = {
        "minus sign": x - lam * (d + 1 - 2 * k) / (d - 1),
        "0-based range": x + lam * (d + 1 - 2 * (k - 1)) / (d - 1),
        "no 1/(d-1)": x + lam * (d + 1 - 2 * k),
    }
    for name, y in wrong.items():
        u = np.empty(d)
        u[order] = pins.isotonic_minmax(y)
        assert pins.certificate_residual(w, u, lam) > 1e-3, name


@pytest.mark.parametrize("d", [8, 50, 200])
def test_isotonic_minmax_formula(d):
    rng = np.random.default_rng(d + 1)
    w = rng.standard_normal(d)
    for lam in (0.0, 0.1, 2.0):
        out, _, _, perm, xs = oracle.prox(w, lam, return_perm=True)
        y = xs + lam * pins.shift_coefficients(d)
        np.testing.assert_allclose(out[perm], pins.isotonic_minmax(y), atol=1e-12)


def test_invariants():
    rng = np.random.default_rng(9)
    for d in (2, 3, 100, 4096):
        w = inputs.normal_with_duplicates(d, seed=d).astype(np.float64)
        for lam in (0.0, 0.1, 1.0, 1000.0):
            out, ids, nc, perm, xs = oracle.prox(w, lam, return_perm=True)
            # Prop. 3.2: momentum is conserved, so the mean is preserved
            assert out.mean() == pytest.approx(w.mean(), abs=1e-12 * (1 + abs(w).max() + lam))
            # particles never cross (Sec. 4.2 item 1): output non-decreasing in sorted order
            assert np.all(np.diff(out[perm]) >= 0)
            assert np.all(np.diff(ids[perm]) >= 0) and ids[perm][0] == 0 and ids[perm][-1] == nc - 1
            if lam == 0.0:
                np.testing.assert_array_equal(out, w)
                assert nc == len(np.unique(w))
            lo, hi = pins.prop41_extremes(xs, lam)
            assert out.min() == pytest.approx(lo, abs=1e-12 * (1 + lam))
            assert out.max() == pytest.approx(hi, abs=1e-12 * (1 + lam))
        lam_max = pins.collapse_threshold(np.sort(w))
        assert oracle.prox(w, lam_max * (1 + 1e-9) + 1e-12)[2] == 1
        if lam_max > 1e-9:
            assert oracle.prox(w, lam_max * (1 - 1e-6))[2] > 1


def test_neighbour_collision_corollary():
    rng = np.random.default_rng(12)
    for d, lam in ((30, 0.2), (300, 0.05), (300, 3.0)):
        w = np.round(rng.standard_normal(d), 2)
        out, ids, nc, perm, xs = oracle.prox(w, lam, return_perm=True)
        for k in range(d - 1):
            s = oracle.neighbour_slack(xs, lam, k)
            same = ids[perm[k]] == ids[perm[k + 1]]
            if abs(s) > 1e-12:
                assert same == (s >= 0), (d, lam, k, s)


def test_sort_total_order_and_stability():
    w = np.array([1.0, -0.0, 0.0, -1.0, 1.0, 0.0, -0.0])
    perm, xs = oracle.sort(w)
    assert perm.tolist() == [3, 1, 6, 2, 5, 0, 4]


@pytest.mark.parametrize("d", [2 ** 10, 2 ** 12, 2 ** 16])
def test_cascade_generator(d):
    """Sec. 4.1 worst case: everything merges into one cluster (merge count d-1),
    and it takes about d/2 imminent-collision rounds (checked by a direct
    simulation of Alg. 3's rounds for the smaller sizes)."""
    w, lam = inputs.cascade(d)
    out, ids, nc = oracle.prox(w, lam)
    assert nc == 1
    ws, lam2 = inputs.cascade(d, shuffle=True)
    assert oracle.prox(ws, lam2)[2] == 1
    if d <= 2 ** 12:
        assert _ic_v2_rounds(np.sort(w.astype(np.float64)), lam) >= d // 2


def _ic_v2_rounds(x, lam):
    """Rounds of Alg. 3 (imminent collisions v2) on sorted x: a new cluster
    starts where y[i-1] < y[i]; each round pools every maximal violating run."""
    d = x.shape[0]
    s = x + lam * pins.shift_coefficients(d)  # y per particle
    m = np.ones(d)
    ysum = s.copy()
    rounds = 0
    while True:
        y = ysum / m
        start = np.concatenate([[True], y[:-1] < y[1:]])
        blk = np.cumsum(start) - 1
        nb = blk[-1] + 1
        rounds += 1
        if nb == y.shape[0]:
            return rounds
        ysum = np.bincount(blk, weights=ysum, minlength=nb)
        m = np.bincount(blk, weights=m, minlength=nb)


@pytest.mark.parametrize("d", [2 ** 10, 2 ** 16])
def test_mirror_generator(d):
    w, lam = inputs.mirror(d, shuffle=True)
    out, ids, nc = oracle.prox(w, lam)
    assert nc == d // 2
    assert np.all(np.bincount(ids) == 2)


@pytest.mark.parametrize("binade", [True, False])
@pytest.mark.parametrize("d", [37, 4096, 70001])
def test_tie_lattice_matches_integer_pav(d, binade):
    # exact ties everywhere (steps of one unit tie adjacent block means); for
    # float inputs every y and every block sum is exact in FP64, so the oracle
    # must pool exactly where integer PAV with >= pooling does (Sec. 4.1)
    from parity import lattice_expected
    w, lam, n = inputs.tie_lattice(d, seed=d % 97 + 3, binade=binade)
    ids_ref, means, nc_ref = lattice_expected(n, d)
    out, ids, nc = oracle.prox(w, lam)
    assert nc == nc_ref
    assert np.array_equal(ids, ids_ref)
    np.testing.assert_array_equal(out, (1.0 if binade else 0.0) + means * 2.0 ** -24)


@pytest.mark.parametrize("lam", [0.0, 1e-2, 0.3, 1.0, 100.0])
def test_ic_v2_converges_to_the_prox_partition(lam):
    # IC v2 (appendix algorithm) only performs collisions that happen, and stops
    # when no destination order is violated: its blocks are the prox clusters
    w = inputs.normal_with_duplicates(5000, seed=11)
    out, ids, nc, rounds, conv = oracle.imminent_collisions_v2(w, lam)
    pout, pids, pnc = oracle.prox(w, lam)
    assert conv and nc == pnc and np.array_equal(ids, pids)
    np.testing.assert_allclose(out, pout, atol=1e-12 * (np.abs(w).max() + lam))


def test_ic_v2_on_tie_lattice_is_exact():
    from parity import lattice_expected
    w, lam, n = inputs.tie_lattice(4096, seed=8)
    ids_ref, _, nc_ref = lattice_expected(n, 4096)
    _, ids, nc, _, conv = oracle.imminent_collisions_v2(w, lam)
    assert conv and nc == nc_ref and np.array_equal(ids, ids_ref)


@pytest.mark.parametrize("d", [16, 1024, 4096])
def test_ic_v2_round_counts(d):
    # Sec. 4.1: on the cascade the right half joins one particle per round, d/2
    # rounds; plus the round that pools the left half and the final round that
    # changes nothing.  The mirror pools every pair in one round.
    w, lam = inputs.cascade(d, seed=1)
    _, _, nc, rounds, conv = oracle.imminent_collisions_v2(w, lam)
    assert conv and nc == 1 and rounds == d // 2 + 2
    w, lam = inputs.mirror(d, seed=2, shuffle=True)
    _, _, nc, rounds, conv = oracle.imminent_collisions_v2(w, lam)
    assert conv and nc == d // 2 and rounds == 2


def test_ic_v2_round_cap_gives_a_refinement():
    # stopped early, every block still lies inside one prox cluster
    w, lam = inputs.cascade(1024, seed=1, shuffle=True)
    _, ids, nc, rounds, conv = oracle.imminent_collisions_v2(w, lam, max_rounds=20)
    assert rounds == 20 and not conv and nc > 1
    _, pids, _ = oracle.prox(w, lam)
    for b in np.unique(ids):
        assert np.unique(pids[ids == b]).shape[0] == 1


def test_backward_is_cluster_average_and_matches_fd():
    rng = np.random.default_rng(4)
    d, lam, eps = 64, 0.05, 1e-6
    w = rng.standard_normal(d)
    out, ids, nc = oracle.prox(w, lam)
    assert 1 < nc < d
    g = rng.standard_normal(d)
    gin = oracle.backward(g, ids)
    for c in range(nc):
        m = ids == c
        np.testing.assert_allclose(gin[m], g[m].mean(), atol=1e-14)
    # central finite differences of <g, prox(w)>
    fd = np.empty(d)
    for i in range(d):
        e = np.zeros(d)
        e[i] = eps
        fd[i] = (g @ oracle.prox(w + e, lam)[0] - g @ oracle.prox(w - e, lam)[0]) / (2 * eps)
    np.testing.assert_allclose(fd, gin, atol=1e-6)


def test_batched_equals_per_segment():
    rng = np.random.default_rng(8)
    lens = [0, 1, 2, 7, 100, 33]
    parts = [rng.standard_normal(n) for n in lens]
    off = np.concatenate([[0], np.cumsum(lens)])
    lam = rng.uniform(0, 1, len(lens))
    out, ids, nc = oracle.prox_batched(np.concatenate(parts), off, lam)
    for s, p in enumerate(parts):
        o, i, n = oracle.prox(p, lam[s])
        np.testing.assert_array_equal(out[off[s]:off[s + 1]], o)
        np.testing.assert_array_equal(ids[off[s]:off[s + 1]], i)
        assert nc[s] == n


def test_exact_rational_partition_agrees():
    rng = np.random.default_rng(21)
    for d in (3, 10, 40):
        for lam in (0.01, 0.3):
            w = np.round(rng.standard_normal(d), 1)
            ref, ref_ids = pins.exact_prox_fraction(list(w), lam)
            out, ids, _ = oracle.prox(w, lam)
            assert ids.tolist() == ref_ids
            np.testing.assert_allclose(out, [float(v) for v in ref], atol=1e-14)


def test_error_paths():
    with pytest.raises(oracle.OracleError):
        oracle.prox(np.array([1.0, np.nan]), 0.1)
    with pytest.raises(oracle.OracleError):
        oracle.prox(np.array([1.0, np.inf]), 0.1)
    with pytest.raises(oracle.OracleError):
        oracle.prox(np.array([1.0, 2.0]), -0.1)
    out, ids, nc = oracle.prox(np.zeros(0), 0.1)
    assert nc == 0
    out, ids, nc = oracle.prox(np.array([3.5]), 10.0)
    assert out.tolist() == [3.5] and ids.tolist() == [0] and nc == 1


# -- weight sharing + l1 with rewinding (Rewinding section, Alg. 2) ----------

def test_l1_rewind_reduces_to_prox_when_beta_zero():
    rng = np.random.default_rng(31)
    for d in (1, 2, 7, 500):
        w = rng.standard_normal(d)
        for lam in (0.0, 0.05, 1.0):
            ref, rid, rn = oracle.prox(w, lam)
            out, ids, nc = oracle.prox_l1(w, lam, 0.0, 0.0)
            assert nc == rn and np.array_equal(ids, rid)
            np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * (1 + np.abs(w).max() + lam))


def test_l1_rewind_without_sharing_is_eq_rewinding_l1():
    # alpha = 0: every cluster is one value, and Alg. 2 reduces to the closed form
    # (w - (1 - rho) beta sign(w)) [|w| > beta] of Eq. rewinding_l1 (no |w| == beta ties here)
    rng = np.random.default_rng(32)
    w = rng.standard_normal(2000)
    for beta in (0.0, 0.3, 1.5):
        for rho in (0.0, 0.25, 1.0):
            out, _, _ = oracle.prox_l1(w, 0.0, beta, rho)
            expect = np.where(np.abs(w) > beta, w - (1 - rho) * beta * np.sign(w), 0.0)
            np.testing.assert_allclose(out, expect, rtol=0, atol=1e-15)


def test_l1_rewind_rho0_is_soft_threshold_of_prox():
    # Prop. D.6: prox of alpha R + beta l1 = soft-thresholding of prox of alpha R
    rng = np.random.default_rng(33)
    for d in (3, 64, 3000):
        w = rng.standard_normal(d)
        for lam in (0.01, 0.4, 3.0):
            p, pid, _ = oracle.prox(w, lam)
            for beta in (0.05, 0.5):
                out, ids, _ = oracle.prox_l1(w, lam, beta, 0.0)
                assert np.array_equal(ids, pid)
                st = np.sign(p) * np.maximum(np.abs(p) - beta, 0.0)
                np.testing.assert_allclose(out, st, rtol=0, atol=1e-12 * (1 + np.abs(w).max() + lam))


def test_l1_rewind_rho1_keeps_cluster_means():
    # rho = 1 removes the whole remaining displacement: surviving clusters sit at
    # the mean of their weights, the others at 0
    rng = np.random.default_rng(34)
    w = rng.standard_normal(1500)
    lam, beta = 0.7, 0.2
    p, pid, nc = oracle.prox(w, lam)
    out, ids, _ = oracle.prox_l1(w, lam, beta, 1.0)
    mean = np.bincount(ids, weights=w, minlength=nc) / np.bincount(ids, minlength=nc)
    keep = np.abs(p) >= beta
    np.testing.assert_allclose(out[keep], mean[ids][keep], rtol=0, atol=1e-12)
    assert np.all(out[~keep] == 0.0)


def test_l1_rewind_is_affine_in_the_displacement_scale():
    rng = np.random.default_rng(35)
    w = rng.standard_normal(800)
    lam, beta, rho = 0.3, 0.1, 0.4
    a = oracle.prox_l1(w, lam, beta, rho, 0.0)[0]
    b = oracle.prox_l1(w, lam, beta, rho, 1.0)[0]
    h = oracle.prox_l1(w, lam, beta, rho, 0.5)[0]
    np.testing.assert_allclose(h, 0.5 * (a + b), rtol=0, atol=1e-13)


def test_l1_rewind_rejects_bad_arguments():
    w = np.zeros(4)
    for args in ((-1.0, 0.0), (0.1, -0.5), (0.1, 1.5), (0.1, float("nan"))):
        with pytest.raises(oracle.OracleError):
            oracle.prox_l1(w, 0.1, args[0], args[1])


# -- weight-sharing measure (CIFAR10 experiment) ----------------------------

def test_ws_measure_definition():
    assert oracle.ws_measure([0.0, -0.0, 1.0, 1.0, 2.0, -3.0]) == 3 / 4
    assert oracle.ws_measure([0.0, 0.0]) == 0.0
    assert oracle.ws_measure([5.0] * 10) == 0.1
    rng = np.random.default_rng(41)
    w = rng.standard_normal(1000)
    assert oracle.ws_measure(w) == 1.0
    assert oracle.ws_measure(rng.permutation(np.repeat(w[:10], 7))) == 10 / 70
    out, _, nc = oracle.prox(w, 2.0)
    assert oracle.ws_measure(out) == nc / np.count_nonzero(out)


# -- d prox / d lambda (partition held fixed) ------------------------------

def test_dlambda_matches_central_fd():
    rng = np.random.default_rng(51)
    for d, lam in ((2, 0.3), (64, 0.05), (500, 0.5), (3000, 2.0)):
        w = rng.standard_normal(d)
        g = rng.standard_normal(d)
        out, ids, _ = oracle.prox(w, lam)
        eps = 1e-7
        ip, _, _ = oracle.prox(w, lam + eps)
        im, _, _ = oracle.prox(w, lam - eps)
        assert np.array_equal(oracle.prox(w, lam + eps)[1], ids) and np.array_equal(oracle.prox(w, lam - eps)[1], ids)
        fd = (g @ ip - g @ im) / (2 * eps)
        got = oracle.dlambda(g, ids)[0]
        assert abs(got - fd) <= 1e-6 * (1 + abs(fd))


def test_dlambda_batched_and_trivial_segments():
    rng = np.random.default_rng(52)
    lens = [0, 1, 5, 40]
    off = np.concatenate([[0], np.cumsum(lens)])
    w = rng.standard_normal(off[-1])
    lam = np.array([0.1, 0.2, 0.3, 0.4])
    out, ids, _ = oracle.prox_batched(w, off, lam)
    g = rng.standard_normal(off[-1])
    res = oracle.dlambda(g, ids, off)
    assert res[0] == 0.0 and res[1] == 0.0
    for s in (2, 3):
        a, b = off[s], off[s + 1]
        assert res[s] == oracle.dlambda(g[a:b], ids[a:b])[0]
    # one cluster: every position moves with the mean velocity, which is 0
    w1 = np.zeros(7)
    o1, i1, n1 = oracle.prox(w1, 1.0)
    assert n1 == 1 and abs(oracle.dlambda(rng.standard_normal(7), i1)[0]) < 1e-15
