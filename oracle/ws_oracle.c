/*
 * ws_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the proximal
 * map of the weight-sharing penalty (arXiv 2311.03096).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library under paper_2311_03096_gb300/) never calls, links or
 * includes anything here, and nothing here is shared with it.
 *
 * What it computes (all in IEEE binary64, round-to-nearest):
 *
 *   R(w)       = 1/(d-1) * sum_{i>j} |w_i - w_j|                      Eq. (1)
 *   prox(w)    = argmin_u  lambda*R(u) + 1/2 ||u - w||^2              Sec. 1, prox definition
 *
 * reached the way the paper describes it:
 *   1. x, perm = sort(w) ascending, ties broken by original index (stable).
 *      Sorting is the pre-processing all algorithms assume (Sec. 4, first
 *      paragraph; Alg. 2 "sort").
 *   2. v_k = lambda*(d + 1 - 2k)/(d - 1), k = 1..d  (Alg. 2: the velocity,
 *      i.e. -lambda * grad R at the sorted point; Sec. 3 particle model),
 *      y = x + v (Sec. 3: particle destinations without collisions).
 *   3. prox in sorted order = isotonic regression of y (Sec. 3, last
 *      paragraph; Eq. iso_regr), computed with the sequential pool adjacent
 *      violators algorithm the paper names in Sec. 4.1: a stack of blocks,
 *      two neighbours are pooled whenever mean(left) >= mean(right)
 *      (a collision is detected when y_i >= y_{i+1}, Sec. 4.1).  The paper's
 *      remark that the order of collisions does not matter (collision is
 *      associative, Sec. 4.1) is what makes the stack order valid.
 *   4. cluster r = r-th pooled block, value = mean of y over the block,
 *      out[perm[k]] = value(block of k), ids[perm[k]] = r  (Alg. 2:
 *      repeat_interleave then scatter by sort_indices).
 *
 * Readings where the paper is silent:
 *   - ties in the merge pool on ">=" (text of Sec. 4.1), so clusters are
 *     maximal runs of equal prox values;
 *   - the sort key is the IEEE-754 total order of binary64 (so -0 < +0), ties
 *     broken by index; NaN/Inf inputs are rejected (return code 2);
 *   - d = 1 returns w unchanged with a single cluster (1/(d-1) is vacuous);
 *   - block sums are carried as an unevaluated pair (s, c) with Neumaier's
 *     compensated summation (Neumaier 1974), so the rounding error of a block
 *     mean stays at a few ulps of the mean no matter how many particles were
 *     pooled; the pooling test compares the two FP64 block means.
 *
 * Backward (Jacobian-vector product with the partition held fixed): the
 * gradient of an output value with respect to every input of its cluster is
 * 1/|cluster|, so grad_in[i] = mean of grad_out over the cluster of i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Sorting: IEEE total order key, stable by index.                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    int64_t idx;
} key_idx;

static uint64_t total_order_key(double v) {
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    /* negative numbers: flip all bits; non-negative: flip the sign bit */
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

static int cmp_key_idx(const void* pa, const void* pb) {
    const key_idx* a = (const key_idx*)pa;
    const key_idx* b = (const key_idx*)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    if (a->idx < b->idx) return -1;
    if (a->idx > b->idx) return 1;
    return 0;
}

/* Sorted permutation of w: perm[k] = index of the k-th smallest (0-based). */
static int sort_perm(const double* w, int64_t d, int64_t* perm) {
    key_idx* ki = (key_idx*)malloc((size_t)(d > 0 ? d : 1) * sizeof(key_idx));
    if (!ki) return 4;
    for (int64_t i = 0; i < d; ++i) {
        ki[i].key = total_order_key(w[i]);
        ki[i].idx = i;
    }
    qsort(ki, (size_t)d, sizeof(key_idx), cmp_key_idx);
    for (int64_t k = 0; k < d; ++k) perm[k] = ki[k].idx;
    free(ki);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Neumaier compensated sums.                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    double s, c;
} csum;

static void csum_add(csum* a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static void csum_merge(csum* a, const csum* b) {
    csum_add(a, b->s);
    a->c += b->c;
}

static double csum_value(const csum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* The prox of one vector.                                                   */
/* ------------------------------------------------------------------------ */

/*
 * ws_oracle_prox: out[i] = prox_{lambda R}(w)_i, ids[i] = cluster rank of i
 * (0 = cluster of the smallest values).  perm (nullable) receives the stable
 * sorting permutation, x_sorted (nullable) the sorted values.  Returns 0 on
 * success, 1 on invalid arguments, 2 on a non-finite input, 4 on OOM.
 * n_clusters (nullable) receives the number of clusters.
 */
int ws_oracle_prox(const double* w, int64_t d, double lambda, double* out, int32_t* ids,
                   int64_t* perm_out, double* x_sorted, int64_t* n_clusters) {
    if (d < 0 || !(lambda >= 0.0) || !isfinite(lambda)) return 1;
    if (d == 0) {
        if (n_clusters) *n_clusters = 0;
        return 0;
    }
    for (int64_t i = 0; i < d; ++i)
        if (!isfinite(w[i])) return 2;
    if (d == 1) {
        out[0] = w[0];
        if (ids) ids[0] = 0;
        if (perm_out) perm_out[0] = 0;
        if (x_sorted) x_sorted[0] = w[0];
        if (n_clusters) *n_clusters = 1;
        return 0;
    }

    int64_t* perm = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    double* y = (double*)malloc((size_t)d * sizeof(double));
    csum* bsum = (csum*)malloc((size_t)d * sizeof(csum));
    int64_t* bcnt = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    if (!perm || !y || !bsum || !bcnt) {
        free(perm); free(y); free(bsum); free(bcnt);
        return 4;
    }
    int rc = sort_perm(w, d, perm);
    if (rc) {
        free(perm); free(y); free(bsum); free(bcnt);
        return rc;
    }

    /* step 2: y_k = x_k + lambda (d + 1 - 2k)/(d - 1), k = 1..d */
    for (int64_t k = 1; k <= d; ++k) {
        double xk = w[perm[k - 1]];
        y[k - 1] = xk + lambda * (double)(d + 1 - 2 * k) / (double)(d - 1);
    }

    /* step 3: pool adjacent violators with a stack of blocks */
    int64_t top = 0; /* number of blocks on the stack */
    for (int64_t k = 0; k < d; ++k) {
        bsum[top].s = y[k];
        bsum[top].c = 0.0;
        bcnt[top] = 1;
        ++top;
        while (top >= 2) {
            double mean_left = csum_value(&bsum[top - 2]) / (double)bcnt[top - 2];
            double mean_right = csum_value(&bsum[top - 1]) / (double)bcnt[top - 1];
            if (mean_left >= mean_right) {
                csum_merge(&bsum[top - 2], &bsum[top - 1]);
                bcnt[top - 2] += bcnt[top - 1];
                --top;
            } else {
                break;
            }
        }
    }

    /* step 4: expand the blocks and scatter back to the original order */
    int64_t k = 0;
    for (int64_t r = 0; r < top; ++r) {
        double value = csum_value(&bsum[r]) / (double)bcnt[r];
        for (int64_t j = 0; j < bcnt[r]; ++j, ++k) {
            out[perm[k]] = value;
            if (ids) ids[perm[k]] = (int32_t)r;
        }
    }
    if (perm_out) memcpy(perm_out, perm, (size_t)d * sizeof(int64_t));
    if (x_sorted)
        for (int64_t j = 0; j < d; ++j) x_sorted[j] = w[perm[j]];
    if (n_clusters) *n_clusters = top;
    free(perm); free(y); free(bsum); free(bcnt);
    return 0;
}

/*
 * ws_oracle_prox_l1: the proximal step with weight sharing, l1 and rewinding
 * (Rewinding section, Alg. 2), following the algorithm's steps:
 *   1. x, perm = sort(w) (stable);
 *   2. v_k = alpha (d + 1 - 2k)/(d - 1), k = 1..d (the velocities, -alpha grad R);
 *      every particle has mass 1;
 *   3. collisions: particles whose destinations x + v cross merge into one
 *      cluster carrying the sums of x and of v (momentum is conserved, so the
 *      cluster moves with the mean velocity); computed as pool adjacent
 *      violators on y = x + v, pooling on >= as in ws_oracle_prox, with the
 *      cluster's x-sum and v-sum carried alongside the y-sum;
 *   4. per cluster with mean position x_C and mean velocity v_C:
 *        zero  = |x_C + v_C| < beta
 *        v_C  -= beta sign(x_C + v_C)
 *        x_C = v_C = 0 where zero
 *        x_C  += v_scale (1 - rho) v_C
 *      (v_scale = 1 is Alg. 2; the experiments' variant multiplies the
 *      remaining displacement by the learning rate instead of scaling alpha
 *      and beta by it, which is v_scale = learning rate);
 *   5. repeat per cluster and scatter back by perm.
 * ids as in ws_oracle_prox (the clusters of the weight-sharing step).
 * Returns 0, 1 (invalid: beta < 0, rho outside [0, 1], v_scale < 0 or any of
 * them non-finite), 2 (non-finite input) or 4 (OOM).
 */
int ws_oracle_prox_l1(const double* w, int64_t d, double alpha, double beta, double rho, double v_scale,
                      double* out, int32_t* ids, int64_t* n_clusters) {
    if (d < 0 || !(alpha >= 0.0) || !isfinite(alpha) || !(beta >= 0.0) || !isfinite(beta) || !(rho >= 0.0) ||
        !(rho <= 1.0) || !(v_scale >= 0.0) || !isfinite(v_scale))
        return 1;
    if (d == 0) {
        if (n_clusters) *n_clusters = 0;
        return 0;
    }
    for (int64_t i = 0; i < d; ++i)
        if (!isfinite(w[i])) return 2;
    int64_t* perm = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    csum* ysum = (csum*)malloc((size_t)d * sizeof(csum));
    csum* xsum = (csum*)malloc((size_t)d * sizeof(csum));
    csum* vsum = (csum*)malloc((size_t)d * sizeof(csum));
    int64_t* bcnt = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    if (!perm || !ysum || !xsum || !vsum || !bcnt) {
        free(perm); free(ysum); free(xsum); free(vsum); free(bcnt);
        return 4;
    }
    int rc = sort_perm(w, d, perm);
    if (rc) {
        free(perm); free(ysum); free(xsum); free(vsum); free(bcnt);
        return rc;
    }
    int64_t top = 0;
    for (int64_t k = 1; k <= d; ++k) {
        const double xk = w[perm[k - 1]];
        const double vk = d > 1 ? alpha * (double)(d + 1 - 2 * k) / (double)(d - 1) : 0.0;
        ysum[top].s = xk + vk; ysum[top].c = 0.0;
        xsum[top].s = xk; xsum[top].c = 0.0;
        vsum[top].s = vk; vsum[top].c = 0.0;
        bcnt[top] = 1;
        ++top;
        while (top >= 2) {
            double mean_left = csum_value(&ysum[top - 2]) / (double)bcnt[top - 2];
            double mean_right = csum_value(&ysum[top - 1]) / (double)bcnt[top - 1];
            if (!(mean_left >= mean_right)) break;
            csum_merge(&ysum[top - 2], &ysum[top - 1]);
            csum_merge(&xsum[top - 2], &xsum[top - 1]);
            csum_merge(&vsum[top - 2], &vsum[top - 1]);
            bcnt[top - 2] += bcnt[top - 1];
            --top;
        }
    }
    int64_t k = 0;
    for (int64_t r = 0; r < top; ++r) {
        double x = csum_value(&xsum[r]) / (double)bcnt[r];
        double v = csum_value(&vsum[r]) / (double)bcnt[r];
        const double s = x + v;
        const int zero = fabs(s) < beta;
        v -= beta * (double)((s > 0.0) - (s < 0.0));
        if (zero) { x = 0.0; v = 0.0; }
        x += v_scale * (1.0 - rho) * v;
        for (int64_t j = 0; j < bcnt[r]; ++j, ++k) {
            out[perm[k]] = x;
            if (ids) ids[perm[k]] = (int32_t)r;
        }
    }
    if (n_clusters) *n_clusters = top;
    free(perm); free(ysum); free(xsum); free(vsum); free(bcnt);
    return 0;
}

/*
 * Batched prox: segment s is w[offsets[s] .. offsets[s+1]) with its own
 * lambdas[s]; cluster ids are local to the segment.  n_clusters (nullable)
 * receives one count per segment.
 */
int ws_oracle_prox_batched(const double* w, const int64_t* offsets, int64_t n_seg,
                           const double* lambdas, double* out, int32_t* ids,
                           int64_t* n_clusters) {
    if (n_seg < 0) return 1;
    for (int64_t s = 0; s < n_seg; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        if (b < a) return 1;
        int64_t nc = 0;
        int rc = ws_oracle_prox(w + a, b - a, lambdas[s], out + a, ids ? ids + a : NULL, NULL,
                                NULL, &nc);
        if (rc) return rc;
        if (n_clusters) n_clusters[s] = nc;
    }
    return 0;
}

/*
 * Backward: grad_in[i] = mean of grad_out over the cluster of i, clusters
 * given by (segment, id).  offsets == NULL means one segment of length n.
 */
int ws_oracle_backward(const double* grad_out, const int32_t* ids, const int64_t* offsets,
                       int64_t n_seg, int64_t n, double* grad_in) {
    int64_t single[2] = {0, n};
    if (!offsets) {
        offsets = single;
        n_seg = 1;
    }
    for (int64_t s = 0; s < n_seg; ++s) {
        int64_t a = offsets[s], b = offsets[s + 1];
        if (b <= a) continue;
        int32_t maxid = 0;
        for (int64_t i = a; i < b; ++i) {
            if (ids[i] < 0) return 1;
            if (ids[i] > maxid) maxid = ids[i];
        }
        csum* sums = (csum*)calloc((size_t)maxid + 1, sizeof(csum));
        int64_t* cnt = (int64_t*)calloc((size_t)maxid + 1, sizeof(int64_t));
        if (!sums || !cnt) {
            free(sums); free(cnt);
            return 4;
        }
        for (int64_t i = a; i < b; ++i) {
            csum_add(&sums[ids[i]], grad_out[i]);
            cnt[ids[i]] += 1;
        }
        for (int64_t i = a; i < b; ++i) grad_in[i] = csum_value(&sums[ids[i]]) / (double)cnt[ids[i]];
        free(sums); free(cnt);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The penalty itself.                                                       */
/* ------------------------------------------------------------------------ */

/* R(w) straight from Eq. (1): O(d^2) pairs, long double accumulator. */
double ws_oracle_R_pairs(const double* w, int64_t d) {
    if (d < 2) return 0.0;
    long double acc = 0.0L;
    for (int64_t i = 0; i < d; ++i)
        for (int64_t j = 0; j < i; ++j) acc += fabsl((long double)w[i] - (long double)w[j]);
    return (double)(acc / (long double)(d - 1));
}

/*
 * R(w) from the sorted form of App. B: R = 1/(d-1) sum_i ((i-1) x_i - s_i),
 * s_i = sum_{j<i} x_j (1-based), x = sort(w).
 */
double ws_oracle_R_sorted(const double* w, int64_t d) {
    if (d < 2) return 0.0;
    int64_t* perm = (int64_t*)malloc((size_t)d * sizeof(int64_t));
    if (!perm || sort_perm(w, d, perm)) {
        free(perm);
        return NAN;
    }
    long double prefix = 0.0L, acc = 0.0L;
    for (int64_t i = 1; i <= d; ++i) {
        long double xi = (long double)w[perm[i - 1]];
        acc += (long double)(i - 1) * xi - prefix;
        prefix += xi;
    }
    free(perm);
    return (double)(acc / (long double)(d - 1));
}

/* ------------------------------------------------------------------------ */
/* Neighbour-collision slack (App. D, Corollary "Neighbour collision").     */
/* ------------------------------------------------------------------------ */

/*
 * For the sorted particles with destinations y (1-based k as in the paper),
 *   slack_k = max_{j<=k} avg(y_{j:k}) - min_{j>=k+1} avg(y_{k+1:j}).
 * Particles k and k+1 end in the same cluster iff slack_k >= 0.  k is given
 * 0-based here as the boundary between sorted positions k and k+1
 * (0 <= k < d-1).  Sums are accumulated outward from the boundary in long
 * double, directly from x (no prefix-sum differences), so the result is
 * accurate near zero, which is where it is used: deciding whether a
 * partition mismatch sits on a near-tie.
 */
double ws_oracle_neighbour_slack(const double* x_sorted, int64_t d, double lambda, int64_t k0) {
    if (d < 2 || k0 < 0 || k0 >= d - 1) return NAN;
    long double lam = (long double)lambda, dm1 = (long double)(d - 1);
    /* left side: blocks [j..k], 1-based k = k0+1 */
    int64_t k = k0 + 1;
    long double sum = 0.0L, best_left = -INFINITY;
    for (int64_t j = k; j >= 1; --j) {
        sum += (long double)x_sorted[j - 1] + lam * (long double)(d + 1 - 2 * j) / dm1;
        long double avg = sum / (long double)(k - j + 1);
        if (avg > best_left) best_left = avg;
    }
    sum = 0.0L;
    long double best_right = INFINITY;
    for (int64_t j = k + 1; j <= d; ++j) {
        sum += (long double)x_sorted[j - 1] + lam * (long double)(d + 1 - 2 * j) / dm1;
        long double avg = sum / (long double)(j - k);
        if (avg < best_right) best_right = avg;
    }
    return (double)(best_left - best_right);
}

/* Sorting helper exposed for the tests (stable, IEEE total order). */
int ws_oracle_sort(const double* w, int64_t d, int64_t* perm, double* x_sorted) {
    if (d < 0) return 1;
    if (d == 0) return 0;
    int rc = sort_perm(w, d, perm);
    if (rc) return rc;
    if (x_sorted)
        for (int64_t k = 0; k < d; ++k) x_sorted[k] = w[perm[k]];
    return 0;
}
