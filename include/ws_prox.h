/*
 * ws_prox.h -- C ABI of libws_prox.so: the proximal map of the weight-sharing
 * penalty on NVIDIA GB300 (sm_103a).
 *
 * The penalty (Eq. (1) of "Weight-Sharing Regularization", arXiv 2311.03096):
 *     R(w) = 1/(d-1) * sum_{i>j} |w_i - w_j|,   w in R^d.
 * Its proximal map (Sec. 1, prox definition; unique by strong convexity):
 *     prox_{lambda R}(w) = argmin_u  lambda R(u) + 1/2 ||u - w||^2.
 * Computed as in Sec. 3-5 / Alg. 2: sort w ascending (x), shift
 * y_k = x_k + lambda (d + 1 - 2k)/(d - 1) (k = 1..d, the particle velocity of
 * Alg. 2), pool adjacent violators of y into clusters at their means (the
 * isotonic regression of y, Sec. 3; pooling on >=, Sec. 4.1), and give every
 * weight the value of its cluster.
 *
 * Conventions shared by every entry point:
 *   - Data pointers (values, out, cluster ids, gradients, lambdas, cluster
 *     counts) are DEVICE pointers owned by the caller, unless a parameter says
 *     "host".  The library never frees them.
 *   - All device scratch memory is owned by a ws_plan and allocated when the
 *     plan is created; a call on an existing plan allocates nothing, never
 *     synchronises the host and only enqueues work on `stream`, so it can be
 *     captured in a CUDA graph.
 *   - Layout: a batch is one flat array of n values; segment s is
 *     values[offsets[s] .. offsets[s+1]), processed independently with its
 *     own lambda.  Cluster ids are 0-based and local to their segment; id 0 is
 *     the cluster of the smallest values and ids increase with the value.
 *   - dtype WS_F32 means float values/out; WS_F64 means double values/out.
 *     Cluster ids are int32.  out may alias values (in-place).
 *   - Degenerate cases: a segment of length 0 is skipped; of length 1 gets
 *     out = w and id 0; lambda = 0 gives out = w with one cluster per distinct
 *     value.  Ties in w always share a cluster (equal x_k = x_{k+1} give
 *     y_k >= y_{k+1}, which pools), so the result does not depend on how ties
 *     are ordered.
 *   - Errors: argument errors are returned synchronously (WS_ERR_INVALID) and
 *     nothing is enqueued.  Errors found on the device (a NaN/Inf input, a
 *     bounded wait that gave up) are OR-ed into the context's status word and
 *     reported by ws_get_status; outputs of that call are then unspecified.
 *   - Concurrency: a plan's scratch (sort buffers, look-back words, hull and
 *     cluster tables) is reused by every call made with that plan.  The
 *     single-vector calls (ws_prox, ws_prox_l1, ws_prox_backward,
 *     ws_prox_dlambda, ws_R) share one plan per (d, dtype) cached in the
 *     context.  So calls that use the same plan -- or the same context with
 *     the same single-vector shape -- must be ordered on one stream (or be
 *     otherwise serialised); if their kernels overlap on the GPU their
 *     results are undefined.  Calls on different plans, or on different
 *     contexts, may run concurrently on different streams.  A context and its
 *     plans may be used from several host threads only if the caller
 *     serialises those calls.
 */
#ifndef WS_PROX_H
#define WS_PROX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WS_OK = 0,
    WS_ERR_INVALID = 1,   /* bad argument (null pointer, negative size, lambda < 0 or not finite, ...) */
    WS_ERR_NONFINITE = 2, /* an input value was NaN or +-Inf (device-detected) */
    WS_ERR_CUDA = 3,      /* a CUDA runtime call failed */
    WS_ERR_NOMEM = 4,     /* device allocation failed (plan creation only) */
    WS_ERR_TIMEOUT = 5,   /* a bounded device-side wait gave up (device-detected) */
    WS_ERR_INTERNAL = 6   /* an internal consistency check failed (device-detected) */
} ws_status;

typedef enum { WS_F32 = 0, WS_F64 = 1 } ws_dtype;

/* Arithmetic used for the cluster values.  Both modes take every merge
 * decision exactly (128-bit fixed-point prefix sums, integer comparisons), so
 * they produce the same partition; they differ in how a cluster mean and its
 * shift are rounded:
 *   WS_PREC_FP32_COMP: FP32 arithmetic on the exact integer cluster sum
 *                      (error a few FP32 ulps of max|w| + lambda);
 *   WS_PREC_FP64:      FP64 arithmetic (error a few FP64 ulps). */
typedef enum { WS_PREC_FP32_COMP = 0, WS_PREC_FP64 = 1 } ws_prec;

typedef struct ws_ctx ws_ctx;   /* device selection + asynchronous status word */
typedef struct ws_plan ws_plan; /* segment layout + all scratch for one batch shape */

/* Create a context on CUDA device `device` (allocates a few bytes of device
 * memory for the status word).  Returns WS_OK and sets *ctx. */
ws_status ws_ctx_create(ws_ctx** ctx, int device);
void ws_ctx_destroy(ws_ctx* ctx);

/* Plan a batch: `offsets` is a HOST array of n_seg + 1 non-decreasing int64
 * with offsets[0] = 0; n = offsets[n_seg] values of type `dtype`.  Segments
 * must be shorter than 2^31.  Allocates every buffer the calls need
 * (synchronous; not capturable).  The plan copies the offsets; the caller may
 * free them afterwards. */
ws_status ws_plan_create(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg,
                         ws_dtype dtype);
void ws_plan_destroy(ws_plan* plan);

/* Autotuned plan for a batch layout.  Segments of at most `threshold`
 * elements run one CTA each (shared-memory sort and hull); longer ones run the
 * device-wide tiled path.  For each candidate threshold (host array of n_cand
 * values, each capped at the one-CTA maximum; NULL for {0, 512, 1024, 2048,
 * 4096}) a plan is built and `reps` forward calls on (values, lambdas, out,
 * cluster_ids, prec) are timed with CUDA events on `stream` after one
 * warm-up; the fastest plan is returned in *plan and the others destroyed.
 * *chosen (nullable) receives its threshold, times_ms (nullable, n_cand
 * doubles) each candidate's mean milliseconds.  The chosen plan then times
 * the round caps {8, 16, 32, 64} the same way and keeps the fastest
 * (ws_plan_params reports it).  A set-up step: it allocates
 * and synchronises the stream, so it is not capturable.  Arguments as for
 * ws_plan_create and ws_prox_batched; reps >= 1, thresholds >= 0, else
 * WS_ERR_INVALID.  Not in the paper: a library convenience. */
ws_status ws_plan_autotune(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg, ws_dtype dtype,
                           const void* values, const double* lambdas, void* out, int32_t* cluster_ids,
                           ws_prec prec, const int64_t* thresholds, int n_cand, int reps, int64_t* chosen,
                           double* times_ms, void* stream);

/* The parameters a plan runs with: its one-CTA length threshold and the round
 * cap of the Imminent Collisions rounds (Sec. 4) in its tile and one-CTA
 * kernels.  ws_plan_autotune times caps {8, 16, 32, 64} on its chosen plan
 * after the thresholds and keeps the fastest for that plan; other plans use
 * the context's cap (ws_debug_set_ic_cap).  Nullable outputs;
 * WS_ERR_INVALID for a NULL plan. */
ws_status ws_plan_params(const ws_plan* plan, int64_t* small_max, int* ic_cap);

/* Batched forward (Alg. 2 per segment, lambda = lambdas[s] from DEVICE memory,
 * n_seg doubles, each >= 0 and finite -- checked on the device, reported as
 * WS_ERR_INVALID through ws_get_status).  values/out: n elements of the
 * plan's dtype; cluster_ids: n int32 (nullable); n_clusters: n_seg int64
 * (nullable) receives the number of clusters of each segment. */
ws_status ws_prox_batched(ws_plan* plan, const void* values, const double* lambdas, void* out,
                          int32_t* cluster_ids, int64_t* n_clusters, ws_prec prec, void* stream);

/* Warm-started batched forward (the paper's Future Work: start from a
 * candidate weight-sharing and edit it into the exact one).  ids_prev: n int32
 * in DEVICE memory, the cluster ids of an earlier call on nearby values (the
 * previous training step's cluster_ids); any values are accepted.  In every
 * segment of the one-CTA kernel, the runs of equal ids_prev (low 16 bits)
 * along the sorted order are the candidate: points that lie on or above the
 * chord of their run cannot be hull vertices and are dropped before the
 * Imminent Collisions rounds (Sec. 4) start.  Outputs are those of
 * ws_prox_batched for ANY ids_prev -- it changes the time only.  ids_prev may
 * alias cluster_ids (a segment reads it before writing); device-wide segments
 * ignore it.  NULL ids_prev with n > 0 is WS_ERR_INVALID; other arguments as
 * for ws_prox_batched. */
ws_status ws_prox_batched_warm(ws_plan* plan, const void* values, const double* lambdas,
                               const int32_t* ids_prev, void* out, int32_t* cluster_ids,
                               int64_t* n_clusters, ws_prec prec, void* stream);

/* Single vector of length d with a host lambda.  Plans (and allocates) on
 * first use of a given (d, dtype) and caches the plan in the context, so the
 * first call for a shape is not capturable; later calls are.  n_clusters is
 * a nullable DEVICE pointer to one int64. */
ws_status ws_prox(ws_ctx* ctx, const void* w, int64_t d, double lambda, void* out,
                  int32_t* cluster_ids, int64_t* n_clusters, ws_dtype dtype, ws_prec prec,
                  void* stream);

/* Weight sharing + l1 with rewinding: the proximal step of Alg. 2 (Rewinding
 * section).  The clusters are those of ws_prox / ws_prox_batched; a cluster
 * with mean weight x and mean shift v (the mean of lambda (d+1-2k)/(d-1) over
 * its sorted positions k) ends at
 *     0                                        if |x + v| < beta,
 *     x + v_scale (1 - rho) (v - beta sign(x + v))   otherwise.
 * rho = 0 and v_scale = 1 give prox of lambda R + beta l1, i.e. the soft
 * threshold of prox_{lambda R} (Prop. D.6); rho = 1 leaves surviving
 * clusters at their mean weight; v_scale = the learning rate is the
 * experiments' variant that scales the remaining displacement instead of
 * lambda and beta.  Computed inside the cluster-value step: no extra pass.
 * beta >= 0, 0 <= rho <= 1, v_scale >= 0, all finite, else WS_ERR_INVALID
 * (nothing is enqueued); epi must not be NULL.  Other arguments, layouts,
 * ownership and errors as for ws_prox_batched / ws_prox.  cluster_ids are the
 * weight-sharing clusters (zeroed clusters keep their own ids). */
typedef struct ws_l1_rewind {
    double beta;     /* l1 coefficient */
    double rho;      /* rewinding, 0 (none) .. 1 (full) */
    double v_scale;  /* scale of the remaining displacement (1 in Alg. 2) */
} ws_l1_rewind;

ws_status ws_prox_batched_l1(ws_plan* plan, const void* values, const double* lambdas,
                             const ws_l1_rewind* epi, void* out, int32_t* cluster_ids,
                             int64_t* n_clusters, ws_prec prec, void* stream);
ws_status ws_prox_l1(ws_ctx* ctx, const void* w, int64_t d, double lambda, const ws_l1_rewind* epi,
                     void* out, int32_t* cluster_ids, int64_t* n_clusters, ws_dtype dtype,
                     ws_prec prec, void* stream);

/* Backward of the forward with the partition held fixed (the Jacobian of the
 * cluster means): grad_in[i] = mean of grad_out over the cluster of i, where
 * clusters are given by (segment, cluster_ids[i]) as written by the forward on
 * the same plan.  grad_out/grad_in: n elements of the plan's dtype, may alias. */
ws_status ws_prox_backward_batched(ws_plan* plan, const void* grad_out, const int32_t* cluster_ids,
                                   void* grad_in, void* stream);

/* Single-vector backward (plan cached in the context as for ws_prox). */
ws_status ws_prox_backward(ws_ctx* ctx, const void* grad_out, const int32_t* cluster_ids, int64_t d,
                           void* grad_in, ws_dtype dtype, void* stream);

/* Derivative with respect to lambda, the partition held fixed: a cluster on
 * sorted positions a..b (1-based) moves with the mean velocity of its
 * particles (Sec. 3), so d out_i / d lambda_s = (d+1-a-b)/(d-1) for every i in
 * it (0 for segments of d <= 1).  grad_lambda[s] (DEVICE, n_seg doubles,
 * overwritten) receives sum_{i in s} grad_out[i] * d out_i / d lambda_s,
 * accumulated in FP64 with atomics (the order of the additions is not fixed).
 * cluster_ids as written by the forward on the same plan layout (ranked by
 * value, which is what fixes each cluster's positions).  grad_out: n elements
 * of the plan's dtype.  Total of the plan's large-segment slots must be
 * < 2^31, else WS_ERR_INVALID.  Stream-ordered. */
ws_status ws_prox_dlambda_batched(ws_plan* plan, const void* grad_out, const int32_t* cluster_ids,
                                  double* grad_lambda, void* stream);
/* Single vector (plan cached as for ws_prox); grad_lambda: one DEVICE double. */
ws_status ws_prox_dlambda(ws_ctx* ctx, const void* grad_out, const int32_t* cluster_ids, int64_t d,
                          double* grad_lambda, ws_dtype dtype, void* stream);

/* R(w) and the weight-sharing measure of one vector of d weights (not part
 * of the proximal step; for monitoring a model).  R(w) = 1/(d-1) *
 * sum_{i>j} |w_i - w_j| (Eq. (1)) is evaluated as the appendix "Computing R"
 * does: sort, then 1/(d-1) sum_k (2k - d - 1) x_k over the sorted x, the sum
 * exact in 128-bit fixed point and rounded once (inputs spanning more than
 * ~34 binades of FP32, or 5 of FP64, lose the bits of their smallest values
 * below 2^-L, as the prox does).  The measure is #distinct nonzero weights /
 * #nonzero weights (the weight-sharing metric of the CIFAR10 experiment), 0
 * when every weight is zero.  w: DEVICE, d elements of dtype; R_out,
 * metric_out: nullable DEVICE pointers to one double each.  d = 0 or 1 gives
 * R = 0.  Plans (allocates) on first use of a (d, dtype); NaN/Inf inputs are
 * reported through ws_get_status.  Stream-ordered. */
ws_status ws_R(ws_ctx* ctx, const void* w, int64_t d, ws_dtype dtype, double* R_out, double* metric_out,
               void* stream);

/* Synchronise `stream`, then return and clear the context's device status
 * word (WS_OK if no device-side error happened since the last call). */
ws_status ws_get_status(ws_ctx* ctx, void* stream);

/* Whether a call since the last query used a fixed point that truncated
 * input values: a segment's nonzero values spanning more than 34 binades
 * (FP32; 5 for FP64) get the scale of its largest values, and values more
 * than that far below lose their lowest bits (toward zero).  The partition is
 * then the exact prox of the truncated values and every output stays within
 * the stated tolerance, but a partition check against an exact reference is
 * not guaranteed (FP64 segments of N(0,1) weights already span more than 5
 * binades).  Information, not an error: ws_get_status does not report it.
 * Synchronises `stream`; *inexact = 1 or 0; the flag is cleared.  Call when
 * no other stream is using the context. */
ws_status ws_get_inexact(ws_ctx* ctx, int* inexact, void* stream);

/* Human-readable name of a status code (static string). */
const char* ws_status_string(ws_status s);

/* Set the iteration bound of every device-side spin-wait (decoupled
 * look-back).  A wait that exceeds it gives up, sets WS_ERR_TIMEOUT and lets
 * its kernel exit.  0 restores the default.  Test hook. */
void ws_debug_set_spin_limit(ws_ctx* ctx, int64_t limit);

/* Segments no longer than `small_max` elements go to the fused single-CTA
 * kernel, longer ones to the device-wide path.  Applies to plans created
 * afterwards (cached single-vector plans are dropped); a negative value
 * restores the default (4096 for float and double, also the maximum).
 * Test hook: lets small inputs exercise the device-wide path. */
void ws_debug_set_small_max(ws_ctx* ctx, int64_t small_max);

/* Round cap of the Imminent Collisions rounds that every hull tile of the
 * device-wide path and every one-CTA segment runs first (appendix algorithm
 * "Imminent collisions algorithm (v2)"); a tile whose rounds have not
 * converged within the cap takes the tree of bridge merges instead.  0 skips
 * the rounds (every tile takes the merges); a negative value restores the
 * default (32).  Takes effect on the next call of every plan of the context
 * except autotuned plans that chose their own cap (ws_plan_params).  Test and
 * benchmark hook. */
void ws_debug_set_ic_cap(ws_ctx* ctx, int cap);

/* How the hull tiles of the last ws_prox call for (d, dtype) on this context
 * were built.  counts (HOST, n_counts >= 3 int64, overwritten):
 * counts[0] = tiles built by the general kernel, counts[1] = tiles whose
 * rounds hit the cap (tree of merges), counts[r + 1] = tiles whose rounds
 * converged after r rounds (the last, unchanged round included; r >=
 * n_counts - 1 is counted in the last slot).  Synchronises the device.
 * All zero if no such call was made.  Benchmark hook. */
ws_status ws_debug_hull_stats(ws_ctx* ctx, int64_t d, ws_dtype dtype, int64_t* counts, int n_counts);

/* Runs only the radix sort of the device-wide path and writes, for every
 * segment that the plan sends down that path, its values sorted ascending in
 * IEEE total order (-0 before +0) at the segment's own position in
 * `sorted_out` (device, plan dtype); other positions are left untouched.
 * Test hook for bit-exact sort parity. */
ws_status ws_debug_sort(ws_plan* plan, const void* values, void* sorted_out, void* stream);

/* Largest d accepted by ws_prox_backward_noalloc (2^20 elements). */
#define WS_NOALLOC_MAX_ELEMS (1 << 20)

/* Backward that allocates no device memory (the paper has no counterpart;
 * this is a library convenience).  Same result as ws_prox_backward for one
 * vector of d <= WS_NOALLOC_MAX_ELEMS elements: grad_in[i] = mean of
 * grad_out over the cluster of i, clusters given by cluster_ids (0-based,
 * < d) as written by the forward.  It exists for callers that must not call
 * cudaMalloc/cudaFree where they run the backward: a framework that has
 * already reserved the device memory for its own pool, or a loop that cannot
 * take the implicit device synchronisation of an allocation.  Its per-cluster
 * sums and counts live in one fixed array of device memory (12 MiB) that the
 * library holds on every GPU that loads it until the process exits.
 *   - grad_out, cluster_ids, grad_in: DEVICE pointers owned by the caller
 *     (d elements of dtype, d int32, d elements of dtype); grad_in may alias
 *     grad_out.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it; make
 *     that first call before any stream capture begins.  The cached address
 *     does not survive cudaDeviceReset: do not use the entry point across a
 *     device reset.  No call allocates.
 *   - The device that is current when the call is made must be the device
 *     that holds grad_out, cluster_ids and grad_in, and `stream` must belong
 *     to it.
 *   - A launch error left pending by earlier, unrelated code is cleared on
 *     entry; WS_ERR_CUDA reports only this call's own launch failures.
 *   - d > WS_NOALLOC_MAX_ELEMS or d < 0 returns WS_ERR_INVALID and enqueues
 *     nothing; d == 0 is a no-op.  Ids outside [0, d) are skipped and leave
 *     their grad_in entry unchanged.
 *   - All calls share the one array: calls whose kernels may overlap on the
 *     GPU (different streams without ordering, several host threads) race
 *     and give wrong results; order them on one stream.  Each call clears the
 *     part of the array it uses before accumulating.
 *   - Stream-ordered on `stream`; the host is not synchronised. */
ws_status ws_prox_backward_noalloc(const void* grad_out, const int32_t* cluster_ids, int64_t d,
                                   void* grad_in, ws_dtype dtype, void* stream);

/* Per-kernel timing for benchmarks.  ws_debug_profile(ctx, 1) starts
 * recording a CUDA event pair around every kernel the context launches (on
 * the launching stream) and clears the totals; 0 stops recording.
 * ws_debug_profile_read synchronises on the last recorded event and returns
 * the summed duration and launch count of one kernel kind (0 <= kind <
 * number of kinds; ws_debug_kernel_name(kind) names it and returns NULL past
 * the last kind). */
ws_status ws_debug_profile(ws_ctx* ctx, int enable);
ws_status ws_debug_profile_read(ws_ctx* ctx, int kind, double* total_ms, int64_t* count);
const char* ws_debug_kernel_name(int kind);

/* Number of kernels this context has launched since it was created. */
int64_t ws_debug_launch_count(ws_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* WS_PROX_H */
