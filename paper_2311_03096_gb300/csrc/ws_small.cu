// ws_small.cu -- fused single-CTA prox for short segments (n <= 4096, float
// and double): one CTA loads a segment once, sorts (key, index)
// pairs in shared memory, builds the exact hull, and writes values and cluster
// ids straight to their original positions.  HBM traffic is the I/O floor:
// read w, write out and id (12 B/element for float).  The lean kernel
// (k_small) builds the hull by Imminent Collisions rounds with a fallback to
// chains and bridge trees; the general kernel (k_small_general) takes the rare
// segments whose fixed-point sums need 128 bits.
#include "ws_hull.cuh"
#include "ws_kernels.cuh"

namespace {

// Shared memory of one segment, laid out so that three CTAs fit on an SM:
// buffers whose lifetimes do not overlap share storage.
//   r1: digit counters of the sort  |  hull vertex list + cluster-start bits
//   r2: sort keys (dead after the prefix sums)  |  chunk hulls  |  values
template <typename T, int NT, int M>
struct SmallSmem {
    typedef typename KeyOf<T>::K K;
    static constexpr int CAP = NT * M;
    static_assert(32 % M == 0 || M % 32 == 0, "a thread's marks must lie in one 32-bit word");
    uint16_t idx[CAP];
    TilePrefix<NT, M> pre;  // fixed-point prefix sums of the sorted segment
    union {
        struct {
            uint32_t whist[(NT / 32) * 256];
            uint32_t dcount[256], dstart[256];
        } sort;
        struct {
            uint16_t V[CAP + 2];        // hull vertices (points)
            uint32_t mark[CAP / 32];    // bit p: a cluster starts at sorted position p
        } ids;
    } r1;
    union {
        K keys[CAP];
        HullSmem<NT, M> hull;
        T val[CAP];
    } r2;
    int wsum_i[NT / 32];
    int flags;
    int emin;
    SegConst sc, sct;
    float muq, muqt;
    int fast, fastt;
};

// The general one-CTA prox of one segment (every input, including values
// whose fixed-point sums need 128 bits): used for the segments the lean
// kernel below sends here.
template <typename T, int NT, int M>
__device__ __forceinline__ void small_general_segment(SmallSmem<T, NT, M>& s, int seg, const T* __restrict__ values,
                                                      const int64_t* __restrict__ offsets,
                                                      const double* __restrict__ lambdas, T* out, int32_t* ids,
                                                      int64_t* n_clusters, int fp64, const WsEpi& ep,
                                                      uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    typedef SmallSmem<T, NT, M> S;
    constexpr int CAP = S::CAP;
    constexpr int ITEMS = M;   // items per thread in the sort
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;

    const int64_t a0 = offsets[seg];
    const int n = (int)(offsets[seg + 1] - a0);
    const double lam = lambdas[seg];
    if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) {
        if (t == 0) ws_flag(status, WS_STATUS_BAD_LAMBDA);
        return;
    }
    if (n <= 0 || n > CAP) {
        if (n > CAP && t == 0) ws_flag(status, WS_STATUS_INTERNAL);
        if (n == 0 && t == 0 && n_clusters) n_clusters[seg] = 0;
        return;
    }

    // ---- load (striped per warp, coalesced), map to keys, check finiteness
    if (t == 0) { s.flags = 0; s.emin = 0x7fffffff; }
    __syncthreads();
    bool bad = false;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        int p = w * 32 * ITEMS + k * 32 + lane;
        if (p < n) {
            T v = values[a0 + p];
            bad |= !ws_isfinite(v);
            s.r2.keys[p] = KO::to_key(v);
            s.idx[p] = (uint16_t)p;
        }
    }
    if (bad) atomicOr(&s.flags, 1);
    __syncthreads();
    if (s.flags) {
        if (t == 0) ws_flag(status, WS_STATUS_NONFINITE);
        return;
    }
    if (n == 1) {
        if (t == 0) {
            const T x = values[a0];   // d = 1: no shift (the 1/(d-1) factor is vacuous)
            out[a0] = fp64 ? (T)ws_epilogue<double>((double)x, 0.0, ep.beta, ep.gamma, ep.on != 0)
                           : (T)ws_epilogue<float>((float)x, 0.0f, ep.beta_f, ep.gamma_f, ep.on != 0);
            if (ids) ids[a0] = 0;
            if (n_clusters) n_clusters[seg] = 1;
        }
        return;
    }

    // ---- LSD radix sort of (key, idx) in shared memory, 8-bit digits
    for (int pass = 0; pass < KO::BITS / 8; ++pass) {
        K kk[ITEMS];
        uint16_t ii[ITEMS];
        uint32_t dg[ITEMS];
        bool valid[ITEMS];
        int pos[ITEMS];
#pragma unroll
        for (int k = 0; k < ITEMS; ++k) {
            int p = w * 32 * ITEMS + k * 32 + lane;
            valid[k] = p < n;
            kk[k] = valid[k] ? s.r2.keys[p] : (K)0;
            ii[k] = valid[k] ? s.idx[p] : (uint16_t)0;
            dg[k] = (uint32_t)((kk[k] >> (8 * pass)) & 0xff);
        }
        __syncthreads();
        ws_rank_digits<NT, ITEMS, 1>(dg, valid, pos, s.r1.sort.whist, s.r1.sort.dcount, s.r1.sort.dstart);
#pragma unroll
        for (int k = 0; k < ITEMS; ++k)
            if (valid[k]) { s.r2.keys[pos[k]] = kk[k]; s.idx[pos[k]] = ii[k]; }
        __syncthreads();
    }

    // ---- fixed point and prefix sums (blocked: thread t owns sorted [t*M, t*M+M))
    int64_t q0;
    i128 total;
    int bsh;
    K kr[M];
    int emin = 0x7fffffff;   // smallest effective exponent of a nonzero value
#pragma unroll
    for (int i = 0; i < M; ++i) {
        kr[i] = (t * M + i < n) ? s.r2.keys[t * M + i] : (K)0;
        const T x = KO::from_key(kr[i]);
        if (t * M + i < n && x != (T)0) emin = min(emin, ws_eff_exp(x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emin = min(emin, __shfl_xor_sync(WS_FULL_MASK, emin, o));
    if (lane == 0) atomicMin(&s.emin, emin);
    __syncthreads();
    const K kfirst = s.r2.keys[0], klast = s.r2.keys[n - 1];
    const T xlo = KO::from_key(kfirst), xhi = KO::from_key(klast);
    const int emax = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), s.emin);
    if (t == 0) {
        s.sc = ws_seg_const<T>(n, lam, emax);
        bool f;
        s.muq = ws_muq(lam, s.sc, f);
        s.fast = f ? 1 : 0;
    }
    if (t == 0) {
        const int sh0 = ws_eff_exp(xlo) - emax + KO::FIX_OFS;
        s.sct = ws_seg_const_L(n, lam, s.sc.L - (sh0 > 0 ? sh0 : 0));
        bool f;
        s.muqt = ws_muq(lam, s.sct, f);
        s.fastt = f ? 1 : 0;
    }
    // (the prefix sums end with a barrier; the keys' storage is reused from here on)
    // this thread's entry of the chain thresholds at the scale the segment's mode
    // uses; the prefix stores it after its first barrier (the keys are dead then)
    static_assert(M * M <= NT, "one threshold entry per thread");
    int thr_v = 0;
    if (t < M * M) {
        int shb;
        const bool tbin = ws_tile_binade<T>(kfirst, klast, n, emax, shb);
        uint64_t mlam;
        int sx;
        ws_thr_consts(lam, KO::L_BASE - emax - (tbin && shb > 0 ? shb : 0), mlam, sx);
        thr_v = ws_thr_entry<M>(t, mlam, sx, n > 1 ? (uint64_t)(n - 1) : 1ull);
    }
    const int mode = ws_tile_prefix<T, NT, M>(s.pre, kr, kfirst, klast, n, emax, q0, total, bsh,
                                              t < M * M ? s.r2.hull.thr + t : nullptr, thr_v);
    const SegConst& sc = s.sc;

    // ---- exact hull (in-CTA merge)
    int nv;
    if (mode == WS_TILE_BINADE) {
        TilePtsDev<M> P = ws_dev_pts<M>(s.pre.s64, s.muqt, s.fastt != 0, (uint64_t)(klast - kfirst), n, s.sct);
        P.thr = s.r2.hull.thr;
        ws_cta_hull<NT, M, TilePtsDev<M>, true>(s.r2.hull, n, P, s.sct, &nv);
    } else if (mode == WS_TILE_NARROW) {
        const uint64_t range = (uint64_t)(ws_fixed<T>(xhi, emax) - q0);
        TilePtsDev<M> P = ws_dev_pts<M>(s.pre.s64, s.muq, s.fast != 0, range, n, sc);
        P.thr = s.r2.hull.thr;
        ws_cta_hull<NT, M, TilePtsDev<M>, true>(s.r2.hull, n, P, sc, &nv);
    } else {
        const TilePtsWide<M> P{s.pre.s64, s.pre.base};
        ws_cta_hull<NT, M>(s.r2.hull, n, P, sc, &nv);
    }
    auto X = [&](int p) -> i128 { return ws_tile_X<M>(s.pre.s64, s.pre.base, mode, q0, bsh, p); };
    {
        int l = s.r2.hull.lo[t], h = s.r2.hull.hi[t], o = s.r2.hull.cum[t];
        for (int i = l; i < h; ++i) s.r1.ids.V[o + (i - l)] = s.r2.hull.H[i * NT + t];
    }
    for (int i = t; i < CAP / 32; i += NT) s.r1.ids.mark[i] = 0u;
    __syncthreads();   // the chunk hulls are dead from here on (their storage holds the values)
    const int c = nv - 1;
    if (s.r1.ids.V[0] != 0 || s.r1.ids.V[c] != n) { if (t == 0) ws_flag(status, WS_STATUS_INTERNAL); }

    // ---- cluster values (a one-element cluster reads its weight back from the input).
    // FP32 arithmetic on deviation tiles: mean = x_first + (sum of deviations / n)
    // 2^-L, all terms exact but the last conversions (error a few FP32 ulps of
    // max |w|); otherwise from the exact 128-bit cluster sum.
    const bool dev32 = !fp64 && mode != WS_TILE_WIDE;
    const int Ldev = mode == WS_TILE_BINADE ? s.sct.L : sc.L;
    const float x0f = (float)xlo;
    for (int r = t; r < c; r += NT) {
        const int a = s.r1.ids.V[r], b = s.r1.ids.V[r + 1];
        const T xs = (b - a == 1) ? values[a0 + s.idx[a]] : (T)0;
        if (dev32) {
            const float mean = (b - a == 1) ? (float)xs
                                            : x0f + ldexpf(ws_u64_to_float((uint64_t)(s.pre.s64[ws_sidx<M>(b)] -
                                                                                   s.pre.s64[ws_sidx<M>(a)])) /
                                                               (float)(b - a),
                                                           -Ldev);
            s.r2.val[r] = (T)ws_epilogue<float>(mean, sc.mu_f * (float)(n - a - b), ep.beta_f, ep.gamma_f,
                                                ep.on != 0);
        } else {
            s.r2.val[r] = ValueOut<T>::value(X(b) - X(a), a, b, xs, sc, fp64 != 0, ep);
        }
        atomicOr(&s.r1.ids.mark[a >> 5], 1u << (a & 31));
    }
    __syncthreads();

    // ---- cluster id of every sorted position, then scatter to the original order
    const uint32_t mymarks = (s.r1.ids.mark[(t * M) >> 5] >> ((t * M) & 31)) & (uint32_t)((1ull << M) - 1ull);
    int tot;
    int run = ws_block_excl_scan<NT, int>(__popc(mymarks), s.wsum_i, &tot);
    for (int i = 0; i < M; ++i) {
        int p = t * M + i;
        if (p < n) {
            run += (mymarks >> i) & 1u;
            int r = run - 1;
            int64_t o = a0 + s.idx[p];
            out[o] = s.r2.val[r];
            if (ids) ids[o] = r;
        }
    }
    if (t == 0 && n_clusters) n_clusters[seg] = c;
}

template <typename T, int NT, int M>
__global__ void __launch_bounds__(NT, 3) k_small_general(const T* __restrict__ values,
                                                      const int64_t* __restrict__ offsets,
                                                      const int32_t* __restrict__ gen_list,
                                                      const int32_t* __restrict__ gen_count,
                                                      const double* __restrict__ lambdas, T* out, int32_t* ids,
                                                      int64_t* n_clusters, int fp64, const WsEpi ep,
                                                      uint32_t* status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem<T, NT, M>& s = *reinterpret_cast<SmallSmem<T, NT, M>*>(smem_raw);
    const int cnt = *gen_count;
    for (int i = blockIdx.x; i < cnt; i += gridDim.x) {
        small_general_segment<T, NT, M>(s, gen_list[i], values, offsets, lambdas, out, ids, n_clusters, fp64, ep,
                                        status);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The lean one-CTA prox: keys and their original positions sorted in shared
// memory, then the hull of the sorted segment by the Imminent Collisions
// rounds with the chain-and-tree fallback (ws_hull.cuh), cluster ids from the
// cluster-start bitmap, values scattered back through the positions.
// Segments whose prefix sums need 128 bits (or whose bridge walks are too
// long) are appended to gen_list for the general kernel above.
// ---------------------------------------------------------------------------
template <typename T>
struct LeanSmem {
    typedef typename KeyOf<T>::K K;
    static constexpr int CAP = wsh::TILE;               // 4096 elements, float and double
    // Arrays read in blocks of 16 consecutive entries per thread are padded
    // (keys: one slot per 16, 16-bit arrays: two) so those reads do not
    // collide in the shared-memory banks; see kpad / ipad.
    uint16_t idx[CAP + CAP / 8];                        // original position of every sorted element
    union {
        K keys[CAP + CAP / 16];                        // the sort, until the hull starts
        T vals[CAP];                                    // cluster values, after it
    } kv;
    union {
        struct {
            uint32_t whist[(wsh::NT / 32) * 256];
            uint32_t dcount[256], dstart[256];
        } sort;
        struct {
            int cnt[CAP + CAP / 16];   // bucket counts, then starts (padded like the keys: kpad)
        } bucket;
        wsh::Smem h;
        uint16_t cid_of[CAP + CAP / 8];   // cluster of every original position (after the values)
    } u;
    K kmin, kmax;
    int bmax;
    int wsumi[wsh::NT / 32];
    uint32_t starts[wsh::TILE / 32 + 1];   // bit p: a cluster starts at sorted position p
    TileScale ts;
    SegConst sc;    // the segment's global fixed-point scale (cluster values)
    int64_t t11;    // round-1 gap threshold (tile units)
    int flags, emin;
};

// Exclusive scan of one int per thread over the CTA with a single barrier:
// every thread reads the warp totals itself.  wsum (one word per warp) must
// not be written again before the next barrier of the caller.
__device__ __forceinline__ int lean_excl_scan(int v, int* wsum, int* total) {
    constexpr int NW = wsh::NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int inc = ws_warp_incl_scan<int>(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int base = 0, tot = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        const int x = wsum[k];
        base += k < w ? x : 0;
        tot += x;
    }
    *total = tot;
    return base + inc - v;
}

__device__ __forceinline__ int lean_kpad(int p) { return p + (p >> 4); }          // keys, counts
__device__ __forceinline__ int lean_ipad(int p) { return p + ((p >> 4) << 1); }   // 16-bit arrays

// The rare paths of k_small live out of line so that the common path's code
// stays compact in the instruction cache.  All threads of the CTA call each.

// LSD radix sort, 8-bit digits, of the n (key, original position) pairs in
// s.kv.keys / s.idx (any order on entry; sorted on return).  Every pass takes
// position w*32*M + k*32 + l of the previous one, which the stable ranking
// keeps in order.
template <typename T>
__device__ __noinline__ void small_radix(LeanSmem<T>& s, int n) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int NT = wsh::NT, M = wsh::M;
    const int t = threadIdx.x, l = t & 31, w = t >> 5;
    for (int pass = 0; pass < KO::BITS / 8; ++pass) {
        K key[M];
        uint16_t ii[M];
        uint32_t dg[M];
        bool valid[M];
        int pos[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const int p = w * 32 * M + k * 32 + l;
            valid[k] = p < n;
            key[k] = valid[k] ? s.kv.keys[lean_kpad(p)] : (K)0;
            ii[k] = valid[k] ? s.idx[lean_ipad(p)] : (uint16_t)0;
            dg[k] = (uint32_t)((key[k] >> (8 * pass)) & 0xff);
        }
        __syncthreads();
        ws_rank_digits<NT, M, 1>(dg, valid, pos, s.u.sort.whist, s.u.sort.dcount, s.u.sort.dstart);
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (valid[k]) { s.kv.keys[lean_kpad(pos[k])] = key[k]; s.idx[lean_ipad(pos[k])] = ii[k]; }
        __syncthreads();
    }
}

// The hull by chains and trees when the rounds hit their cap (no CTA cap:
// never fails).  Ends synchronised.
__device__ __noinline__ void small_chain_tree(wsh::Smem& h, const wsh::Test& tst, int first, int last, int n,
                                              int64_t Xf) {
    wsh::chain_tree_hull(h, tst, threadIdx.x, first, last, n, Xf, 1 << 30);
}

// Warm start: the runs of equal earlier cluster ids (low 16 bits; any values
// are valid) along the sorted order, then candidate_boundaries on the
// round-1 survivors G.  The earlier
// ids are staged by original position in `cprev` (the keys' storage: the
// keys are in registers by now).  Prefix sums of every point must be written
// (the barriers here publish them).
template <typename T>
__device__ __noinline__ uint32_t small_warm(LeanSmem<T>& s, const wsh::Test& tst, const int32_t* ids_prev,
                                            int64_t a0, int first, int n, uint32_t G) {
    constexpr int M = wsh::M;
    const int t = threadIdx.x;
    uint16_t* cprev = reinterpret_cast<uint16_t*>(s.kv.keys);
    if (first < n) {
        const int32_t* src = ids_prev + a0 + first;
        if (first + M <= n && (((uintptr_t)src) & 15) == 0) {
#pragma unroll
            for (int i = 0; i < M; i += 4) {
                const int4 q = __ldcs(reinterpret_cast<const int4*>(src + i));
                cprev[lean_ipad(first + i)] = (uint16_t)q.x;
                cprev[lean_ipad(first + i + 1)] = (uint16_t)q.y;
                cprev[lean_ipad(first + i + 2)] = (uint16_t)q.z;
                cprev[lean_ipad(first + i + 3)] = (uint16_t)q.w;
            }
        } else {
            for (int i = 0; i < M && first + i < n; ++i) cprev[lean_ipad(first + i)] = (uint16_t)src[i];
        }
    }
    __syncthreads();
    // bit i: a run starts at point first + i
    uint32_t R = 0;
    if (first < n) {
        uint16_t cp = first >= 1 ? cprev[lean_ipad(s.idx[lean_ipad(first - 1)])] : (uint16_t)0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = first + i;
            if (p < n) {
                const uint16_t c = cprev[lean_ipad(s.idx[lean_ipad(p)])];
                if (p >= 1 && c != cp) R |= 1u << i;
                cp = c;
            }
        }
    }
    return wsh::candidate_boundaries(s.u.h, tst, t, first, n, R, G);
}

template <typename T>
__global__ void __launch_bounds__(wsh::NT, sizeof(T) == 4 ? 3 : 2) k_small(const T* __restrict__ values,
                                                   const int64_t* __restrict__ offsets,
                                                   const int32_t* __restrict__ seg_list,
                                                   const double* __restrict__ lambdas, T* out, int32_t* ids,
                                                   int64_t* n_clusters, int fp64, const WsEpi ep, uint32_t* status,
                                                   int32_t* gen_list, int32_t* gen_count, int ic_cap,
                                                   const int32_t* ids_prev) {   // (may alias ids)
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    typedef LeanSmem<T> S;
    constexpr int NT = wsh::NT, M = wsh::M, CAP = S::CAP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& s = *reinterpret_cast<S*>(smem_raw);
    wsh::Smem& h = s.u.h;
    auto kpad = [](int p) { return p + (p >> 4); };          // keys
    auto ipad = [](int p) { return p + ((p >> 4) << 1); };   // 16-bit arrays
    const int t = threadIdx.x, l = t & 31, w = t >> 5;
    const int seg = seg_list[blockIdx.x];
    const int64_t a0 = offsets[seg];
    const int n = (int)(offsets[seg + 1] - a0);
    const double lam = lambdas[seg];
    if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) {
        if (t == 0) ws_flag(status, WS_STATUS_BAD_LAMBDA);
        return;
    }
    if (n <= 0 || n > CAP) {
        if (n > CAP && t == 0) ws_flag(status, WS_STATUS_INTERNAL);
        if (n == 0 && t == 0 && n_clusters) n_clusters[seg] = 0;
        return;
    }
    // ---- load this thread's 16 consecutive elements (16-byte loads when whole and aligned)
    const int first = t * M;
    K key[M];
    bool bad = false;
    int emin = 0x7fffffff;
    {
        T v[M];
        const T* src = values + a0 + first;
        if (first + M <= n && (((uintptr_t)src) & 15) == 0) {
            constexpr int NV = M * (int)sizeof(T) / 16;
            uint4 buf[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) buf[i] = __ldcs(reinterpret_cast<const uint4*>(src) + i);
            const T* bv = reinterpret_cast<const T*>(buf);
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = bv[i];
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) v[i] = (first + i < n) ? src[i] : (T)0;
        }
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (first + i < n) {
                bad |= !ws_isfinite(v[i]);
                if (v[i] != (T)0) emin = min(emin, ws_eff_exp(v[i]));
            }
            key[i] = KO::to_key(v[i]);
        }
    }
    if (t == 0) {
        s.emin = 0x7fffffff;
        s.kmin = ~(K)0;
        s.kmax = 0;
        s.bmax = 0;
    }
    if (__syncthreads_or(bad)) {
        if (t == 0) ws_flag(status, WS_STATUS_NONFINITE);
        return;
    }
    if (n == 1) {
        if (t == 0) {
            const T x = KO::from_key(key[0]);   // d = 1: no shift (the 1/(d-1) factor is vacuous)
            out[a0] = fp64 ? (T)ws_epilogue<double>((double)x, 0.0, ep.beta, ep.gamma, ep.on != 0)
                           : (T)ws_epilogue<float>((float)x, 0.0f, ep.beta_f, ep.gamma_f, ep.on != 0);
            if (ids) ids[a0] = 0;
            if (n_clusters) n_clusters[seg] = 1;
        }
        return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) emin = min(emin, __shfl_xor_sync(WS_FULL_MASK, emin, o));
    if (l == 0) atomicMin(&s.emin, emin);

    // ---- sort (key, original position).  First an interpolation bucket sort:
    // bucket(x) = floor((x - x_min) n / (x_max - x_min)) in FP32 is monotone
    // in x (every step rounds monotonically), so equal keys share a bucket and
    // sorting each bucket by key sorts the segment; for the smooth
    // distributions of weights a bucket holds a few elements.  If a bucket is
    // larger than BUCKET_MAX the segment takes the LSD radix passes instead.
    constexpr int BUCKET_MAX = 32;
    {
        K lo = ~(K)0, hi = 0;
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (first + i < n) { lo = min(lo, key[i]); hi = max(hi, key[i]); }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, ws_shfl_xor_k(lo, o));
            hi = max(hi, ws_shfl_xor_k(hi, o));
        }
        int* cnt = s.u.bucket.cnt;
        for (int i = t; i < n; i += NT) cnt[kpad(i)] = 0;
        if (l == 0) { ws_atomic_min_k(&s.kmin, lo); ws_atomic_max_k(&s.kmax, hi); }
    }
    __syncthreads();
    // ---- the fixed point of the segment, from its extreme keys (the first and
    // last sorted ones): a segment whose prefix sums need more than 64 bits
    // goes to the general kernel before any sorting
    const K kfirst = s.kmin, klast = s.kmax;
    const T xlo = KO::from_key(kfirst), xhi = KO::from_key(klast);
    const int emax = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), s.emin);
    if (t == 0) ws_note_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), s.emin, status);
    int sh;
    const bool bin = ws_tile_binade<T>(kfirst, klast, n, emax, sh);
    const int64_t q0 = ws_fixed<T>(xlo, emax);
    const uint64_t range = bin ? (uint64_t)(klast - kfirst) : (uint64_t)(ws_fixed<T>(xhi, emax) - q0);
    const bool lean = ws_lean_x(range, n);   // prefix sums in 64 bits
    const bool d64 = ws_lean_tile(range, n);  // every Delta too
    if (!lean) {   // (uniform)
        if (t == 0) gen_list[atomicAdd(gen_count, 1)] = seg;
        return;
    }
    bool radix = false;
    {
        int* cnt = s.u.bucket.cnt;
        const float f0 = (float)KO::from_key(s.kmin), f1 = (float)KO::from_key(s.kmax);
        const float span = f1 - f0;
        const float scale = (span > 0.0f && span <= 3.0e38f) ? (float)n / span : 0.0f;
        int bk[M], rk[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (first + i < n) {
                const float f = ((float)KO::from_key(key[i]) - f0) * scale;
                bk[i] = min(n - 1, max(0, (int)f));
                rk[i] = atomicAdd(&cnt[kpad(bk[i])], 1);
            }
        }
        __syncthreads();
        // bucket starts: this thread's 16 consecutive buckets, then the CTA scan
        int c[M], sum = 0, big = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            c[i] = (first + i < n) ? cnt[kpad(first + i)] : 0;
            sum += c[i];
            big = max(big, c[i]);
        }
        int tot;
        int run = lean_excl_scan(sum, s.wsumi, &tot);
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (first + i < n) { cnt[kpad(first + i)] = run; run += c[i]; }
        radix = __syncthreads_or(big > BUCKET_MAX);
        if (!radix) {
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (first + i < n) {
                    const int pp = cnt[kpad(bk[i])] + rk[i];
                    s.kv.keys[kpad(pp)] = key[i];
                    s.idx[ipad(pp)] = (uint16_t)(first + i);
                }
            __syncthreads();
            // each bucket by key (ties may end in any order): up to four
            // elements by a sorting network in registers, larger buckets by
            // insertion in shared memory.  Bucket ends from the starts (no
            // indexing of c[] by a loop variable: it would live in local memory).
            uint32_t multi = 0;
#pragma unroll
            for (int i = 0; i < M; ++i)
                if (first + i < n && c[i] >= 2) multi |= 1u << i;
            while (multi) {
                const int i = __ffs((int)multi) - 1;
                multi &= multi - 1;
                const int b0 = cnt[kpad(first + i)];
                const int b1 = first + i + 1 < n ? cnt[kpad(first + i + 1)] : n;
                if (b1 - b0 <= 4) {
                    K k[4];
                    uint16_t x[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = b0 + j < b1;
                        k[j] = in ? s.kv.keys[kpad(b0 + j)] : ~(K)0;
                        x[j] = in ? s.idx[ipad(b0 + j)] : (uint16_t)0;
                    }
                    auto cs = [&](int a, int b) {
                        const bool sw = k[a] > k[b];
                        const K ka = sw ? k[b] : k[a], kb = sw ? k[a] : k[b];
                        const uint16_t xa = sw ? x[b] : x[a], xb = sw ? x[a] : x[b];
                        k[a] = ka; k[b] = kb; x[a] = xa; x[b] = xb;
                    };
                    cs(0, 1); cs(2, 3); cs(0, 2); cs(1, 3); cs(1, 2);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (b0 + j < b1) { s.kv.keys[kpad(b0 + j)] = k[j]; s.idx[ipad(b0 + j)] = x[j]; }
                    continue;
                }
                for (int a = b0 + 1; a < b1; ++a) {
                    const K kk = s.kv.keys[kpad(a)];
                    const uint16_t ii = s.idx[ipad(a)];
                    int j = a - 1;
                    while (j >= b0 && s.kv.keys[kpad(j)] > kk) {
                        s.kv.keys[kpad(j + 1)] = s.kv.keys[kpad(j)];
                        s.idx[ipad(j + 1)] = s.idx[ipad(j)];
                        --j;
                    }
                    s.kv.keys[kpad(j + 1)] = kk;
                    s.idx[ipad(j + 1)] = ii;
                }
            }
            __syncthreads();
        }
    }
    // ---- otherwise: LSD radix sort, 8-bit digits (out of line)
    if (radix) {
#pragma unroll
        for (int k = 0; k < M; ++k)
            if (first + k < n) { s.kv.keys[kpad(first + k)] = key[k]; s.idx[ipad(first + k)] = (uint16_t)(first + k); }
        __syncthreads();
        small_radix<T>(s, n);
    }

    // ---- the sorted segment as one hull tile: this thread's 16 sorted keys
    K kr[M];
#pragma unroll
    for (int i = 0; i < M; ++i) kr[i] = (first + i < n) ? s.kv.keys[kpad(first + i)] : s.kv.keys[0];
    const K kprev = (t > 0 && first < n) ? s.kv.keys[kpad(first - 1)] : kfirst;
    if (t == 0) {   // (no FP64 on this critical path)
        s.sc = ws_seg_const_f(n, lam, KO::L_BASE - emax, fp64 != 0);
        TileScale& ts = s.ts;
        ts.sc = bin ? ws_seg_const_f(n, lam, s.sc.L - sh, false) : s.sc;
        bool f;
        ts.muq = ws_muq_f(ts.sc, f);
        ts.fast = f ? 1 : 0;
        if (ts.sc.mlam == 0) { ts.modd = 0; ts.sodd = 0; }
        else { const int tz = __ffsll((long long)ts.sc.mlam) - 1; ts.modd = ts.sc.mlam >> tz; ts.sodd = ts.sc.s + tz; }
        // lower bound of floor(2 mu) (muq is within 1e-6 relative of mu)
        const float m2 = 2.0f * ts.muq * (1.0f - 1.0e-6f);
        s.t11 = !f ? (int64_t)-1 : (m2 < 3.9e18f ? (int64_t)floorf(m2) - 1 : (int64_t)3.9e18);
        h.general = 0;
    }
    auto devk = [&](K k) -> int64_t {
        return bin ? (int64_t)(k - kfirst) : ws_fixed<T>(KO::from_key(k), emax) - q0;
    };
    auto dev = [&](int i) -> int64_t { return devk(kr[i]); };
    // the deviations, once: their running sums (this lane's prefix sums
    // relative to its first point) go straight into the prefix-sum slots (the
    // sort's scratch is dead); the lane's offset is added below
    int64_t csum = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (first + i < n) {
            csum += dev(i);
            wsh::xref(h, first + i + 1) = csum;
        }
    const int64_t winc = ws_warp_incl_scan<long long>((long long)csum);
    if (l == 31) h.wtot[w] = winc;
    if (t == 0) wsh::xref(h, 0) = 0;
    __syncthreads();
    int64_t wbase = 0;
    for (int k = 0; k < w; ++k) wbase += h.wtot[k];
    const int64_t Xf = wbase + winc - csum;
    const int last = min(first + M, n);
    wsh::Test tst;
    tst.sc = s.ts.sc;
    tst.P.s64 = nullptr;
    tst.P.muq = s.ts.muq;
    tst.P.fast = s.ts.fast != 0;
    tst.P.d64 = d64;
    tst.P.thr = nullptr;
    tst.P.modd = s.ts.modd;
    tst.P.sodd = s.ts.sodd;
    // round 1 of the Imminent Collisions rounds: point p stays a boundary iff
    // y_{p-1} < y_p, i.e. the gap x_p - x_{p-1} exceeds 2 lambda/(d-1) = 2 mu.
    // t11 is a lower bound of floor(2 mu) in tile units, so a few points at
    // the threshold may stay too: a superset of the hull vertices is all the
    // rounds need (their first round tests every boundary exactly).  Warm:
    // of these, the candidate's run boundaries and the points below their
    // run's chord.
    // (with the lane's offset added to its prefix sums)
    uint32_t B = 0;
    if (first < n) {
        const int64_t t11 = s.t11;
        int64_t dprev = devk(kprev), prevX = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = first + i;
            if (p < n) {
                int64_t& slot = wsh::xref(h, p + 1);
                const int64_t Xl = slot;
                const int64_t di = Xl - prevX;   // the deviation of element p
                prevX = Xl;
                slot = Xl + Xf;
                if (p >= 1 && di - dprev > t11) B |= 1u << i;
                dprev = di;
            }
        }
    }
    if (ids_prev) B = small_warm<T>(s, tst, ids_prev, a0, first, n, B);
    int rounds = 0;
    bool converged = false;
    if (ic_cap > 0) converged = wsh::ic_rounds(h, tst, t, first, n, B, ic_cap, rounds);
    uint16_t* st16 = reinterpret_cast<uint16_t*>(s.starts);
    if (converged) {
        st16[t] = (uint16_t)(B | (t == 0 ? 1u : 0u));
    } else {
        small_chain_tree(h, tst, first, last, n, Xf);
        st16[t] = 0;
        __syncthreads();
        for (int k = h.lo[t]; k < (int)h.hi[t]; ++k) {
            const int p = h.st[k * NT + t];
            if (p < n) atomicOr(&s.starts[p >> 5], 1u << (p & 31));
        }
    }
    __syncthreads();
    // ---- cluster ids: rank of every start; values of the clusters this thread starts
    const uint32_t mine = (uint32_t)st16[t] & (first < n ? (n - first >= M ? 0xffffu : ((1u << (n - first)) - 1u)) : 0u);
    int C;
    const int base = lean_excl_scan(__popc(mine), h.wsum, &C);
    const float x0f = (float)xlo;
    {
        uint32_t rest = mine;
        int r = base;
        while (rest) {
            const int i = __ffs((int)rest) - 1;
            rest &= rest - 1;
            const int a = first + i;
            // end of the cluster: the next start (in this thread, else the next set bit of the bitmap), or n
            int b = n;
            if (rest) b = first + __ffs((int)rest) - 1;
            else {
                for (int wd = (first + M) >> 5; (wd << 5) < n; ++wd) {
                    uint32_t bits = s.starts[wd];
                    if ((wd << 5) < first + M) bits &= 0xffffffffu << ((first + M) & 31);
                    if (bits) { b = min((wd << 5) + __ffs((int)bits) - 1, n); break; }
                }
            }
            const int64_t xd = wsh::xat(h, b) - wsh::xat(h, a);
            K ki = kr[0];   // kr[i] by selects (a loop-variable index would put kr in local memory)
#pragma unroll
            for (int j = 1; j < M; ++j) ki = (i == j) ? kr[j] : ki;
            if (KO::BITS == 32 && !fp64) {
                // FP32: mean = x_0 + (deviation sum / count) in tile units; every
                // term exact but the conversions (a few FP32 ulps of max |w|)
                const float xa = (float)KO::from_key(ki);
                const float mean = (b - a == 1) ? xa
                                                : x0f + ldexpf(ws_u64_to_float((uint64_t)xd) / (float)(b - a), -s.ts.sc.L);
                s.kv.vals[r] = (T)ws_epilogue<float>(mean, s.sc.mu_f * (float)(n - a - b), ep.beta_f, ep.gamma_f,
                                                     ep.on != 0);
            } else {
                const i128 SX = (i128)(b - a) * (i128)q0 + (bin ? ((i128)xd << sh) : (i128)xd);
                s.kv.vals[r] = ValueOut<T>::value(SX, a, b, KO::from_key(ki), s.sc, fp64 != 0, ep);
            }
            ++r;
        }
    }
    __syncthreads();   // (the prefix sums are dead: their storage takes the cluster of every position)
    // ---- the cluster of every original position, then this thread's 16
    // consecutive outputs (coalesced stores)
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const int p = first + i;
        if (p < n) s.u.cid_of[ipad(s.idx[ipad(p)])] = (uint16_t)(base + __popc(mine & ((2u << i) - 1u)) - 1);
    }
    __syncthreads();
    if (first < n) {
        T ov[M];
        int32_t oi[M];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int c = (first + i < n) ? (int)s.u.cid_of[ipad(first + i)] : 0;
            oi[i] = c;
            ov[i] = s.kv.vals[c];
        }
        T* od = out + a0 + first;
        int32_t* id = ids ? ids + a0 + first : nullptr;
        if (first + M <= n && (((uintptr_t)od) & 15) == 0 && (!id || (((uintptr_t)id) & 15) == 0)) {
            constexpr int VT = 16 / (int)sizeof(T);
#pragma unroll
            for (int i = 0; i < M; i += VT) __stcs(reinterpret_cast<uint4*>(od + i), *reinterpret_cast<const uint4*>(ov + i));
            if (id) {
#pragma unroll
                for (int i = 0; i < M; i += 4) __stcs(reinterpret_cast<uint4*>(id + i), *reinterpret_cast<const uint4*>(oi + i));
            }
        } else {
            for (int i = 0; i < M && first + i < n; ++i) {
                od[i] = ov[i];
                if (id) id[i] = oi[i];
            }
        }
    }
    if (t == 0 && n_clusters) n_clusters[seg] = C;
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t ws_launch_small(const T* values, const int64_t* offsets, const int32_t* seg_list, int n_list,
                            const double* lambdas, T* out, int32_t* ids, int64_t* n_clusters, int fp64,
                            const WsEpi& ep, uint32_t* status, cudaStream_t st, WsProf* prof, int32_t* gen_list,
                            int32_t* gen_count, int ic_cap, const int32_t* ids_prev) {
    constexpr int NT = 256;
    constexpr int M = SmallCfg<T>::M;
    if (n_list <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(gen_count, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(LeanSmem<T>);
    e = cudaFuncSetAttribute(k_small<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    WS_LAUNCH(prof, WSK_SMALL, st,
              (k_small<T><<<n_list, NT, smem, st>>>(values, offsets, seg_list, lambdas, out, ids, n_clusters, fp64, ep,
                                                    status, gen_list, gen_count, ic_cap, ids_prev)));
    // the segments the lean kernel passed on (none on ordinary inputs): a
    // small grid that walks the list
    const size_t gsmem = sizeof(SmallSmem<T, NT, M>);
    auto gk = k_small_general<T, NT, M>;
    e = cudaFuncSetAttribute(gk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsmem);
    if (e != cudaSuccess) return e;
    WS_LAUNCH(prof, WSK_SMALL, st,
              (gk<<<n_list < 456 ? n_list : 456, NT, gsmem, st>>>(values, offsets, gen_list, gen_count, lambdas, out, ids,
                                                               n_clusters, fp64, ep, status)));
    return cudaGetLastError();
}

template cudaError_t ws_launch_small<float>(const float*, const int64_t*, const int32_t*, int, const double*, float*,
                                            int32_t*, int64_t*, int, const WsEpi&, uint32_t*, cudaStream_t, WsProf*,
                                            int32_t*, int32_t*, int, const int32_t*);
template cudaError_t ws_launch_small<double>(const double*, const int64_t*, const int32_t*, int, const double*,
                                             double*, int32_t*, int64_t*, int, const WsEpi&, uint32_t*, cudaStream_t,
                                             WsProf*, int32_t*, int32_t*, int, const int32_t*);
