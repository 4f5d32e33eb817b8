// ws_small.cu -- fused single-CTA prox for short segments (n <= 4096 for
// float, 2048 for double): one CTA loads a segment once, sorts (key, index)
// pairs in shared memory, builds the exact hull, and writes values and cluster
// ids straight to their original positions.  HBM traffic is the I/O floor:
// read w, write out and id (12 B/element for float).
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

template <typename T, int NT, int M>
__global__ void __launch_bounds__(NT, 3) k_small(const T* __restrict__ values, const int64_t* __restrict__ offsets,
                                              const int32_t* __restrict__ seg_list, const double* __restrict__ lambdas,
                                              T* out, int32_t* ids, int64_t* n_clusters, int fp64,
                                              const WsEpi ep, uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    typedef SmallSmem<T, NT, M> S;
    constexpr int CAP = S::CAP;
    constexpr int ITEMS = M;   // items per thread in the sort
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& s = *reinterpret_cast<S*>(smem_raw);
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;

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

// Backward for short segments: per-cluster mean of grad_out (shared-memory sums).
template <typename T, int NT, int CAP>
__global__ void __launch_bounds__(NT) k_small_backward(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                       const int64_t* __restrict__ offsets,
                                                       const int32_t* __restrict__ seg_list, T* gin,
                                                       uint32_t* status) {
    __shared__ T sum[CAP];
    __shared__ int cnt[CAP];
    const int seg = seg_list[blockIdx.x];
    const int64_t a0 = offsets[seg];
    const int n = (int)(offsets[seg + 1] - a0);
    if (n <= 0) return;
    if (n > CAP) { if (threadIdx.x == 0) ws_flag(status, WS_STATUS_INTERNAL); return; }
    for (int i = threadIdx.x; i < n; i += NT) { sum[i] = (T)0; cnt[i] = 0; }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NT) {
        int id = ids[a0 + i];
        if (id < 0 || id >= n) { ws_flag(status, WS_STATUS_INTERNAL); continue; }
        atomicAdd(&sum[id], g[a0 + i]);
        atomicAdd(&cnt[id], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += NT) {
        int id = ids[a0 + i];
        if (id >= 0 && id < n) gin[a0 + i] = sum[id] / (T)cnt[id];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t ws_launch_small(const T* values, const int64_t* offsets, const int32_t* seg_list, int n_list,
                            const double* lambdas, T* out, int32_t* ids, int64_t* n_clusters, int fp64,
                            const WsEpi& ep, uint32_t* status, cudaStream_t st, WsProf* prof) {
    constexpr int NT = 256;
    constexpr int M = SmallCfg<T>::M;
    if (n_list <= 0) return cudaSuccess;
    size_t smem = sizeof(SmallSmem<T, NT, M>);
    auto kern = k_small<T, NT, M>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    WS_LAUNCH(prof, WSK_SMALL, st,
              (kern<<<n_list, NT, smem, st>>>(values, offsets, seg_list, lambdas, out, ids, n_clusters, fp64, ep,
                                              status)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t ws_launch_small_backward(const T* g, const int32_t* ids, const int64_t* offsets, const int32_t* seg_list,
                                     int n_list, T* gin, uint32_t* status, cudaStream_t st, WsProf* prof) {
    constexpr int NT = 256;
    if (n_list <= 0) return cudaSuccess;
    WS_LAUNCH(prof, WSK_BWD, st,
              (k_small_backward<T, NT, SmallCfg<T>::CAP><<<n_list, NT, 0, st>>>(g, ids, offsets, seg_list, gin, status)));
    return cudaGetLastError();
}

template cudaError_t ws_launch_small<float>(const float*, const int64_t*, const int32_t*, int, const double*, float*,
                                            int32_t*, int64_t*, int, const WsEpi&, uint32_t*, cudaStream_t, WsProf*);
template cudaError_t ws_launch_small<double>(const double*, const int64_t*, const int32_t*, int, const double*,
                                             double*, int32_t*, int64_t*, int, const WsEpi&, uint32_t*, cudaStream_t,
                                             WsProf*);
template cudaError_t ws_launch_small_backward<float>(const float*, const int32_t*, const int64_t*, const int32_t*,
                                                     int, float*, uint32_t*, cudaStream_t, WsProf*);
template cudaError_t ws_launch_small_backward<double>(const double*, const int32_t*, const int64_t*,
                                                      const int32_t*, int, double*, uint32_t*, cudaStream_t, WsProf*);
