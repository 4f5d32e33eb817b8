// ws_block.cuh -- CTA-level building blocks: scans, stable digit ranking, and
// the exact lower hull of a tile of points (the in-CTA cluster merge).
#pragma once
#include "ws_common.cuh"

#define WS_FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// Scans
// ---------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V ws_shfl_up(V v, int delta);
template <> __device__ __forceinline__ int ws_shfl_up<int>(int v, int delta) {
    return __shfl_up_sync(WS_FULL_MASK, v, delta);
}
template <> __device__ __forceinline__ long long ws_shfl_up<long long>(long long v, int delta) {
    return __shfl_up_sync(WS_FULL_MASK, v, delta);
}
template <> __device__ __forceinline__ i128 ws_shfl_up<i128>(i128 v, int delta) {
    long long lo = (long long)(uint64_t)v, hi = (long long)(uint64_t)(v >> 64);
    lo = __shfl_up_sync(WS_FULL_MASK, lo, delta);
    hi = __shfl_up_sync(WS_FULL_MASK, hi, delta);
    return (i128)(((u128)(uint64_t)hi << 64) | (u128)(uint64_t)lo);
}

// Butterfly shuffle of a sort key (32 or 64 bits).
__device__ __forceinline__ uint32_t ws_shfl_xor_k(uint32_t v, int o) { return __shfl_xor_sync(WS_FULL_MASK, v, o); }
__device__ __forceinline__ uint64_t ws_shfl_xor_k(uint64_t v, int o) {
    return (uint64_t)__shfl_xor_sync(WS_FULL_MASK, (unsigned long long)v, o);
}

__device__ __forceinline__ void ws_atomic_min_k(uint32_t* p, uint32_t v) { atomicMin(p, v); }
__device__ __forceinline__ void ws_atomic_max_k(uint32_t* p, uint32_t v) { atomicMax(p, v); }
__device__ __forceinline__ void ws_atomic_min_k(uint64_t* p, uint64_t v) {
    atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ void ws_atomic_max_k(uint64_t* p, uint64_t v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}

template <typename V> __device__ __forceinline__ V ws_warp_incl_scan(V v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V t = ws_shfl_up<V>(v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Warp sum of a 128-bit integer (every lane gets it).
__device__ __forceinline__ i128 ws_warp_reduce_i128(i128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const long long lo = __shfl_xor_sync(WS_FULL_MASK, (long long)(uint64_t)v, o);
        const long long hi = __shfl_xor_sync(WS_FULL_MASK, (long long)(uint64_t)((u128)v >> 64), o);
        v += (i128)(((u128)(uint64_t)hi << 64) | (u128)(uint64_t)lo);
    }
    return v;
}

// Block exclusive scan; returns the exclusive prefix, *total gets the sum.
// `wsum` is NT/32 elements of shared scratch.  Contains __syncthreads.
template <int NT, typename V>
__device__ __forceinline__ V ws_block_excl_scan(V v, V* wsum, V* total) {
    constexpr int NW = NT / 32;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    V inc = ws_warp_incl_scan<V>(v);
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    if (w == 0) {
        V s = (lane < NW) ? wsum[lane] : (V)0;
        s = ws_warp_incl_scan<V>(s);
        if (lane < NW) wsum[lane] = s;
    }
    __syncthreads();
    V base = (w > 0) ? wsum[w - 1] : (V)0;
    if (total) *total = wsum[NW - 1];
    V r = base + inc - v;
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// Fixed-point prefix sums of a sorted tile (points 0..n).
// Per-point arrays are stored at padded index p + p/M so that the threads of
// a warp, which own consecutive chunks of M points, hit distinct banks.
// Narrow tiles (n * (q_{n-1} - q_0) <= 2^62) store D_p = sum_{j<p} (q_j - q_0)
// in s64; wide tiles store the chunk-relative prefix in s64 and the chunk
// starts in base (128-bit).  Returns true for a narrow tile.  Contains
// __syncthreads; ends synchronised.
// ---------------------------------------------------------------------------
template <int M> __device__ __forceinline__ int ws_sidx(int p) { return p + p / M; }

template <int NT, int M>
struct TilePrefix {
    int64_t s64[NT * M + 1 + NT + 1];
    i128 base[NT + 1];
    i128 wsum128[NT / 32];
    long long wsum64[NT / 32];
};

// Representation of a tile's prefix sums.
enum { WS_TILE_WIDE = 0, WS_TILE_NARROW = 1, WS_TILE_BINADE = 2 };

// Is a tile with first/last keys k0, kn (n elements) a BINADE tile, and the
// binade's shift sh against the segment scale (see ws_tile_prefix)?
template <typename T>
__device__ __forceinline__ bool ws_tile_binade(typename KeyOf<T>::K k0, typename KeyOf<T>::K kn, int n, int emax,
                                               int& sh) {
    typedef KeyOf<T> KO;
    sh = ws_eff_exp(KO::from_key(k0)) - emax + KO::FIX_OFS;
    const bool same_binade = ((k0 ^ kn) >> KO::MANT) == 0 && sh >= 0;
    return same_binade && (uint64_t)(kn - k0) <= ((uint64_t)1 << 62) / (uint64_t)n;
}

// kr[i] = key of sorted element first + i (first = threadIdx.x * M); k0, kn =
// keys of elements 0 and n - 1.  Modes:
//   BINADE: all keys share sign and exponent, so key - k0 is the value
//           difference in ulps of that binade, exactly; s64 holds prefix sums
//           of (key - k0) in ulp units; one ulp = 2^sh global fixed-point units
//           (sh >= 0 is required: otherwise the global image truncates).
//   NARROW: s64 holds D_p = sum (q_j - q_0) in global units.
//   WIDE:   s64 holds chunk-relative prefixes, base[] the chunk starts (128-bit).
// q0_out = global fixed-point image of element 0; total_out = X_n (global).
// thr_dst/thr_val: an optional shared-memory store that is issued after the
// prefix's first barrier (so it may overwrite storage that was read before
// the call) and is visible to every thread on return.
template <typename T, int NT, int M>
__device__ int ws_tile_prefix(TilePrefix<NT, M>& tp, const typename KeyOf<T>::K (&kr)[M], typename KeyOf<T>::K k0,
                              typename KeyOf<T>::K kn, int n, int emax, int64_t& q0_out, i128& total_out,
                              int& binade_sh, int* thr_dst = nullptr, int thr_val = 0) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int CAP = NT * M;
    const int t = threadIdx.x;
    const int first = t * M;
    const T x0 = KO::from_key(k0);
    const int64_t q0 = ws_fixed<T>(x0, emax);
    q0_out = q0;
    int sh;
    const bool binade = ws_tile_binade<T>(k0, kn, n, emax, sh);
    int mode;
    if (binade) {
        mode = WS_TILE_BINADE;
    } else {
        const int64_t qn = ws_fixed<T>(KO::from_key(kn), emax);
        mode = ((uint64_t)(qn - q0) <= ((uint64_t)1 << 62) / (uint64_t)n) ? WS_TILE_NARROW : WS_TILE_WIDE;
    }
    binade_sh = sh;
    long long run = 0;
    long long dq_last = 0;   // narrow: the chunk's last deviation (the others wait in s64, see below)
    if (mode == WS_TILE_BINADE) {
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (first + i < n) run += (long long)(kr[i] - k0);
    } else if (mode == WS_TILE_NARROW) {
        // deviation of element first+i parked at point first+i+1 of this chunk
        // (overwritten by the prefix only after it has been read back)
#pragma unroll
        for (int i = 0; i < M; ++i) {
            if (first + i < n) {
                const long long dq = ws_fixed<T>(KO::from_key(kr[i]), emax) - q0;
                run += dq;
                if (i + 1 < M) tp.s64[ws_sidx<M>(first + i + 1)] = dq;
                else dq_last = dq;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < M; ++i)
            if (first + i < n) run += ws_fixed<T>(KO::from_key(kr[i]), emax);
    }
    if (mode != WS_TILE_WIDE) {
        long long tot;
        long long acc = ws_block_excl_scan<NT, long long>(run, tp.wsum64, &tot);
        if (thr_dst) *thr_dst = thr_val;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = first + i;
            long long dq = 0;
            if (mode == WS_TILE_BINADE) dq = (long long)(kr[i] - k0);
            else if (p < n) dq = (i + 1 < M) ? tp.s64[ws_sidx<M>(p + 1)] : dq_last;
            if (p <= n) tp.s64[ws_sidx<M>(p)] = acc;
            if (p < n) acc += dq;
        }
        if (t == 0 && n == CAP) tp.s64[ws_sidx<M>(CAP)] = tot;
        total_out = (mode == WS_TILE_BINADE) ? (i128)n * (i128)q0 + ((i128)tot << sh)
                                             : (i128)tot + (i128)n * (i128)q0;
    } else {
        i128 tot;
        const i128 ex = ws_block_excl_scan<NT, i128>((i128)run, tp.wsum128, &tot);
        if (thr_dst) *thr_dst = thr_val;
        long long acc = 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = first + i;
            if (p <= n) tp.s64[ws_sidx<M>(p)] = acc;
            if (p < n) acc += ws_fixed<T>(KO::from_key(kr[i]), emax);
        }
        tp.base[t] = ex;
        if (t == 0) { tp.base[NT] = tot; if (n == CAP) tp.s64[ws_sidx<M>(CAP)] = 0; }
        total_out = tot;
    }
    __syncthreads();
    return mode;
}

// Global fixed-point prefix X_p for any tile mode.
template <int M>
__device__ __forceinline__ i128 ws_tile_X(const int64_t* s64, const i128* base, int mode, int64_t q0, int sh, int p) {
    const int64_t v = s64[ws_sidx<M>(p)];
    if (mode == WS_TILE_BINADE) return (i128)p * (i128)q0 + ((i128)v << sh);
    if (mode == WS_TILE_NARROW) return (i128)p * (i128)q0 + (i128)v;
    return base[p / M] + (i128)v;
}

// lambda * 2^L / (d - 1) as float for the FP32 filter; usable if finite and
// small enough that muq * (c - a) * n1 * n2 stays far from overflow.
__device__ __forceinline__ float ws_muq(double lam, const SegConst& sc, bool& usable) {
    double m = (sc.d > 1) ? ldexp(lam, sc.L) / (double)(sc.d - 1) : 0.0;
    usable = (m == m) && m < 1.0e26;
    return usable ? (float)m : 0.0f;
}

// ---------------------------------------------------------------------------
// Stable ranking of a CTA's keys by one 8-bit digit.
// Arrangement: warp w owns positions [w*32*ITEMS, (w+1)*32*ITEMS); item k of
// lane l is position w*32*ITEMS + k*32 + l.  The warp's items are split into
// NC contiguous runs ("chains") of ITEMS/NC items; each chain keeps its own
// digit counters, so the NC read-modify-write chains through shared memory
// are independent and overlap.  Within a chain, processing items in order
// and lanes in order (peer mask + popc) visits positions in order; chains
// and warps are combined in position order, so the ranking is stable.
// Returns, per item, the position of the key in the digit-sorted tile;
// digit_count/digit_start (shared, 256 entries) receive the tile histogram
// and its exclusive scan.  whist: shared [NT/32][NC][256] uint32.
// ---------------------------------------------------------------------------
// Lanes of the warp holding the same 8-bit digit (valid lanes only), built
// from eight ballots; measured faster than __match_any_sync on sm_103a.
__device__ __forceinline__ unsigned ws_peers8(uint32_t dg, bool valid) {
    unsigned m = __ballot_sync(WS_FULL_MASK, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const unsigned bal = __ballot_sync(WS_FULL_MASK, (dg >> b) & 1u);
        m &= ((dg >> b) & 1u) ? bal : ~bal;
    }
    return m;
}

template <int NT, int ITEMS, int NC>
__device__ __forceinline__ void ws_rank_digits(const uint32_t (&dig)[ITEMS], const bool (&valid)[ITEMS],
                                               int (&pos)[ITEMS], uint32_t* whist, uint32_t* digit_count,
                                               uint32_t* digit_start) {
    static_assert(ITEMS % NC == 0, "items must split evenly into chains");
    constexpr int NW = NT / 32, IPC = ITEMS / NC;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* my = whist + w * NC * 256;
    for (int i = lane; i < NC * 256; i += 32) my[i] = 0;
    __syncwarp();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int st = 0; st < IPC; ++st) {
        unsigned peers[NC];
        int before[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int k = c * IPC + st;
            peers[c] = ws_peers8(dig[k], valid[k]);
            before[c] = valid[k] ? (int)my[c * 256 + dig[k]] : 0;
        }
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int k = c * IPC + st;
            if (valid[k]) {
                const int r = __popc(peers[c] & lt);
                pos[k] = before[c] + r;
                if (r == 0) my[c * 256 + dig[k]] = (uint32_t)(before[c] + __popc(peers[c]));
            } else {
                pos[k] = -1;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive scan across (warp, chain) in position order, tile count
    for (int dgt = threadIdx.x; dgt < 256; dgt += NT) {
        uint32_t run = 0;
        for (int ww = 0; ww < NW * NC; ++ww) {
            const uint32_t c = whist[ww * 256 + dgt];
            whist[ww * 256 + dgt] = run;
            run += c;
        }
        digit_count[dgt] = run;
    }
    __syncthreads();
    // exclusive scan over the 256 digits
    if (threadIdx.x < 32) {
        uint32_t v[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { v[i] = digit_count[lane * 8 + i]; sum += v[i]; }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t tt = __shfl_up_sync(WS_FULL_MASK, inc, o);
            if (lane >= o) inc += tt;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) { digit_start[lane * 8 + i] = run; run += v[i]; }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (valid[k]) pos[k] += (int)(digit_start[dig[k]] + whist[(w * NC + k / IPC) * 256 + dig[k]]);
}

// ---------------------------------------------------------------------------
// Exact lower hull of a tile of points (the in-CTA merge).
//
// Points p = 0..n (n elements), X(p) = fixed-point prefix sum up to p.  Thread
// t owns "chunk" t = points [t*M, min((t+1)*M, n)] (consecutive chunks share
// their end point).  Each thread builds the hull of its chunk with the
// sequential monotone chain (the stack form of pool-adjacent-violators), then
// chunks are merged pairwise up a binary tree; merging two adjacent hulls
// keeps a prefix of the left one and a suffix of the right one, joined by the
// bridge (the common lower tangent), so every chunk just narrows the range
// [lo, hi) of its own vertex list that survives.  The bridge search is the
// divide-and-conquer step of Search Collisions (Sec. 4.3, Thm 4.2) re-derived
// as a tangent search on convex chains.
// ---------------------------------------------------------------------------
template <int NT, int M>
struct HullSmem {
    uint16_t H[(M + 1) * NT];   // chunk hull lists, transposed: entry k of chunk c at k*NT + c
    uint16_t lo[NT], hi[NT];    // surviving range of each list
    int cum[NT + 1];            // exclusive scan of surviving counts (warp- or CTA-relative)
    int wtot[NT / 32];          // per-warp totals during the warp levels
    int res_i[NT], res_j[NT];
    int wsum_i[NT / 32];
    int thr[M * M];             // chain thresholds (ws_thr_entry), indexed n1 * M + n2
};

// ---------------------------------------------------------------------------
// The hull test on tile-local points.
//
// Wide tiles (prefix sums that need 128 bits): the exact integer test only.
// Binade and narrow tiles (64-bit deviations from the tile's first point)
// use TilePtsDev below.
// ---------------------------------------------------------------------------
static __device__ __noinline__ bool ws_convex_exact(i128 Xa, i128 Xb, i128 Xc, int a, int b, int c,
                                                    const SegConst& sc) {
    return ws_convex(Xa, Xb, Xc, a, b, c, sc);
}

template <int M>
struct TilePtsWide {
    static constexpr bool kThr = false;   // no chain thresholds
    const int64_t* s64;   // chunk-relative prefix sums
    const i128* base;     // prefix sum at each chunk start
    __device__ __forceinline__ int64_t v(int p) const { return s64[ws_sidx<M>(p)]; }
    __device__ __forceinline__ i128 Xv(int p, int64_t vp) const { return base[p / M] + (i128)vp; }
    __device__ __forceinline__ bool convex_v(int a, int64_t va, int b, int64_t vb, int c, int64_t vc,
                                             const SegConst& sc) const {
        return ws_convex_exact(Xv(a, va), Xv(b, vb), Xv(c, vc), a, b, c, sc);
    }
    __device__ __forceinline__ bool convex(int a, int b, int c, const SegConst& sc) const {
        return convex_v(a, v(a), b, v(b), c, v(c), sc);
    }
};

// Exact test for tiles inside one binade.  s64 holds prefix sums of ulp
// deviations, so A, B are 64-bit integers and Delta = B n1 - A n2 is exact in
// 128 bits; Delta (d-1) is compared with mlam (c-a) n1 n2 2^s by bit length,
// then by aligned 128-bit magnitudes -- no rounding anywhere.
static __device__ __noinline__ bool ws_convex_binade_exact(int64_t A, int64_t B, int64_t n1, int64_t n2,
                                                           int64_t cma, const SegConst& sc) {
    const i128 D = (i128)B * (i128)n1 - (i128)A * (i128)n2;
    if (D <= 0) return false;
    if (sc.mlam == 0) return true;
    const u128 Lv = (u128)D * (u128)sc.dm1;
    const u128 Rv = (u128)sc.mlam * (u128)((uint64_t)cma * (uint64_t)(n1 * n2));
    const int bl = ws_bitlen128(Lv), br = ws_bitlen128(Rv);
    const int s = sc.s;
    const int el = bl + (s < 0 ? -s : 0), er = br + (s > 0 ? s : 0);
    if (el != er) return el > er;
    return (Lv << (128 - bl)) > (Rv << (128 - br));
}

// Tiles whose prefix sums are 64-bit deviations: binade tiles (ulps from the
// first key, scale of the tile) and narrow tiles (q - q_0, scale of the
// segment).  When range * n^2 <= 2^62 (every FP32 binade tile), Delta =
// B n1 - A n2 is exact in 64 bits and only the right-hand side mu (c-a) n1 n2
// is rounded, so the FP32 filter's error is relative to |Delta| + rhs rather
// than to the cancelling terms B n1 and A n2: converting Delta > 0 costs <= 3
// roundings (2^-24 each), mu, the product and the multiply add <= 4 to rhs,
// the subtraction one more, < 3.1e-7 (Delta + rhs) in all; the 6e-7 margin
// covers that.  Otherwise (FP64 keys spread over a wide range) the
// filter runs on the rounded terms.  Near-ties fall through to
// the exact integer test.
template <int M>
struct TilePtsDev {
    static constexpr bool kThr = true;    // may carry chain thresholds
    const int64_t* s64;
    float muq;       // lambda 2^L_tile / (d - 1)
    bool fast;
    bool d64;        // range * n^2 <= 2^62: Delta is exact in 64 bits
    const int* thr;  // chain thresholds (ws_thr_entry) or null
    uint64_t modd;   // lambda 2^L_tile = modd * 2^sodd with modd odd (0 if lambda = 0)
    int sodd;
    __device__ __forceinline__ int64_t v(int p) const { return s64[ws_sidx<M>(p)]; }
    // Exact test Delta (d-1) > modd K 2^sodd for Delta > 0 when both sides fit
    // in 63 bits (the usual near-tie: lambda 2^L / (d-1) close to a short
    // dyadic number); 1 = convex, 0 = not, -1 = too wide here.
    __device__ __forceinline__ int near_tie64(int64_t D, uint64_t K, const SegConst& sc) const {
        const uint64_t Lh = __umul64hi((uint64_t)D, sc.dm1), Ll = (uint64_t)D * sc.dm1;
        const uint64_t Rh = __umul64hi(modd, K), Rl = modd * K;
        if (Lh != 0 || Rh != 0 || (Ll >> 63) != 0 || (Rl >> 63) != 0) return -1;
        if (sodd >= 0) {
            if (sodd > 62 || (Rl >> (63 - sodd)) != 0) return -1;
            return Ll > (Rl << sodd) ? 1 : 0;
        }
        if (-sodd > 62 || (Ll >> (63 + sodd)) != 0) return -1;
        return (Ll << -sodd) > Rl ? 1 : 0;
    }
    __device__ __forceinline__ bool convex_v(int a, int64_t va, int b, int64_t vb, int c, int64_t vc,
                                             const SegConst& sc) const {
        const int64_t A = vb - va, B = vc - vb;
        if (d64) {
            const int64_t D = B * (int64_t)(b - a) - A * (int64_t)(c - b);
            if (D <= 0) return false;
            if (modd == 0) return true;
            if (fast) {
                const float Df = ws_u64_to_float((uint64_t)D);
                const float rhs = muq * ((float)(c - a) * (float)((b - a) * (c - b)));
                const float diff = Df - rhs;
                const float err = 6.0e-7f * (Df + rhs);
                if (diff > err) return true;
                if (diff < -err) return false;
            }
            const int r = near_tie64(D, (uint64_t)(c - a) * (uint64_t)(b - a) * (uint64_t)(c - b), sc);
            if (r >= 0) return r != 0;
        } else if (fast) {
            const float n1 = (float)(b - a), n2 = (float)(c - b);
            // A, B >= 0 (deviations from the tile's first point, sorted order)
            const float fB = ws_u64_to_float((uint64_t)B) * n1;
            const float fA = ws_u64_to_float((uint64_t)A) * n2;
            const float rhs = muq * (float)(c - a) * n1 * n2;
            const float diff = (fB - fA) - rhs;
            const float err = 5.0e-7f * (fabsf(fB) + fabsf(fA) + rhs);
            if (diff > err) return true;
            if (diff < -err) return false;
        }
        return ws_convex_binade_exact(A, B, b - a, c - b, c - a, sc);
    }
    __device__ __forceinline__ bool convex(int a, int b, int c, const SegConst& sc) const {
        return convex_v(a, v(a), b, v(b), c, v(c), sc);
    }
};

// Thresholds of the hull test inside one chunk.  Three points a < b < c of
// one chunk have n1 = b - a and n2 = c - b in [1, M - 1], and the test is
// Delta (d - 1) > mlam K 2^s with K = (n1 + n2) n1 n2 (lambda 2^L = mlam 2^s).
// Delta is an integer, so this holds exactly when Delta > T with
// T = floor(mlam K 2^s / (d - 1)); thr[n1 M + n2] = T, clamped to INT32_MAX,
// turns the chain's test into one integer compare.  T is computed in integer
// and FP32 arithmetic only (a float quotient, then exact remainder
// corrections); entries with n1 + n2 > M are never read (0).
__device__ __forceinline__ bool ws_gt_muK(int64_t D, uint64_t K, const SegConst& sc) {
    return ws_convex_binade_exact(0, D, 1, 1, (int64_t)K, sc);   // D (d - 1) > mlam K 2^s
}

template <int M>
__device__ __forceinline__ int ws_thr_entry(int i, uint64_t mlam, int s, uint64_t dm1) {
    const int n1 = i / M, n2 = i % M;
    if (!(n1 >= 1 && n2 >= 1 && n1 + n2 <= M) || mlam == 0) return 0;
    const uint64_t K = (uint64_t)((n1 + n2) * n1 * n2);
    const uint64_t N = mlam * K;   // mlam < 2^53, K <= M^3 / 4: N < 2^63
    u128 Nn;                       // floor(N 2^s)
    if (s >= 0) {
        if (ws_bitlen64(N) - 1 + s >= ws_bitlen64(dm1) + 31) return INT32_MAX;   // N 2^s >= 2^31 (d - 1)
        Nn = (u128)N << s;
    } else {
        Nn = (s <= -64) ? (u128)0 : (u128)(N >> -s);
    }
    if (Nn >= ((u128)dm1 << 31)) return INT32_MAX;
    // T = floor(Nn / (d - 1)) < 2^31
    const float fd = ws_u64_to_float(dm1);
    float q = ws_i128_to_float_scaled((i128)Nn, 0) / fd;
    int64_t T = (int64_t)fminf(fmaxf(q, 0.0f), 2147483648.0f);
    i128 r = (i128)Nn - (i128)((u128)(uint64_t)T * (u128)dm1);
    T += (int64_t)floorf(ws_i128_to_float_scaled(r, 0) / fd);   // |r / (d - 1)| < 2^10 here
    r = (i128)Nn - (i128)T * (i128)dm1;
    for (int it = 0; it < 4 && (r < 0 || r >= (i128)dm1); ++it) {
        if (r < 0) { --T; r += (i128)dm1; } else { ++T; r -= (i128)dm1; }
    }
    if (r < 0 || r >= (i128)dm1) {   // not reached for the bounds above; exact bisection
        SegConst c{};
        c.mlam = mlam; c.s = s; c.dm1 = dm1;
        int64_t lo = 0, hi = INT32_MAX;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo + 1) / 2;
            if (ws_gt_muK(mid, K, c)) hi = mid - 1; else lo = mid;
        }
        T = lo;
    }
    return (int)min(T, (int64_t)INT32_MAX);
}

// Integer constants of the hull test at fixed-point scale 2^L, for ws_thr_entry.
__device__ __forceinline__ void ws_thr_consts(double lam, int L, uint64_t& mlam, int& s) {
    int elam;
    ws_split_lambda(lam, mlam, elam);
    s = elam + L;
}

// True when a tile of n points whose deviations span `range` keeps
// B n1 - A n2 exact in 64 bits: |B n1|, |A n2| <= n1 n2 range <= n^2 range / 4.
__device__ __forceinline__ bool ws_dev_d64(uint64_t range, int n) {
    return n <= 1 || range <= (((uint64_t)1 << 62) / (uint64_t)n) / (uint64_t)n;
}

// Deviation points of a tile with constants sc (its fixed-point scale).
template <int M>
__device__ __forceinline__ TilePtsDev<M> ws_dev_pts(const int64_t* s64, float muq, bool fast, uint64_t range, int n,
                                                    const SegConst& sc) {
    TilePtsDev<M> P;
    P.s64 = s64; P.muq = muq; P.fast = fast; P.d64 = ws_dev_d64(range, n); P.thr = nullptr;
    if (sc.mlam == 0) { P.modd = 0; P.sodd = 0; }
    else { const int tz = __ffsll((long long)sc.mlam) - 1; P.modd = sc.mlam >> tz; P.sodd = sc.s + tz; }
    return P;
}

// Rank -> point in the hull of chunks [c0, c1) (ranks relative to cum[c0]).
template <int NT, int M>
__device__ __forceinline__ int ws_hull_point(const HullSmem<NT, M>& s, int c0, int c1, int r) {
    const int target = r + s.cum[c0];
    int lo = c0, hi = c1 - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s.cum[mid] <= target) lo = mid; else hi = mid - 1;
    }
    return (int)s.H[(s.lo[lo] + (target - s.cum[lo])) * NT + lo];
}

// Bridge search between the hulls of chunks [cL0, cL1) (ranks 0..p) and
// [cR0, cR1) (ranks 0..q) that share their junction point L_p = R_0.
// On return: flag 0 = the junction stays a vertex (keep L, drop R_0, the
// duplicate); flag 1 = the merged hull is L[0..istar] + R[jstar..q].
// L_i survives iff it is strictly below the chord from L_{i-1} to its
// tangent point on R; survivors form a prefix of L, so istar is found by a
// gallop from the junction plus bisection, and each tangent the same way.
template <int NT, int M, class Pts>
struct TileBridge {
    const HullSmem<NT, M>& s;
    const Pts& P;
    const SegConst& sc;
    int cL0, cL1, cR0, cR1, q;
    __device__ __forceinline__ int Lpt(int r) const { return ws_hull_point<NT, M>(s, cL0, cL1, r); }
    __device__ __forceinline__ int Rpt(int r) const { return ws_hull_point<NT, M>(s, cR0, cR1, r); }
    // R_{j+1} on or below the line (L_i, R_j): keep moving right
    __device__ __forceinline__ bool right(int pi, int64_t vi, int j) const {
        const int rj = Rpt(j), rk = Rpt(j + 1);
        return !P.convex_v(pi, vi, rj, P.v(rj), rk, P.v(rk), sc);
    }
    __device__ __forceinline__ int tangent(int pi, int64_t vi) const {
        if (!right(pi, vi, 0)) return 0;
        int good = 0, step = 1, bad;
        while (true) {
            const int j = good + step;
            if (j >= q) { bad = q; break; }
            if (right(pi, vi, j)) { good = j; step <<= 1; } else { bad = j; break; }
        }
        while (bad - good > 1) {
            const int mid = (good + bad) >> 1;
            if (right(pi, vi, mid)) good = mid; else bad = mid;
        }
        return bad;
    }
    __device__ __forceinline__ bool survives(int i, int* jt) const {
        const int pi = Lpt(i);
        const int64_t vi = P.v(pi);
        *jt = tangent(pi, vi);
        if (i == 0) return true;
        const int pm = Lpt(i - 1), pt = Rpt(*jt);
        return P.convex_v(pm, P.v(pm), pi, vi, pt, P.v(pt), sc);
    }
    // galloping search (logarithmic on long bridges)
    __device__ __noinline__ void search(int p, int& istar, int& jstar) const {
        int jt;
        if (survives(p - 1, &jt)) { istar = p - 1; jstar = jt; return; }
        int bad = p - 1, good = 0, step = 1, jgood = 0;
        while (true) {
            const int i = p - 1 - step;
            if (i <= 0) { good = 0; survives(0, &jgood); break; }
            int jj;
            if (survives(i, &jj)) { good = i; jgood = jj; break; }
            bad = i; step <<= 1;
        }
        while (bad - good > 1) {
            const int mid = (good + bad) >> 1;
            int jj;
            if (survives(mid, &jj)) { good = mid; jgood = jj; } else bad = mid;
        }
        istar = good; jstar = jgood;
    }
    // cursor over a chunk range: (chunk, entry); rank = cum[c] - cum[c0] + (k - lo[c]).
    // Moving across chunk lists jumps over empty chunks with a binary search
    // on the rank scan (cum), not a linear walk.
    __device__ __forceinline__ void locate(int c0, int c1, int r, int& c, int& k) const {
        const int target = r + s.cum[c0];
        int lo = c0, hi = c1 - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s.cum[mid] <= target) lo = mid; else hi = mid - 1;
        }
        c = lo;
        k = s.lo[lo] + (target - s.cum[lo]);
    }
    __device__ __forceinline__ bool prevL(int& c, int& k) const {
        if (k > s.lo[c]) { --k; return true; }
        const int r = s.cum[c] - s.cum[cL0] - 1;   // rank of the previous vertex of L
        if (r < 0) return false;
        locate(cL0, c, r, c, k);
        return true;
    }
    __device__ __forceinline__ bool nextR(int& c, int& k) const {
        if (k + 1 < s.hi[c]) { ++k; return true; }
        const int r = s.cum[c] - s.cum[cR0] + (s.hi[c] - s.lo[c]);   // rank of the next vertex of R
        if (r > q) return false;
        locate(cR0, cR1, r, c, k);
        return true;
    }
    __device__ __forceinline__ int at(int c, int k) const { return (int)s.H[k * NT + c]; }
    // Bridge: start at the junction and walk outward (the linear merge of
    // two convex chains); after a few steps fall back to the gallop.
    __device__ void run(int p, int& flag, int& istar, int& jstar) const {
        flag = 0; istar = p; jstar = 0;
        if (p <= 0 || q <= 0) return;
        // cursors on L_{p-1} and R_1 (the junction J = L_p = R_0 sits between them)
        int lc, lk, rc, rk, jc, jk;
        locate(cL0, cL1, p - 1, lc, lk);
        locate(cR0, cR1, 0, jc, jk);
        locate(cR0, cR1, 1, rc, rk);
        int li = at(lc, lk), rj = at(rc, rk);
        int64_t vli = P.v(li), vrj = P.v(rj);
        {
            const int pj = at(jc, jk);
            if (P.convex_v(li, vli, pj, P.v(pj), rj, vrj, sc)) return;   // junction stays a vertex
        }
        flag = 1;
        int steps = 0;
        constexpr int WALK_MAX = 24;
        while (true) {
            bool moved = false;
            while (true) {   // move left while L_{i-1} is on/below the line (L_i, R_j)
                int c2 = lc, k2 = lk;
                if (!prevL(c2, k2)) break;
                const int lm = at(c2, k2);
                const int64_t vlm = P.v(lm);
                if (P.convex_v(lm, vlm, li, vli, rj, vrj, sc)) break;
                lc = c2; lk = k2; li = lm; vli = vlm; moved = true;
                if (++steps > WALK_MAX) { search(p, istar, jstar); return; }
            }
            while (true) {   // move right while R_{j+1} is on/below the line (L_i, R_j)
                int c2 = rc, k2 = rk;
                if (!nextR(c2, k2)) break;
                const int rn = at(c2, k2);
                const int64_t vrn = P.v(rn);
                if (P.convex_v(li, vli, rj, vrj, rn, vrn, sc)) break;
                rc = c2; rk = k2; rj = rn; vrj = vrn; moved = true;
                if (++steps > WALK_MAX) { search(p, istar, jstar); return; }
            }
            if (!moved) break;
        }
        istar = s.cum[lc] - s.cum[cL0] + (lk - s.lo[lc]);
        jstar = s.cum[rc] - s.cum[cR0] + (rk - s.lo[rc]);
    }
};

// Narrow this chunk's surviving range after the merge of node `node`
// (children [node, node+half) and [node+half, node+2half)).
template <int NT, int M>
__device__ __forceinline__ void ws_apply_merge(HullSmem<NT, M>& s, int t, int node, int half, int nL, int nR) {
    if (nL <= 0 || nR <= 0) return;
    int r0, keep_lo, keep_hi;
    if (t < node + half) { r0 = s.cum[t] - s.cum[node]; keep_lo = 0; keep_hi = s.res_i[node]; }
    else { r0 = s.cum[t] - s.cum[node + half]; keep_lo = s.res_j[node]; keep_hi = 1 << 30; }
    const int l = s.lo[t], h = s.hi[t];
    const int a = max(keep_lo - r0, 0), b = min(keep_hi - r0 + 1, h - l);
    if (b <= a) { s.hi[t] = (uint16_t)l; }
    else { s.lo[t] = (uint16_t)(l + a); s.hi[t] = (uint16_t)(l + b); }
}

template <int NT, int M, class Pts>
__device__ __forceinline__ void ws_merge_node(HullSmem<NT, M>& s, const Pts& P, const SegConst& sc, int node, int half,
                                              int c1, int nL, int nR) {
    int flag = 0, is = nL - 1, js = 0;
    if (nL > 0 && nR > 0) {
        TileBridge<NT, M, Pts> br{s, P, sc, node, node + half, node + half, c1, nR - 1};
        br.run(nL - 1, flag, is, js);
        if (flag == 0) { is = nL - 1; js = 1; }
    }
    s.res_i[node] = is;
    s.res_j[node] = js;
}

// Is the junction point b a strict vertex between a and c?  (out of line)
template <class Pts>
__device__ __noinline__ bool ws_junction_convex(const Pts& P, const SegConst& sc, int a, int b, int c) {
    return P.convex(a, b, c, sc);
}

// Junction tests of the hull shortcuts (kept out of line: they run once per
// thread and would otherwise add register pressure to the chain).
template <class Pts>
__device__ __noinline__ void ws_junction_checks(const Pts& P, const SegConst& sc, int first, int last, int next_last,
                                                bool& conv_ok, bool& conc_ok) {
    if (conv_ok) conv_ok = P.convex(last - 1, last, last + 1, sc);
    if (conc_ok) conc_ok = !P.convex(first, last, next_last, sc);
}

// Build the hull of points 0..n of a tile.  Thread t owns chunk t = points
// [t*M, min((t+1)*M, n)] and runs the sequential monotone chain (the stack
// form of pool-adjacent-violators) over it; chunk hulls are then merged up a
// binary tree -- five warp-synchronous levels, then log2(NT/32) CTA levels.
// A merge keeps a prefix of the left hull and a suffix of the right one
// joined by their bridge (the divide-and-conquer step of Search Collisions,
// Sec. 4.3 / Thm 4.2, as a tangent search), so every chunk only narrows the
// surviving range [lo, hi) of its own list.  On return s.cum is the CTA
// exclusive scan of the surviving counts and *total_vertices their sum.
template <int NT, int M, class Pts, bool JSKIP = false>
__device__ void ws_cta_hull(HullSmem<NT, M>& s, int n, const Pts& P, const SegConst& sc, int* total_vertices) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    int cnt = 0;
    {
        const int first = t * M;
        bool c32 = false;
        if constexpr (Pts::kThr) {
            // chunk span S: every Delta = B n1 - A n2 of the chunk is at most (M - 1) S
            if (P.thr != nullptr && first < n)
                c32 = (uint64_t)(P.v(min(first + M, n)) - P.v(first)) <= (uint64_t)(INT32_MAX - 1) / (M - 1);
        }
        if (c32) {
            if constexpr (Pts::kThr) {
                // exact 32-bit chain: A, B and Delta are exact in 32 bits (differences of
                // the low words), the right-hand side is the threshold table
                const int32_t* w32 = reinterpret_cast<const int32_t*>(P.s64);
                const int last = min(first + M, n);
                int p0 = 0, p1 = 0;
                uint32_t r0 = 0, r1 = 0;
                for (int pnt = first; pnt <= last; ++pnt) {
                    const uint32_t rp = (uint32_t)w32[2 * ws_sidx<M>(pnt)];
                    while (cnt >= 2) {
                        const int n1 = p1 - p0, n2 = pnt - p1;
                        const int D = (int)((rp - r1) * (uint32_t)n1 - (r1 - r0) * (uint32_t)n2);
                        if (D > P.thr[n1 * M + n2]) break;
                        --cnt;
                        p1 = p0; r1 = r0;
                        if (cnt >= 2) { p0 = s.H[(cnt - 2) * NT + t]; r0 = (uint32_t)w32[2 * ws_sidx<M>(p0)]; }
                    }
                    s.H[cnt * NT + t] = (uint16_t)pnt;
                    p0 = p1; r0 = r1;
                    p1 = pnt; r1 = rp;
                    ++cnt;
                }
            }
        } else if (first < n) {
            const int last = min(first + M, n);
            int p0 = 0, p1 = 0;          // the two top entries of the stack
            int64_t v0 = 0, v1 = 0;
            for (int pnt = first; pnt <= last; ++pnt) {
                const int64_t vp = P.v(pnt);
                while (cnt >= 2 && !P.convex_v(p0, v0, p1, v1, pnt, vp, sc)) {
                    --cnt;
                    p1 = p0; v1 = v0;
                    if (cnt >= 2) { p0 = s.H[(cnt - 2) * NT + t]; v0 = P.v(p0); }
                }
                s.H[cnt * NT + t] = (uint16_t)pnt;
                p0 = p1; v0 = v1;
                p1 = pnt; v1 = vp;
                ++cnt;
            }
        }
    }
    s.lo[t] = 0;
    s.hi[t] = (uint16_t)cnt;
    // ---- shortcuts (two hull tests per thread and two barriers):
    //  * every chunk kept all its points and every junction triple is convex:
    //    the tile is a convex sequence, its hull is every point;
    //  * every chunk hull is its two end points and the chain of chunk end
    //    points is concave at every junction: the hull is the chord (0, n).
    bool skip_tree;
    {
        const int first = t * M;
        bool conv_ok = true, conc_ok = true;
        if (first < n) {
            const int last = min(first + M, n);
            conv_ok = cnt == last - first + 1;
            conc_ok = cnt == 2;
            if (last < n && (conv_ok || conc_ok))
                ws_junction_checks<Pts>(P, sc, first, last, min(last + M, n), conv_ok, conc_ok);
        }
        const int all_conv = __syncthreads_and(conv_ok);
        const int all_conc = __syncthreads_and(conc_ok);
        skip_tree = all_conv || all_conc;
        if (all_conv) {
            if (t > 0 && first < n) s.lo[t] = 1;   // the junction point is the previous chunk's last
        } else if (all_conc) {
            if (t == 0) { s.H[0] = 0; s.H[NT] = (uint16_t)n; s.lo[0] = 0; s.hi[0] = 2; }
            else { s.lo[t] = 0; s.hi[t] = 0; }
        }
    }
    // ---- warp shortcut (JSKIP; pays off where most junctions are vertices,
    // i.e. small lambda against the gaps): when every junction between the warp's chunks is a
    // strict vertex of (its hull neighbour on the left, it, its hull neighbour
    // on the right), the concatenated chunk hulls are a convex chain, hence
    // the warp's hull: only the duplicated junction points go.
    bool warp_skip = skip_tree;
    if (JSKIP && !skip_tree) {
        const int first = t * M;
        bool jok = true;
        if (lane < 31 && first + M < n) {
            const int c0 = cnt, c1 = (int)s.hi[t + 1];
            jok = c0 >= 2 && c1 >= 2 &&
                  ws_junction_convex<Pts>(P, sc, (int)s.H[(c0 - 2) * NT + t], first + M, (int)s.H[NT + t + 1]);
        }
        warp_skip = __all_sync(WS_FULL_MASK, jok);
        if (warp_skip && lane > 0 && first < n) s.lo[t] = 1;
    }
    __syncwarp();
    // ---- warp levels: chunks of one warp, warp-relative ranks
    for (int half = warp_skip ? 32 : 1; half < 32; half <<= 1) {
        const int c = (int)s.hi[t] - (int)s.lo[t];
        const int inc = ws_warp_incl_scan<int>(c);
        s.cum[t] = inc - c;
        if (lane == 31) s.wtot[w] = inc;
        __syncwarp();
        const int mask = 2 * half - 1;
        const int node = t & ~mask;
        const int endR = ((node & 31) + 2 * half == 32) ? s.wtot[w] : s.cum[node + 2 * half];
        const int nL = s.cum[node + half] - s.cum[node], nR = endR - s.cum[node + half];
        if ((lane & mask) == 0) ws_merge_node<NT, M, Pts>(s, P, sc, node, half, node + 2 * half, nL, nR);
        __syncwarp();
        ws_apply_merge<NT, M>(s, t, node, half, nL, nR);
        __syncwarp();
    }
    // ---- CTA shortcut: the same test at the junctions between warps
    bool cta_skip = skip_tree;
    if (JSKIP && !skip_tree && NT > 32) {
        __syncthreads();
        bool jok = true;
        // lane 31 of warp w tests the junction J = end of warp w's range
        const int J = (w + 1) * 32 * M;
        const int has = (int)s.hi[t] - (int)s.lo[t];
        const unsigned ne = __ballot_sync(WS_FULL_MASK, has > 0);
        if (lane == 31 && w + 1 < NT / 32 && J < n) {
            // left neighbour of J in warp w's hull: the vertex before J (J ends lane 31's list)
            int left = -1;
            if (has >= 2) left = (int)s.H[((int)s.hi[t] - 2) * NT + t];
            else {
                const unsigned before = ne & ((has >= 1) ? 0x7fffffffu : 0xffffffffu) & 0x7fffffffu;
                if (before) { const int l = w * 32 + (31 - __clz(before)); left = (int)s.H[((int)s.hi[l] - 1) * NT + l]; }
            }
            // right neighbour: the second vertex of warp w+1's hull (its lane 0 list starts at J)
            int right = -1;
            const int t0 = (w + 1) * 32;
            const int h0 = (int)s.hi[t0] - (int)s.lo[t0];
            if (h0 >= 2) right = (int)s.H[((int)s.lo[t0] + 1) * NT + t0];
            else {
                for (int l = t0 + 1; l < t0 + 32 && l < NT; ++l)
                    if (s.hi[l] > s.lo[l]) { right = (int)s.H[(int)s.lo[l] * NT + l]; break; }
            }
            jok = left >= 0 && right >= 0 && ws_junction_convex<Pts>(P, sc, left, J, right);
        }
        cta_skip = __syncthreads_and(jok);
        if (cta_skip && lane == 0 && w > 0 && t * M < n && s.hi[t] > s.lo[t]) s.lo[t] = (uint16_t)(s.lo[t] + 1);
    }
    // ---- CTA levels
    for (int half = cta_skip ? NT : 32; half < NT; half <<= 1) {
        const int c = (int)s.hi[t] - (int)s.lo[t];
        int tot;
        const int ex = ws_block_excl_scan<NT, int>(c, s.wsum_i, &tot);
        s.cum[t] = ex;
        if (t == 0) s.cum[NT] = tot;
        __syncthreads();
        const int node = t - (t % (2 * half));
        const int c1 = min(node + 2 * half, NT);
        const int nL = s.cum[node + half] - s.cum[node];
        const int nR = s.cum[c1] - s.cum[node + half];
        if (t == node) ws_merge_node<NT, M, Pts>(s, P, sc, node, half, c1, nL, nR);
        __syncthreads();
        ws_apply_merge<NT, M>(s, t, node, half, nL, nR);
        __syncthreads();
    }
    const int c = (int)s.hi[t] - (int)s.lo[t];
    int tot;
    const int ex = ws_block_excl_scan<NT, int>(c, s.wsum_i, &tot);
    s.cum[t] = ex;
    if (t == 0) s.cum[NT] = tot;
    __syncthreads();
    *total_vertices = tot;
}

// Bridge search between convex chains L (ranks 0..p) and R (ranks 0..q) that
// share their junction point L_p = R_0.  Accessors: getL(r, pt, X), getR(r, pt, X).
// On return: flag = 0 if the junction stays a vertex (keep L, drop R_0 as a
// duplicate); flag = 1 if the merged hull is L[0..istar] + R[jstar..q].
template <class GL, class GR>
__device__ __forceinline__ void ws_bridge(const GL& getL, int p, const GR& getR, int q, const SegConst& sc,
                                          int& flag, int& istar, int& jstar) {
    flag = 0; istar = p; jstar = 0;
    if (p <= 0 || q <= 0) return;
    int64_t a, b, c; i128 Xa, Xb, Xc;
    getL(p - 1, a, Xa); getL(p, b, Xb); getR(1, c, Xc);
    if (ws_convex(Xa, Xb, Xc, a, b, c, sc)) return;
    flag = 1;
    // tangent from L_i to R: first j in [0, q] where R_{j+1} is strictly above line (L_i, R_j)
    auto tangent = [&](int64_t pi, i128 Xi) -> int {
        auto Mtrue = [&](int j) -> bool {   // R_{j+1} on/below line L_i R_j  (move right)
            if (j >= q) return false;
            int64_t pj, pk; i128 Xj, Xk;
            getR(j, pj, Xj); getR(j + 1, pk, Xk);
            return !ws_convex(Xi, Xj, Xk, pi, pj, pk, sc);
        };
        if (!Mtrue(0)) return 0;
        int good = 0, step = 1, bad;
        while (true) {
            int j = good + step;
            if (j >= q) { bad = q; break; }
            if (Mtrue(j)) { good = j; step <<= 1; } else { bad = j; break; }
        }
        while (bad - good > 1) {
            int mid = (good + bad) >> 1;
            if (Mtrue(mid)) good = mid; else bad = mid;
        }
        return bad;
    };
    auto survives = [&](int i, int& jt) -> bool {
        int64_t pi; i128 Xi;
        getL(i, pi, Xi);
        jt = tangent(pi, Xi);
        if (i == 0) return true;
        int64_t pm, pt; i128 Xm, Xt;
        getL(i - 1, pm, Xm);
        getR(jt, pt, Xt);
        return ws_convex(Xm, Xi, Xt, pm, pi, pt, sc);
    };
    int jt;
    if (survives(p - 1, jt)) { istar = p - 1; jstar = jt; return; }
    int bad = p - 1, good = -1, step = 1, jgood = 0;
    while (true) {
        int i = p - 1 - step;
        if (i <= 0) { good = 0; survives(0, jgood); break; }
        int jj;
        if (survives(i, jj)) { good = i; jgood = jj; break; }
        bad = i; step <<= 1;
    }
    while (bad - good > 1) {
        int mid = (good + bad) >> 1;
        int jj;
        if (survives(mid, jj)) { good = mid; jgood = jj; } else bad = mid;
    }
    istar = good; jstar = jgood;
}

