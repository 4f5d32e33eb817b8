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

template <typename V> __device__ __forceinline__ V ws_warp_incl_scan(V v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V t = ws_shfl_up<V>(v, o);
        if (lane >= o) v += t;
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
// Stable ranking of a CTA's keys by one 8-bit digit.
// Arrangement: warp w owns positions [w*32*ITEMS, (w+1)*32*ITEMS); item k of
// lane l is position w*32*ITEMS + k*32 + l, so processing k in order and lanes
// in order visits positions in order (stability).  Returns, per item, the
// position of the key in the digit-sorted tile; digit_count/digit_start
// (shared, 256 entries) receive the tile histogram and its exclusive scan.
// whist: shared [NW][256] uint32.
// ---------------------------------------------------------------------------
template <int NT, int ITEMS>
__device__ __forceinline__ void ws_rank_digits(const uint32_t (&dig)[ITEMS], const bool (&valid)[ITEMS],
                                               int (&pos)[ITEMS], uint32_t* whist, uint32_t* digit_count,
                                               uint32_t* digit_start, uint32_t* scratch32) {
    constexpr int NW = NT / 32;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t* my = whist + w * 256;
    for (int i = lane; i < 256; i += 32) my[i] = 0;
    __syncwarp();
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        unsigned act = __ballot_sync(WS_FULL_MASK, valid[k]);
        uint32_t dg = valid[k] ? dig[k] : 256u + lane;   // invalid lanes get private digits
        unsigned peers = __match_any_sync(WS_FULL_MASK, dg) & act;
        int before = 0;
        if (valid[k]) before = (int)my[dg];
        __syncwarp();
        if (valid[k]) {
            int r = __popc(peers & lt);
            pos[k] = before + r;
            if (r == 0) my[dg] = (uint32_t)(before + __popc(peers));
        } else {
            pos[k] = -1;
        }
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive scan across warps, tile count
    for (int dgt = threadIdx.x; dgt < 256; dgt += NT) {
        uint32_t run = 0;
        for (int ww = 0; ww < NW; ++ww) {
            uint32_t c = whist[ww * 256 + dgt];
            whist[ww * 256 + dgt] = run;
            run += c;
        }
        digit_count[dgt] = run;
    }
    __syncthreads();
    // exclusive scan over the 256 digits
    if (threadIdx.x < 32) {
        uint32_t v[8], s = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) { v[i] = digit_count[lane * 8 + i]; s += v[i]; }
        uint32_t inc = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(WS_FULL_MASK, inc, o);
            if (lane >= o) inc += t;
        }
        uint32_t run = inc - s;
#pragma unroll
        for (int i = 0; i < 8; ++i) { digit_start[lane * 8 + i] = run; run += v[i]; }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (valid[k]) pos[k] += (int)(digit_start[dig[k]] + whist[w * 256 + dig[k]]);
    (void)scratch32;
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
    uint16_t H[NT * (M + 1)];   // chunk hull vertex lists (tile-local point indices)
    uint16_t lo[NT], hi[NT];    // surviving range of each list
    int cum[NT + 1];            // exclusive scan of surviving counts
    int res_flag[NT], res_i[NT], res_j[NT];
    int wsum_i[NT / 32];
};

// rank -> point within the children of a node (chunks [c0, c1), ranks relative to cum[c0])
template <int NT, int M>
__device__ __forceinline__ int ws_hull_point(const HullSmem<NT, M>& s, int c0, int c1, int r) {
    int target = r + s.cum[c0];
    int lo = c0, hi = c1 - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (s.cum[mid] <= target) lo = mid; else hi = mid - 1;
    }
    return (int)s.H[lo * (M + 1) + s.lo[lo] + (target - s.cum[lo])];
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

// Build the hull of points 0..n.  XOf: functor p -> i128.  After return (and a
// __syncthreads inside), s.lo/s.hi give each chunk's surviving vertices and
// s.cum the exclusive scan of their counts (total = number of hull vertices).
template <int NT, int M, class XOf>
__device__ void ws_cta_hull(HullSmem<NT, M>& s, int n, const XOf& X, const SegConst& sc, int* total_vertices) {
    const int t = threadIdx.x;
    // 1. per-thread monotone chain over the chunk's points
    int first = t * M;
    int cnt = 0;
    if (first < n) {
        int last = min(first + M, n);
        uint16_t* st = s.H + t * (M + 1);
        for (int pnt = first; pnt <= last; ++pnt) {
            i128 Xp = X(pnt);
            while (cnt >= 2) {
                int pa = st[cnt - 2], pb = st[cnt - 1];
                if (ws_convex(X(pa), X(pb), Xp, pa, pb, pnt, sc)) break;
                --cnt;
            }
            st[cnt++] = (uint16_t)pnt;
        }
    }
    s.lo[t] = 0;
    s.hi[t] = (uint16_t)cnt;
    __syncthreads();
    // 2. pairwise merges up the tree
    for (int half = 1; half < NT; half <<= 1) {
        int c = (int)s.hi[t] - (int)s.lo[t];
        int tot;
        int ex = ws_block_excl_scan<NT, int>(c, s.wsum_i, &tot);
        s.cum[t] = ex;
        if (t == 0) s.cum[NT] = tot;
        __syncthreads();
        if ((t % (2 * half)) == 0 && t + half < NT) {
            int cL0 = t, cL1 = t + half, cR0 = t + half, cR1 = min(t + 2 * half, NT);
            int nL = s.cum[cL1] - s.cum[cL0], nR = s.cum[cR1] - s.cum[cR0];
            int flag = 0, is = 0, js = 0;
            if (nL > 0 && nR > 0) {
                auto getL = [&](int r, int64_t& pt, i128& Xv) {
                    pt = ws_hull_point<NT, M>(s, cL0, cL1, r);
                    Xv = X((int)pt);
                };
                auto getR = [&](int r, int64_t& pt, i128& Xv) {
                    pt = ws_hull_point<NT, M>(s, cR0, cR1, r);
                    Xv = X((int)pt);
                };
                ws_bridge(getL, nL - 1, getR, nR - 1, sc, flag, is, js);
                if (flag == 0) { is = nL - 1; js = 1; }
            } else {
                is = nL - 1; js = 0;   // one side empty: nothing to merge
            }
            s.res_flag[t] = flag; s.res_i[t] = is; s.res_j[t] = js;
        }
        __syncthreads();
        {
            int node = t - (t % (2 * half));
            if (node + half < NT) {
                int nL = s.cum[node + half] - s.cum[node];
                int nR = s.cum[min(node + 2 * half, NT)] - s.cum[node + half];
                if (nL > 0 && nR > 0) {
                    int r0, keep_lo, keep_hi;   // ranks of this chunk and the kept rank window
                    if (t < node + half) { r0 = s.cum[t] - s.cum[node]; keep_lo = 0; keep_hi = s.res_i[node]; }
                    else { r0 = s.cum[t] - s.cum[node + half]; keep_lo = s.res_j[node]; keep_hi = 1 << 30; }
                    int l = s.lo[t], h = s.hi[t];
                    int cntc = h - l;
                    int a = max(keep_lo - r0, 0), b = min(keep_hi - r0 + 1, cntc);
                    if (b <= a) { s.lo[t] = (uint16_t)l; s.hi[t] = (uint16_t)l; }
                    else { s.lo[t] = (uint16_t)(l + a); s.hi[t] = (uint16_t)(l + b); }
                }
            }
        }
        __syncthreads();
    }
    int c = (int)s.hi[t] - (int)s.lo[t];
    int tot;
    int ex = ws_block_excl_scan<NT, int>(c, s.wsum_i, &tot);
    s.cum[t] = ex;
    if (t == 0) s.cum[NT] = tot;
    __syncthreads();
    *total_vertices = tot;
}
