// ws_hull.cuh -- lean exact lower hull of one tile of sorted points (the
// in-tile cluster merge of Sec. 4, re-derived as a convex-hull computation).
//
// Points P_p = (p, X_p), p = 0..n, with X the fixed-point prefix sum of the
// tile's sorted values in "tile units" (ulps of the tile's binade, or units of
// the segment's fixed-point scale); the shift lambda(d-1-2j)/(d-1) is folded
// into the hull test (ws_common.cuh), so the lower hull of these points is the
// pool-adjacent-violators partition of the tile considered on its own.
//
// Layout: NT lanes, lane t owns the "chunk" of points [t*M, min(t*M+M, n)]
// (consecutive chunks share an end point).
//   1. Every lane runs the stack form of pool-adjacent-violators over its M
//      elements while it accumulates their prefix sums (no block scan: the
//      lane's base comes from one warp scan of chunk totals).
//   2. Chunk hulls merge up a binary tree -- five warp-synchronous levels,
//      then the CTA levels.  A merge keeps a prefix of the left hull and a
//      suffix of the right one, joined by their bridge (common lower tangent,
//      Search Collisions' Merge of Sec. 4.3 / Thm 4.2 as a tangent search),
//      found by walking outward from the junction.  The walk steps across
//      lanes with the warp's non-empty-lane bitmask, so each step is O(1).
// Every decision is the exact integer hull test of the tile (TilePtsDev with
// 64-bit deviations), so the partition is exact.
#pragma once
#include "ws_block.cuh"

__device__ __forceinline__ int ws_bitlen_u64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// range n^2 <= 2^62: every Delta = B n1 - A n2 of a tile of n points whose
// deviations span `range` is exact in 64 bits (|B n1|, |A n2| <= range n^2 / 4).
__device__ __forceinline__ bool ws_lean_tile(uint64_t range, int n) {
    const uint64_t nn = (uint64_t)n * (uint64_t)n;
    return __umul64hi(range, nn) == 0 && range * nn <= ((uint64_t)1 << 62);
}
// range n <= 2^62: every prefix sum of deviations of the tile fits 64 bits
// (the lean kernels' requirement; Delta may then need the 128-bit test).
__device__ __forceinline__ bool ws_lean_x(uint64_t range, int n) {
    return __umul64hi(range, (uint64_t)n) == 0 && range * (uint64_t)n <= ((uint64_t)1 << 62);
}

// floor(lambda 2^L K / (d - 1)) exactly (the largest D with D (d-1) <= mlam K 2^s),
// saturated at 2^62.
static __device__ __noinline__ int64_t ws_floor_muK64(uint64_t K, const SegConst& sc) {
    if (sc.mlam == 0) return 0;
    const double est = ldexp((double)sc.mlam * (double)K, sc.s) / (double)sc.dm1;
    if (!(est < 4.0e18)) return (int64_t)1 << 62;
    const int64_t q = (int64_t)est;
    // the estimate is within q 2^-50 + 2 of the answer; bisect a window around it
    int64_t lo = q > (1 << 14) ? q - (1 << 14) : 0, hi = q + (1 << 14);
    if (ws_gt_muK(lo, K, sc)) lo = 0;                      // (not reached)
    if (!ws_gt_muK(hi, K, sc)) return (int64_t)1 << 62;   // (not reached)
    while (hi - lo > 1) {   // invariant: !gt(lo), gt(hi)
        const int64_t mid = lo + (hi - lo) / 2;
        if (ws_gt_muK(mid, K, sc)) hi = mid; else lo = mid;
    }
    return lo;
}

// lambda 2^L / (d - 1) in FP32 for the hull-test filter, without FP64: two
// roundings (the integer mantissa of lambda, the quotient), covered by the
// filter's margin.  usable: finite and far from overflow in the filter.
__device__ __forceinline__ float ws_muq_f(const SegConst& sc, bool& usable) {
    const float m = ldexpf(ws_u64_to_float(sc.mlam), sc.s) / ws_u64_to_float(sc.dm1);
    usable = (m == m) && m < 1.0e26f;
    return usable ? m : 0.0f;
}

namespace wsh {

constexpr int NT = 256;                // lanes per tile
constexpr int M = 16;                  // elements per lane
constexpr int NW = NT / 32;
constexpr int WP = 32 * M;             // elements per warp
constexpr int TILE = NT * M;           // 4096 elements per tile
constexpr int XSLOT = WP + 1 + WP / M; // prefix slots of one warp (point q stored at q + q / M)
constexpr uint16_t NONE = 0xffff;

// Shared memory of one tile.
struct Smem {
    // X of point p lives in the array of warp own(p) = (p - 1) / WP (p = 0: warp 0),
    // at slot q + q / M, q = p - own(p) WP in [0, WP]: the lane holding element
    // p - 1 writes it, so every point has exactly one writer.
    int64_t X[NW][XSLOT];
    uint16_t st[(M + 1) * NT];   // lane stacks (hull vertex points), entry k of lane t at k * NT + t
    uint16_t lo[NT], hi[NT];     // surviving range [lo, hi) of each lane's stack
    uint32_t ne[NW];             // non-empty lanes of every warp
    int64_t wtot[NW];            // prefix total of every warp's elements
    uint16_t res[NT][4];         // merge result at the node's first lane: last kept left (lane, entry),
                                 // first kept right (lane, entry) or NONE
    int wsum[NW];
    int general;                 // a bridge walk hit its cap: the tile needs the general kernel
    int all_conc;
    // IC rounds, per warp: last survivor / removal, first ones (read as int4)
    __align__(16) int wl[NW];
    __align__(16) int wlr[NW];
    __align__(16) int wf[NW];
    __align__(16) int wfr[NW];
};
static_assert(NW % 4 == 0, "per-warp words are read four at a time");

__device__ __forceinline__ int own_warp(int p) { return p ? (p - 1) / WP : 0; }
__device__ __forceinline__ int64_t& xref(Smem& s, int p) {
    const int w = own_warp(p), q = p - w * WP;
    return s.X[w][q + q / M];
}
__device__ __forceinline__ int64_t xat(const Smem& s, int p) {
    const int w = own_warp(p), q = p - w * WP;
    return s.X[w][q + q / M];
}

// The exact hull test on tile-unit prefix values: P_b strictly below the
// chord from P_a to P_c, i.e. Delta (d - 1) > lambda 2^L K with
// Delta = B n1 - A n2 (exact in 64 bits on lean tiles) and K = (c-a) n1 n2.
// Inline: the sign of Delta, lambda = 0, and the FP32 filter (error bounded
// relative to Delta + rhs, see TilePtsDev); the rest out of line.
struct Test {
    TilePtsDev<M> P;   // (its muq, fast, modd, sodd, d64)
    SegConst sc;
    __device__ __noinline__ bool slow(int64_t D, uint64_t K) const {
        const int r = P.near_tie64(D, K, sc);
        if (r >= 0) return r != 0;
        return ws_gt_muK(D, K, sc);
    }
    // Three points of one chunk whose prefix span is at most (2^31 - 2) / (M - 1)
    // (every FP32 one-binade tile): A n2 and B n1 stay below 2^31, so Delta is
    // exact from the low 32 bits of X.
    __device__ __forceinline__ bool t32(int a, uint32_t Xa, int b, uint32_t Xb, int c, uint32_t Xc) const {
        const int n1 = b - a, n2 = c - b;
        const int D = (int)((Xc - Xb) * (uint32_t)n1 - (Xb - Xa) * (uint32_t)n2);
        if (D <= 0) return false;
        if (P.modd == 0) return true;
        const int K = (c - a) * n1 * n2;   // <= M^3 / 4: exact in FP32
        if (P.fast) {
            const float Df = (float)D;
            const float rhs = P.muq * (float)K;
            const float diff = Df - rhs;
            const float err = 6.0e-7f * (Df + rhs);
            if (diff > err) return true;
            if (diff < -err) return false;
        }
        return slow((int64_t)D, (uint64_t)K);
    }
    __device__ __forceinline__ bool operator()(int a, int64_t Xa, int b, int64_t Xb, int c, int64_t Xc) const {
        const int n1 = b - a, n2 = c - b;
        if (!P.d64) return P.convex_v(a, Xa, b, Xb, c, Xc, sc);   // Delta may need 128 bits
        const int64_t D = (Xc - Xb) * (int64_t)n1 - (Xb - Xa) * (int64_t)n2;
        if (D <= 0) return false;
        if (P.modd == 0) return true;
        const int nn = n1 * n2;   // <= 2^24: exact in FP32
        if (P.fast) {
            const float Df = ws_u64_to_float((uint64_t)D);
            const float rhs = P.muq * ((float)(c - a) * (float)nn);
            const float diff = Df - rhs;
            const float err = 6.0e-7f * (Df + rhs);
            if (diff > err) return true;
            if (diff < -err) return false;
        }
        return slow(D, (uint64_t)(c - a) * (uint64_t)nn);
    }
};

// Stack form of pool-adjacent-violators over the lane's chunk (points
// first .. last, prefix sums already in s.X; Xf = X at point first), as a
// rolled loop (small code).  Writes the stack; returns its depth.
__device__ __forceinline__ int lane_chain(Smem& s, const Test& T, int t, int first, int last, int64_t Xf) {
    s.st[t] = (uint16_t)first;
    int cnt = 1;
    int p0 = 0, p1 = first;
    if (xat(s, last) - Xf <= (int64_t)((INT32_MAX - 1) / (M - 1))) {
        // 32-bit chain: the low words of X differ exactly
        uint32_t X0 = 0, X1 = (uint32_t)Xf;
#pragma unroll 1
        for (int p = first + 1; p <= last; ++p) {
            const uint32_t X = (uint32_t)xat(s, p);
            while (cnt >= 2 && !T.t32(p0, X0, p1, X1, p, X)) {
                --cnt;
                p1 = p0;
                X1 = X0;
                if (cnt >= 2) {
                    p0 = s.st[(cnt - 2) * NT + t];
                    X0 = (cnt == 2) ? (uint32_t)Xf : (uint32_t)xat(s, p0);
                }
            }
            s.st[cnt * NT + t] = (uint16_t)p;
            ++cnt;
            p0 = p1;
            X0 = X1;
            p1 = p;
            X1 = X;
        }
        return cnt;
    }
    int64_t X0 = 0, X1 = Xf;
#pragma unroll 1
    for (int p = first + 1; p <= last; ++p) {
        const int64_t X = xat(s, p);
        while (cnt >= 2 && !T(p0, X0, p1, X1, p, X)) {
            --cnt;
            p1 = p0;
            X1 = X0;
            if (cnt >= 2) {
                p0 = s.st[(cnt - 2) * NT + t];
                X0 = (cnt == 2) ? Xf : xat(s, p0);   // entry 0 is `first`, written by the previous lane
            }
        }
        s.st[cnt * NT + t] = (uint16_t)p;
        ++cnt;
        p0 = p1;
        X0 = X1;
        p1 = p;
        X1 = X;
    }
    return cnt;
}

// Junction-local merge of the 32 chunk hulls of a warp.  Lane l finds the
// bridge between its chain and lane l+1's by walking outward from their
// common point J inside the two chains only.  If afterwards every lane keeps
// at least the vertices [a, b] with a < b -- a the left bridge's landing
// index (0 when J stays a vertex), b the right bridge's -- the kept ranges
// joined by the bridges are convex (every bridge slope lies strictly between
// the slopes of the chain edges it meets) and below every point, so they are
// the warp's hull; the lanes' ranges are set and true is returned.  Otherwise
// (a bridge would reach past a neighbouring chunk) nothing is changed and
// false is returned.  Uniform over the warp; cnt = the lane's chain depth.
__device__ __forceinline__ bool warp_junctions(Smem& s, const Test& T, int t, int cnt) {
    const int l = t & 31;
    const int cntR = __shfl_down_sync(WS_FULL_MASK, cnt, 1);
    int bR = cnt - 1;      // last kept index of this lane
    int aN = 0, f0N = 1;   // next lane: bridge landing index, junction point kept
    if (l < 31 && cnt >= 2 && cntR >= 2) {
        const int J = s.st[(cnt - 1) * NT + t];
        const int64_t XJ = xat(s, J);
        int i = cnt - 2, j = 1;
        int pl = s.st[i * NT + t], pr = s.st[j * NT + t + 1];
        int64_t Xl = xat(s, pl), Xr = xat(s, pr);
        if (!T(pl, Xl, J, XJ, pr, Xr)) {
            f0N = 0;
            while (true) {
                bool moved = false;
                while (i > 0) {
                    const int pu = s.st[(i - 1) * NT + t];
                    const int64_t Xu = xat(s, pu);
                    if (T(pu, Xu, pl, Xl, pr, Xr)) break;
                    --i; pl = pu; Xl = Xu; moved = true;
                }
                while (j + 1 < cntR) {
                    const int pu = s.st[(j + 1) * NT + t + 1];
                    const int64_t Xu = xat(s, pu);
                    if (T(pl, Xl, pr, Xr, pu, Xu)) break;
                    ++j; pr = pu; Xr = Xu; moved = true;
                }
                if (!moved) break;
            }
            bR = i;
            aN = j;
        }
    }
    const int a = __shfl_up_sync(WS_FULL_MASK, aN, 1);
    const int f0 = __shfl_up_sync(WS_FULL_MASK, f0N, 1);
    const bool ok = cnt == 0 || (l == 0 ? 0 : a) < bR;
    if (!__all_sync(WS_FULL_MASK, ok)) return false;
    if (cnt > 0) {
        s.lo[t] = (uint16_t)(l == 0 ? 0 : (f0 ? 1 : a));
        s.hi[t] = (uint16_t)(bR + 1);
    }
    return true;
}

// Cursor on a lane's stack entry.
struct Cur {
    int c, k;
};

// Previous vertex of a node's hull (lanes >= g0), stepping across empty lanes
// with the non-empty masks.
__device__ __forceinline__ bool prev_v(const Smem& s, int g0, Cur& u) {
    if (u.k > (int)s.lo[u.c]) { --u.k; return true; }
    int c = u.c - 1;
    while (c >= g0) {
        const int w = c >> 5;
        unsigned m = s.ne[w] & (0xffffffffu >> (31 - (c & 31)));
        if (w == (g0 >> 5)) m &= 0xffffffffu << (g0 & 31);
        if (m) {
            u.c = (w << 5) + 31 - __clz((int)m);
            u.k = (int)s.hi[u.c] - 1;
            return true;
        }
        c = (w << 5) - 1;
    }
    return false;
}

// Next vertex of a node's hull (lanes < g1).
__device__ __forceinline__ bool next_v(const Smem& s, int g1, Cur& u) {
    if (u.k + 1 < (int)s.hi[u.c]) { ++u.k; return true; }
    int c = u.c + 1;
    while (c < g1) {
        const int w = c >> 5;
        unsigned m = s.ne[w] & (0xffffffffu << (c & 31));
        if (w == ((g1 - 1) >> 5) && (g1 & 31)) m &= 0xffffffffu >> (32 - (g1 & 31));
        if (m) {
            u.c = (w << 5) + __ffs((int)m) - 1;
            u.k = (int)s.lo[u.c];
            return true;
        }
        c = (w + 1) << 5;
    }
    return false;
}

// Last non-empty lane in [g0, g1) (-1 if none) / first one.
__device__ __forceinline__ int last_ne(const Smem& s, int g0, int g1) {
    int c = g1 - 1;
    while (c >= g0) {
        const int w = c >> 5;
        unsigned m = s.ne[w] & (0xffffffffu >> (31 - (c & 31)));
        if (w == (g0 >> 5)) m &= 0xffffffffu << (g0 & 31);
        if (m) return (w << 5) + 31 - __clz((int)m);
        c = (w << 5) - 1;
    }
    return -1;
}
__device__ __forceinline__ int first_ne(const Smem& s, int g0, int g1) {
    int c = g0;
    while (c < g1) {
        const int w = c >> 5;
        unsigned m = s.ne[w] & (0xffffffffu << (c & 31));
        if (w == ((g1 - 1) >> 5) && (g1 & 31)) m &= 0xffffffffu >> (32 - (g1 & 31));
        if (m) return (w << 5) + __ffs((int)m) - 1;
        c = (w + 1) << 5;
    }
    return -1;
}

__device__ __forceinline__ int vpt(const Smem& s, const Cur& u) { return (int)s.st[u.k * NT + u.c]; }

// Merge the hulls of lanes [g0, gm) and [gm, g1) (both non-empty): the bridge
// by walking outward from the junction (the linear merge of two convex
// chains).  Writes the node result at s.res[g0]; returns false if the walk
// took more than `cap` steps (result not written).
static __device__ __noinline__ bool node_merge(Smem& s, const Test& T, int g0, int gm, int g1, int cap) {
    Cur a{last_ne(s, g0, gm), 0};
    a.k = (int)s.hi[a.c] - 1;
    Cur b{first_ne(s, gm, g1), 0};
    b.k = (int)s.lo[b.c];
    const int J = vpt(s, a);   // == vpt(s, b): the junction point
    const int64_t XJ = xat(s, J);
    Cur li = a, rj = b;
    const bool hasL = prev_v(s, g0, li);
    const bool hasR = next_v(s, g1, rj);
    uint16_t* r = s.res[g0];
    if (!hasR) {   // (a node's hull always ends at its last point, so this is not reached)
        r[0] = (uint16_t)a.c; r[1] = (uint16_t)a.k; r[2] = NONE; r[3] = NONE;
        return true;
    }
    int pl = hasL ? vpt(s, li) : J, pr = vpt(s, rj);
    int64_t Xl = xat(s, pl), Xr = xat(s, pr);
    if (!hasL || T(pl, Xl, J, XJ, pr, Xr)) {   // the junction stays a vertex: drop its right copy
        r[0] = (uint16_t)a.c; r[1] = (uint16_t)a.k; r[2] = (uint16_t)rj.c; r[3] = (uint16_t)rj.k;
        return true;
    }
    int steps = 0;
    while (true) {
        bool moved = false;
        while (true) {   // move left while L_i is not strictly below the chord from L_{i-1} to R_j
            Cur u = li;
            if (!prev_v(s, g0, u)) break;
            const int pu = vpt(s, u);
            const int64_t Xu = xat(s, pu);
            if (T(pu, Xu, pl, Xl, pr, Xr)) break;
            li = u; pl = pu; Xl = Xu; moved = true;
            if (++steps > cap) return false;
        }
        while (true) {   // move right while R_j is not strictly below the chord from L_i to R_{j+1}
            Cur u = rj;
            if (!next_v(s, g1, u)) break;
            const int pu = vpt(s, u);
            const int64_t Xu = xat(s, pu);
            if (T(pl, Xl, pr, Xr, pu, Xu)) break;
            rj = u; pr = pu; Xr = Xu; moved = true;
            if (++steps > cap) return false;
        }
        if (!moved) break;
    }
    r[0] = (uint16_t)li.c; r[1] = (uint16_t)li.k; r[2] = (uint16_t)rj.c; r[3] = (uint16_t)rj.k;
    return true;
}

// Narrow lane t's range after the merge of node [g0, gm) + [gm, g1).
__device__ __forceinline__ void apply_merge(Smem& s, int t, int g0, int gm) {
    const uint16_t* r = s.res[g0];
    if (t < gm) {
        if (t > (int)r[0]) s.hi[t] = s.lo[t];
        else if (t == (int)r[0]) s.hi[t] = (uint16_t)(r[1] + 1);
    } else {
        if (r[2] == NONE || t < (int)r[2]) s.hi[t] = s.lo[t];
        else if (t == (int)r[2]) s.lo[t] = r[3];
    }
}

// Bridge of a warp-level node: lanes [g0, g0+half) and [g0+half, g0+2half)
// of the warp starting at CTA lane `base`, both non-empty; ne = the warp's
// non-empty lanes (cursor steps across lanes are O(1) bit operations).
// Returns the last kept left vertex and the first kept right vertex (packed
// lane << 8 | entry; right = -1 if none).
__device__ __forceinline__ void warp_node(const Smem& s, const Test& T, int base, int g0, int half, unsigned ne,
                                          int& resL, int& resR) {
    const unsigned mL = (half == 16 ? 0xffffu : ((1u << half) - 1u)) << g0;
    const unsigned mR = mL << half;
    const unsigned neL = ne & mL, neR = ne & mR;
    auto prevL = [&](int& c, int& k) -> bool {
        if (k > (int)s.lo[base + c]) { --k; return true; }
        const unsigned m = neL & ((1u << c) - 1u);
        if (!m) return false;
        c = 31 - __clz((int)m);
        k = (int)s.hi[base + c] - 1;
        return true;
    };
    auto nextR = [&](int& c, int& k) -> bool {
        if (k + 1 < (int)s.hi[base + c]) { ++k; return true; }
        const unsigned m = neR & ~((2u << c) - 1u);
        if (!m) return false;
        c = __ffs((int)m) - 1;
        k = (int)s.lo[base + c];
        return true;
    };
    auto pt = [&](int c, int k) { return (int)s.st[k * NT + base + c]; };
    int lc = 31 - __clz((int)neL), lk = (int)s.hi[base + lc] - 1;   // J on the left
    int rc = __ffs((int)neR) - 1, rk = (int)s.lo[base + rc];        // J on the right
    const int J = pt(lc, lk);
    const int64_t XJ = xat(s, J);
    const int jc = lc, jk = lk;
    const bool hasL = prevL(lc, lk);
    const bool hasR = nextR(rc, rk);
    if (!hasR) { resL = (jc << 8) | jk; resR = -1; return; }
    int pl = hasL ? pt(lc, lk) : J, pr = pt(rc, rk);
    int64_t Xl = xat(s, pl), Xr = xat(s, pr);
    if (!hasL || T(pl, Xl, J, XJ, pr, Xr)) {   // the junction stays a vertex
        resL = (jc << 8) | jk;
        resR = (rc << 8) | rk;
        return;
    }
    while (true) {
        bool moved = false;
        while (true) {
            int c = lc, k = lk;
            if (!prevL(c, k)) break;
            const int pu = pt(c, k);
            const int64_t Xu = xat(s, pu);
            if (T(pu, Xu, pl, Xl, pr, Xr)) break;
            lc = c; lk = k; pl = pu; Xl = Xu; moved = true;
        }
        while (true) {
            int c = rc, k = rk;
            if (!nextR(c, k)) break;
            const int pu = pt(c, k);
            const int64_t Xu = xat(s, pu);
            if (T(pl, Xl, pr, Xr, pu, Xu)) break;
            rc = c; rk = k; pr = pu; Xr = Xu; moved = true;
        }
        if (!moved) break;
    }
    resL = (lc << 8) | lk;
    resR = (rc << 8) | rk;
}

// Five warp-synchronous merge levels over the 32 lanes of the caller's warp.
// Entry: s.lo/s.hi hold every lane's chain; exit: the warp's hull.
__device__ __forceinline__ void warp_tree(Smem& s, const Test& T, int t) {
    const int l = t & 31, base = t & ~31;
    unsigned ne = __ballot_sync(WS_FULL_MASK, s.hi[t] > s.lo[t]);
    for (int half = 1; half < 32; half <<= 1) {
        const int g0 = l & ~(2 * half - 1);
        const unsigned mL = (half == 16 ? 0xffffu : ((1u << half) - 1u)) << g0;
        const bool lead = l == g0 && (ne & mL) && (ne & (mL << half));
        int resL = 0, resR = 0;
        if (lead) warp_node(s, T, base, g0, half, ne, resL, resR);
        // every lane of the node learns its leader's result
        const int rL = __shfl_sync(WS_FULL_MASK, resL, g0);
        const int rR = __shfl_sync(WS_FULL_MASK, resR, g0);
        const bool merged = __shfl_sync(WS_FULL_MASK, (int)lead, g0) != 0;
        __syncwarp();
        if (merged) {
            if (l < g0 + half) {
                const int c = rL >> 8;
                if (l > c) s.hi[t] = s.lo[t];
                else if (l == c) s.hi[t] = (uint16_t)((rL & 0xff) + 1);
            } else {
                const int c = rR < 0 ? 32 : (rR >> 8);
                if (l < c) s.hi[t] = s.lo[t];
                else if (l == c) s.lo[t] = (uint16_t)(rR & 0xff);
            }
        }
        ne = __ballot_sync(WS_FULL_MASK, s.hi[t] > s.lo[t]);
        __syncwarp();
    }
    if (l == 0) s.ne[t >> 5] = ne;
}

// CTA levels (warp hulls merged pairwise).  Entry: every warp has run
// warp_tree; exit (synchronised): the tile's hull, or s.general = 1 if a
// bridge walk took more than `cap` steps.
__device__ __forceinline__ void cta_tree(Smem& s, const Test& T, int t, int cap) {
    const int l = t & 31, w = t >> 5;
    for (int half = 32; half < NT; half <<= 1) {
        __syncthreads();
        const int g0 = t & ~(2 * half - 1);
        int merged = 0;
        if (t == g0 && !s.general && first_ne(s, g0, g0 + half) >= 0 && first_ne(s, g0 + half, g0 + 2 * half) >= 0) {
            if (node_merge(s, T, g0, g0 + half, g0 + 2 * half, cap)) merged = 1;
            else s.general = 1;
        }
        if (t == g0) s.wsum[w] = merged;   // (g0 is a multiple of 32: one node per leading warp)
        __syncthreads();
        if (s.general) return;
        if (s.wsum[g0 >> 5]) apply_merge(s, t, g0, g0 + half);
        const unsigned m = __ballot_sync(WS_FULL_MASK, s.hi[t] > s.lo[t]);
        if (l == 0) s.ne[w] = m;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Imminent Collisions rounds on the tile as a closed system (appendix
// algorithm "Imminent collisions algorithm (v2)", Sec. 4), exact.
//   Round 1 (done by the caller): point p (1 <= p < n) starts a new block iff
//            y_{p-1} < y_p, i.e. the gap x_p - x_{p-1} exceeds 2 lambda/(d-1).
//   Round r: every surviving block boundary b, with neighbouring boundaries
//            a < b < c (0 and n at the ends), stays iff the mean of y over
//            [a, b) is strictly below the mean over [b, c) -- the hull test
//            at b; all boundaries are decided at once, as the paper's rounds
//            do.  A boundary whose neighbours did not change keeps last
//            round's answer, so only boundaries next to a removal are tested
//            again.
// When a round removes nothing, every adjacent pair of blocks has increasing
// means: the blocks are the tile's pool-adjacent-violators partition and
// their boundaries (with points 0 and n) the vertices of its lower hull.
// For this lane's range of points: the last set point before it and the first
// one after it, over the whole CTA, for two point sets at once (B: current
// boundaries, R: last round's removals; bit i = point first + i).  Inside the
// warp by ballots and one shuffle each, across warps through one word per
// warp and set (one barrier).  -1 / BIG when there is none.
struct Around { int pS, nS, pR, nR; };
__device__ __forceinline__ Around around(Smem& s, int t, int first, uint32_t B, uint32_t R) {
    const int l = t & 31, w = t >> 5;
    const int BIG = 1 << 20;
    const int myLS = B ? first + 31 - __clz((int)B) : -1, myFS = B ? first + __ffs((int)B) - 1 : BIG;
    const int myLR = R ? first + 31 - __clz((int)R) : -1, myFR = R ? first + __ffs((int)R) - 1 : BIG;
    const unsigned bS = __ballot_sync(WS_FULL_MASK, B != 0), bR = __ballot_sync(WS_FULL_MASK, R != 0);
    const unsigned lt = (1u << l) - 1u, gt = l == 31 ? 0u : ~((2u << l) - 1u);
    auto below = [&](unsigned m, int v) {   // v of the highest lane of m below this one
        const unsigned mm = m & lt;
        const int x = __shfl_sync(WS_FULL_MASK, v, mm ? 31 - __clz((int)mm) : l);
        return mm ? x : -1;
    };
    auto above = [&](unsigned m, int v) {   // v of the lowest lane of m above this one
        const unsigned mm = m & gt;
        const int x = __shfl_sync(WS_FULL_MASK, v, mm ? __ffs((int)mm) - 1 : l);
        return mm ? x : BIG;
    };
    Around r;
    r.pS = below(bS, myLS);
    r.pR = below(bR, myLR);
    r.nS = above(bS, myFS);
    r.nR = above(bR, myFR);
    // the warp's own last / first points of each set
    const int wLS = __shfl_sync(WS_FULL_MASK, myLS, bS ? 31 - __clz((int)bS) : 0);
    const int wLR = __shfl_sync(WS_FULL_MASK, myLR, bR ? 31 - __clz((int)bR) : 0);
    const int wFS = __shfl_sync(WS_FULL_MASK, myFS, bS ? __ffs((int)bS) - 1 : 0);
    const int wFR = __shfl_sync(WS_FULL_MASK, myFR, bR ? __ffs((int)bR) - 1 : 0);
    if (l == 0) {
        s.wl[w] = bS ? wLS : -1;
        s.wlr[w] = bR ? wLR : -1;
        s.wf[w] = bS ? wFS : BIG;
        s.wfr[w] = bR ? wFR : BIG;
    }
    __syncthreads();
    int wl[NW], wlr[NW], wf[NW], wfr[NW];
#pragma unroll
    for (int j = 0; j < NW / 4; ++j) {
        const int4 a = reinterpret_cast<const int4*>(s.wl)[j], b = reinterpret_cast<const int4*>(s.wlr)[j];
        const int4 c = reinterpret_cast<const int4*>(s.wf)[j], d = reinterpret_cast<const int4*>(s.wfr)[j];
        wl[4 * j] = a.x; wl[4 * j + 1] = a.y; wl[4 * j + 2] = a.z; wl[4 * j + 3] = a.w;
        wlr[4 * j] = b.x; wlr[4 * j + 1] = b.y; wlr[4 * j + 2] = b.z; wlr[4 * j + 3] = b.w;
        wf[4 * j] = c.x; wf[4 * j + 1] = c.y; wf[4 * j + 2] = c.z; wf[4 * j + 3] = c.w;
        wfr[4 * j] = d.x; wfr[4 * j + 1] = d.y; wfr[4 * j + 2] = d.z; wfr[4 * j + 3] = d.w;
    }
#pragma unroll
    for (int k = 0; k < NW; ++k) {
        if (k < w) { r.pS = max(r.pS, wl[k]); r.pR = max(r.pR, wlr[k]); }
        if (k > w) { r.nS = min(r.nS, wf[k]); r.nR = min(r.nR, wfr[k]); }
    }
    return r;
}

// B: this lane's round-1 boundaries (bit i = point first + i); on return the
// surviving ones.  Returns true if the rounds converged within `cap` rounds
// (rounds = rounds run, the final unchanged one included).  Prefix sums of
// every point must be in s.X (the first barrier here publishes them).  All
// threads of the CTA call this.
__device__ __forceinline__ bool ic_rounds(Smem& s, const Test& T, int t, int first, int n, uint32_t& B, int cap,
                                          int& rounds) {
    rounds = 1;
    if (!__syncthreads_or(B != 0)) { rounds = 2; return true; }   // one block: the chord (round 2 has nothing to do)
    uint32_t D = B, Rprev = 0;
    const int BIG = 1 << 20;
    while (true) {
        ++rounds;
        // neighbouring boundaries outside this lane's range, and where last
        // round's removals were
        const Around ar = around(s, t, first, B, Rprev);
        const int pS = ar.pS, nS = ar.nS, pR = ar.pR, nR = ar.nR;
        const int prevS = pS < 0 ? 0 : pS, nextS = nS >= BIG ? n : nS;
        // the end survivors' outer neighbours changed if a removal lay between
        if (B) {
            if (pR > prevS) D |= B & (0u - B);
            if (nR < nextS) D |= 1u << (31 - __clz((int)B));
        }
        // decide every boundary to retest against the current blocks
        uint32_t Rm = 0, bits = B & D;
        while (bits) {
            const int i = __ffs((int)bits) - 1;
            bits &= bits - 1;
            const int p = first + i;
            const uint32_t below = B & ((1u << i) - 1u), above = B & ~((2u << i) - 1u);
            const int a = below ? first + 31 - __clz((int)below) : prevS;
            const int c = above ? first + __ffs((int)above) - 1 : nextS;
            if (!T(a, xat(s, a), p, xat(s, p), c, xat(s, c))) Rm |= 1u << i;
        }
        if (!__syncthreads_or(Rm != 0)) return true;
        if (rounds >= cap) return false;
        // survivors whose in-lane neighbourhood changed
        const uint32_t B2 = B & ~Rm;
        D = 0;
        {
            uint32_t rest = B2;
            int pq = -1;
            while (rest) {
                const int q = __ffs((int)rest) - 1;
                rest &= rest - 1;
                const uint32_t gap = ((1u << q) - 1u) & (pq >= 0 ? ~((2u << pq) - 1u) : 0xffffffffu);
                if (Rm & gap) { D |= 1u << q; if (pq >= 0) D |= 1u << pq; }
                pq = q;
            }
            if (pq >= 0 && (Rm & ~((2u << pq) - 1u))) D |= 1u << pq;   // removal above the last survivor
        }
        Rprev = Rm;
        B = B2;
    }
}

// Warm start from a candidate partition given as runs of points (the paper's
// Future Work: start from a candidate weight-sharing and edit it into the
// exact one).  R: this lane's run boundaries (bit i = point first + i).
// G: the points that survive round 1 (gap test; every hull vertex does).
// Returns the run boundaries in G plus every interior point of a run, in G,
// that lies strictly below the chord of its run.  A vertex of the lower hull
// lies strictly below every chord that spans it, so the result holds every
// hull vertex whatever the runs are, and the Imminent Collisions rounds
// started from it remove the rest: the runs only change the time, never the
// partition.  Prefix sums of every
// point must be in s.X (the barrier here publishes them).  All threads call
// this.
__device__ __forceinline__ uint32_t candidate_boundaries(Smem& s, const Test& T, int t, int first, int n,
                                                         uint32_t R, uint32_t G) {
    const int BIG = 1 << 20;
    const Around ar = around(s, t, first, R, 0u);
    const int pS = ar.pS, nS = ar.nS;
    const int prevS = pS < 0 ? 0 : pS, nextS = nS >= BIG ? n : nS;
    // interior points of this lane: 1 <= p <= n - 1 and not a run boundary
    uint32_t bits = 0;
    if (first < n) {
        const int lo = first < 1 ? 1 : first, hi = min(first + M, n);   // points [lo, hi)
        if (hi > lo) bits = (0xffffffffu >> (32 - (hi - lo))) << (lo - first);
    }
    bits &= ~R & G;
    uint32_t F = 0;
    while (bits) {
        const int i = __ffs((int)bits) - 1;
        bits &= bits - 1;
        const int p = first + i;
        const uint32_t below = R & ((1u << i) - 1u), above = R & ~((2u << i) - 1u);
        const int a = below ? first + 31 - __clz((int)below) : prevS;
        const int c = above ? first + __ffs((int)above) - 1 : nextS;
        if (T(a, xat(s, a), p, xat(s, p), c, xat(s, c))) F |= 1u << i;
    }
    return (R & G) | F;
}

// The tile's hull by per-lane chains (stack form of pool-adjacent-violators),
// the chord shortcut, a junction-local warp merge or the warp's tree of
// bridge merges, and the CTA tree.  On return s.lo/s.hi/s.st hold the hull
// (lane ranges of the lane stacks); returns false if a CTA-level bridge walk
// took more than cta_cap steps (s.general = 1; the tile needs the general
// kernel).  Prefix sums of every point must be in s.X.  All threads call
// this; it ends synchronised.
__device__ __forceinline__ bool chain_tree_hull(Smem& s, const Test& T, int t, int first, int last, int n, int64_t Xf,
                                                int cta_cap) {
    const int l = t & 31, w = t >> 5;
    __syncthreads();   // (every lane's prefix sums are written)
    int cnt = 0;
    if (first < n) cnt = lane_chain(s, T, t, first, last, Xf);
    s.lo[t] = 0;
    s.hi[t] = (uint16_t)cnt;
    __syncthreads();
    // every chunk hull is its chord and the chain of chunk end points is
    // concave at every junction: the tile's hull is the chord (0, n)
    bool conc = true;
    if (first < n) {
        conc = cnt == 2;
        if (conc && last < n) {
            const int nx = min(last + M, n);
            conc = !T(first, Xf, last, xat(s, last), nx, xat(s, nx));
        }
    }
    if (__syncthreads_and(conc)) {
        if (t == 0) { s.st[0] = 0; s.st[NT] = (uint16_t)n; s.hi[0] = 2; }
        else s.hi[t] = s.lo[t];
        __syncthreads();
        return true;
    }
    // junction-local merge of the warp's chunks; the warp's tree of merges
    // only where a bridge reaches past a neighbouring chunk
    if (!warp_junctions(s, T, t, cnt)) warp_tree(s, T, t);
    {
        const unsigned m = __ballot_sync(WS_FULL_MASK, s.hi[t] > s.lo[t]);
        if (l == 0) s.ne[w] = m;
    }
    cta_tree(s, T, t, cta_cap);
    return !s.general;   // (uniform after cta_tree's barrier)
}

}  // namespace wsh
