// ws_tile.cu -- the cluster merge of the device-wide path (Sec. 4): per-tile
// exact lower hulls, then every junction between neighbouring tiles resolved
// from the two tile hulls alone.
//
// A segment's sorted keys are cut into hull tiles of 4096 elements.
//   k_hull_fast  builds each tile's exact lower hull (ws_hull.cuh) and writes
//                its vertices (tile-local point, fixed-point prefix X);
//                tiles whose prefix sums do not fit the 64-bit lean path are
//                listed for the general tile kernel (ws_large.cu).
//   k_junction   finds the bridge (common lower tangent) between the hulls of
//                tiles T and T+1 for every junction, one thread each.
//   k_resolve    per segment: if every tile keeps at least two vertices
//                between its left and right bridge, the concatenation of the
//                kept ranges is convex and lies below every point, hence it
//                is the segment's hull, and it is written as the root piece
//                list directly.
//   k_chord,     otherwise: if every tile-hull vertex lies on or above the
//   k_decide     chord from the segment's first point to its last, the
//                segment is one cluster; else it takes the tree of bridge
//                merges (k_climb in ws_large.cu).
// With small lambda the clusters are short and every tile keeps many
// vertices, so the first case holds; with a lambda above the collapse
// threshold (Prop. 4.1) the second does.
#include "ws_hull.cuh"
#include "ws_kernels.cuh"

namespace {

using wsh::NT;
using wsh::M;
using wsh::NW;
constexpr int HT = WS_HULL_TILE;
static_assert(wsh::TILE == WS_HULL_TILE, "lean and general tile kernels share the tiling");

// Bridge walks of the CTA levels longer than this send the tile to the
// general kernel (whose CTA-parallel search handles long bridges).
constexpr int CTA_WALK_CAP = 512;

// ---------------------------------------------------------------------------
// Per-segment scale constants (one CTA of WS_NSCALE threads per segment)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(WS_NSCALE) k_scales(const typename KeyOf<T>::K* __restrict__ sorted,
                                                      const LargeSeg* __restrict__ lsegs,
                                                      const double* __restrict__ lambdas,
                                                      const int32_t* __restrict__ seg_emin, SegRuntime* rt,
                                                      TileScale* scales, uint32_t* status) {
    typedef KeyOf<T> KO;
    const int lseg = blockIdx.x, j = threadIdx.x;
    const LargeSeg ls = lsegs[lseg];
    const double lam = lambdas[ls.seg];
    const bool lam_ok = lam >= 0.0 && lam <= 1.7976931348623157e308;
    const double lamv = lam_ok ? lam : 0.0;
    const T xlo = KO::from_key(sorted[ls.kpos]), xhi = KO::from_key(sorted[ls.kpos + ls.len - 1]);
    const int emax = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[lseg]);
    if (j == 0) {
        rt[lseg].emax = emax;
        if (!lam_ok) ws_flag(status, WS_STATUS_BAD_LAMBDA);
        ws_note_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[lseg], status);
    }
    if (j > KO::FIX_OFS && j != WS_NSCALE - 1) return;
    TileScale ts;
    ts.sc = ws_seg_const_L(ls.len, lamv, KO::L_BASE - emax - (j == WS_NSCALE - 1 ? 0 : j));
    bool f;
    ts.muq = ws_muq(lamv, ts.sc, f);
    ts.fast = f ? 1 : 0;
    if (ts.sc.mlam == 0) { ts.modd = 0; ts.sodd = 0; }
    else { const int tz = __ffsll((long long)ts.sc.mlam) - 1; ts.modd = ts.sc.mlam >> tz; ts.sodd = ts.sc.s + tz; }
    ts.pad = 0;
    ts.t11 = ws_floor_muK64(2, ts.sc);
    scales[(size_t)lseg * WS_NSCALE + j] = ts;
}

// ---------------------------------------------------------------------------
// The lean tile kernel
// ---------------------------------------------------------------------------
struct FastSmem {
    wsh::Smem h;
    TileScale ts;
};

// Tile hull: Imminent Collisions rounds (appendix algorithm "Imminent
// collisions algorithm (v2)", Sec. 4) on the tile as a closed system, with
// exact tests; a tile that has not converged after ic_cap rounds (or
// ic_cap = 0) takes the chain and tree merges instead.
//   Round 1: point p (1 <= p < n) starts a new block iff y_{p-1} < y_p, i.e.
//            the gap x_p - x_{p-1} exceeds 2 lambda/(d-1): gap > t11 units.
//   Round r: every surviving block boundary b, with neighbouring boundaries
//            a < b < c, stays iff the mean of y over [a, b) is strictly below
//            the mean over [b, c) (the exact hull test at b); all boundaries
//            are decided at once, as the paper's rounds do.  A boundary whose
//            neighbours did not change keeps last round's answer, so only
//            boundaries next to a removal are tested again.
// When a round removes nothing every adjacent pair of blocks has increasing
// means: the blocks are the tile's pool-adjacent-violators partition, and
// their boundaries (with points 0 and n) its hull vertices.
// The hull by chains and trees for a tile whose rounds hit the cap: out of
// line (rare), so that the rounds' code stays compact in the instruction
// cache.  All threads call it; false if a CTA-level bridge walk hit its cap.
__device__ __noinline__ bool tile_chain_tree(wsh::Smem& s, const wsh::Test& tst, int first, int last, int n,
                                             int64_t Xf) {
    return wsh::chain_tree_hull(s, tst, threadIdx.x, first, last, n, Xf, CTA_WALK_CAP);
}

template <typename T>
__global__ void __launch_bounds__(NT, 4) k_hull_fast(const typename KeyOf<T>::K* __restrict__ sorted,
                                                   const TileDesc* __restrict__ htiles,
                                                   const LargeSeg* __restrict__ lsegs,
                                                   const SegRuntime* __restrict__ rt,
                                                   const TileScale* __restrict__ scales, uint16_t* vp, i128* vx,
                                                   int32_t* nvert, i128* tile_total, int32_t* gen_list,
                                                   int32_t* gen_count, int32_t* tile_rounds, int ic_cap) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FastSmem& S = *reinterpret_cast<FastSmem*>(smem_raw);
    wsh::Smem& s = S.h;
    const int t = threadIdx.x, l = t & 31, w = t >> 5;
    const int tile = blockIdx.x;
    const TileDesc td = htiles[tile];
    const int n = td.len;
    const K* kp = sorted + td.kpos;
    const K kfirst = kp[0], klast = kp[n - 1];
    const int emax = rt[td.lseg].emax;
    // tile units: ulps of the binade for one-binade tiles, else the segment's scale
    int sh;
    const bool bin = ws_tile_binade<T>(kfirst, klast, n, emax, sh);
    const int64_t q0 = ws_fixed<T>(KO::from_key(kfirst), emax);
    const uint64_t range = bin ? (uint64_t)(klast - kfirst) : (uint64_t)(ws_fixed<T>(KO::from_key(klast), emax) - q0);
    const bool lean = ws_lean_x(range, n);   // prefix sums in 64 bits
    const bool d64 = ws_lean_tile(range, n);  // every Delta too
    if (t == 0) {
        if (!lean) { gen_list[atomicAdd(gen_count, 1)] = tile; tile_rounds[tile] = -2; }
        else S.ts = scales[(size_t)td.lseg * WS_NSCALE + (bin ? sh : WS_NSCALE - 1)];
        s.general = 0;
    }
    if (!lean) return;   // (uniform over the CTA)

    // ---- this lane's 16 consecutive keys, the key before them, deviations
    const int first = t * M;
    K kr[M];
    {
        const K* src = kp + first;
        if (first + M <= n && (((uintptr_t)src) & 15) == 0) {
            constexpr int NV = M * (int)sizeof(K) / 16;
            uint4 buf[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) buf[i] = reinterpret_cast<const uint4*>(src)[i];
            const K* bk = reinterpret_cast<const K*>(buf);
#pragma unroll
            for (int i = 0; i < M; ++i) kr[i] = bk[i];
        } else {
#pragma unroll
            for (int i = 0; i < M; ++i) kr[i] = (first + i < n) ? src[i] : kfirst;
        }
    }
    const K kprev = (t > 0 && first < n) ? kp[first - 1] : kfirst;
    auto devk = [&](K k) -> int64_t {
        return bin ? (int64_t)(k - kfirst) : ws_fixed<T>(KO::from_key(k), emax) - q0;
    };
    auto dev = [&](int i) -> int64_t { return devk(kr[i]); };
    int64_t csum = 0;
#pragma unroll
    for (int i = 0; i < M; ++i)
        if (first + i < n) csum += dev(i);
    const int64_t winc = ws_warp_incl_scan<long long>((long long)csum);
    if (l == 31) s.wtot[w] = winc;
    if (t == 0) wsh::xref(s, 0) = 0;
    __syncthreads();
    int64_t wbase = 0;
    for (int k = 0; k < w; ++k) wbase += s.wtot[k];
    const int64_t Xf = wbase + winc - csum;   // tile-local X at point `first`
    const int last = min(first + M, n);

    wsh::Test tst;
    tst.sc = S.ts.sc;
    tst.P.s64 = nullptr;
    tst.P.muq = S.ts.muq;
    tst.P.fast = S.ts.fast != 0;
    tst.P.d64 = d64;
    tst.P.thr = nullptr;
    tst.P.modd = S.ts.modd;
    tst.P.sodd = S.ts.sodd;

    // ---- round 1: boundaries where consecutive elements do not collide.
    // Bit i of B stands for point first + i (1 <= point <= n - 1).
    // (with the prefix sums of this lane's points: one pass over its deviations)
    uint32_t B = 0;
    if (first < n) {
        const int64_t t11 = S.ts.t11;
        int64_t dprev = devk(kprev), X = Xf;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const int p = first + i;
            if (p < n) {
                const int64_t di = dev(i);
                X += di;
                wsh::xref(s, p + 1) = X;
                if (p >= 1 && di - dprev > t11) B |= 1u << i;
                dprev = di;
            }
        }
    }
    int rounds = 0;
    bool converged = false;
    if (ic_cap > 0) converged = wsh::ic_rounds(s, tst, t, first, n, B, ic_cap, rounds);
    if (t == 0) tile_rounds[tile] = converged ? rounds : -1;
    int c;      // vertices this lane writes
    int lo = 0;
    if (converged) {
        c = __popc(B) + (t == 0 ? 1 : 0) + (first < n && last == n ? 1 : 0);
    } else {
        if (!tile_chain_tree(s, tst, first, last, n, Xf)) {
            if (t == 0) { gen_list[atomicAdd(gen_count, 1)] = tile; tile_rounds[tile] = -2; }
            return;
        }
        lo = s.lo[t];
        c = (int)s.hi[t] - lo;
    }

    // ---- write the hull: tile-local points and tile-local X in the segment's
    // fixed point (binade tiles: X = p q0 + (deviation sum << sh))
    int nv;
    const int o = ws_block_excl_scan<NT, int>(c, s.wsum, &nv);
    i128* vxo = vx + (size_t)tile * (HT + 1) + o;
    uint16_t* vpo = vp + (size_t)tile * (HT + 1) + o;
    auto put = [&](int k, int p) {
        const int64_t xu = wsh::xat(s, p);
        vpo[k] = (uint16_t)p;
        vxo[k] = (i128)p * (i128)q0 + (bin ? ((i128)xu << sh) : (i128)xu);
    };
    if (converged) {
        // the vertex points staged in the (idle) lane-stack storage, then both
        // arrays written by consecutive threads at consecutive vertices
        static_assert((wsh::M + 1) * wsh::NT >= wsh::TILE + 1, "every vertex has a staging slot");
        uint16_t* stage = s.st;
        int k = o;
        if (t == 0) stage[k++] = 0;
        uint32_t rest = B;
        while (rest) {
            const int i = __ffs((int)rest) - 1;
            rest &= rest - 1;
            stage[k++] = (uint16_t)(first + i);
        }
        if (first < n && last == n) stage[k++] = (uint16_t)n;
        __syncthreads();
        i128* vxt = vx + (size_t)tile * (HT + 1);
        uint16_t* vpt = vp + (size_t)tile * (HT + 1);
        for (int i = t; i < nv; i += NT) {
            const int p = stage[i];
            const int64_t xu = wsh::xat(s, p);
            vpt[i] = (uint16_t)p;
            vxt[i] = (i128)p * (i128)q0 + (bin ? ((i128)xu << sh) : (i128)xu);
        }
    } else {
        for (int k = 0; k < c; ++k) put(k, s.st[(lo + k) * NT + t]);
    }
    if (t == 0) {
        nvert[tile] = nv;
        const int64_t xu = wsh::xat(s, n);
        const i128 tot = (i128)n * (i128)q0 + (bin ? ((i128)xu << sh) : (i128)xu);
        __stcg(reinterpret_cast<uint4*>(tile_total + tile), *reinterpret_cast<const uint4*>(&tot));
    }
}

// ---------------------------------------------------------------------------
// Junctions: the bridge between the hulls of tiles T and T+1 (one thread each)
// ---------------------------------------------------------------------------
// Result per junction (stored at the left tile T):
//   keepR[T]   index of the last vertex of T's hull on the segment's hull side
//              of the junction (its last vertex when the junction point stays);
//   keepL[T+1] index of the first kept vertex of T+1's hull (0 when the
//              junction point stays: the bridge then is that point itself);
//   jflag0[T+1] 1 when the junction point stays a vertex (T+1 then drops its
//              copy of it).
struct JVert {
    int64_t p;   // position relative to tile T's first point
    i128 X;      // prefix relative to tile T's first point
};

template <typename T>
__global__ void __launch_bounds__(256) k_junction(const TileDesc* __restrict__ htiles, const LargeSeg* __restrict__ lsegs,
                                                  const double* __restrict__ lambdas, const SegRuntime* __restrict__ rt,
                                                  const uint16_t* __restrict__ vp, const i128* __restrict__ vx,
                                                  const int32_t* __restrict__ nvert,
                                                  const i128* __restrict__ tile_total, int32_t* keepR, int32_t* keepL,
                                                  int32_t* jflag0, int n_hull) {
    const int gw = (int)(blockIdx.x * blockDim.x + threadIdx.x);   // one thread per junction
    if (gw >= n_hull) return;
    const TileDesc td = htiles[gw];
    const LargeSeg ls = lsegs[td.lseg];
    if (td.tin + 1 >= ls.hull_count) return;
    double lam = lambdas[ls.seg];
    if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) lam = 0.0;
    const SegConst sc = ws_seg_const<T>(ls.len, lam, rt[td.lseg].emax);
    const int TL = gw, TR = gw + 1;
    const int p = nvert[TL] - 1, q = nvert[TR] - 1;
    const size_t bL = (size_t)TL * (HT + 1), bR = (size_t)TR * (HT + 1);
    const i128 baseR = tile_total[TL];
    const int64_t offR = td.len;   // (a tile that has a right neighbour is whole)
    auto L = [&](int i) -> JVert { return JVert{(int64_t)vp[bL + i], vx[bL + i]}; };
    auto R = [&](int j) -> JVert { return JVert{offR + (int64_t)vp[bR + j], baseR + vx[bR + j]}; };
    auto cvx = [&](const JVert& a, const JVert& b, const JVert& c) { return ws_convex(a.X, b.X, c.X, a.p, b.p, c.p, sc); };
    // L_p = R_0 is the junction point
    int i = p - 1, j = 1;
    if (p < 1 || q < 1 || cvx(L(i), L(p), R(j))) {
        keepR[TL] = p;
        keepL[TR] = 0;
        jflag0[TR] = 1;
        return;
    }
    JVert li = L(i), rj = R(j);
    while (true) {
        bool moved = false;
        while (i > 0) {   // move left while L_i is not strictly below the chord from L_{i-1} to R_j
            const JVert u = L(i - 1);
            if (cvx(u, li, rj)) break;
            --i; li = u; moved = true;
        }
        while (j < q) {   // move right while R_j is not strictly below the chord from L_i to R_{j+1}
            const JVert u = R(j + 1);
            if (cvx(li, rj, u)) break;
            ++j; rj = u; moved = true;
        }
        if (!moved) break;
    }
    keepR[TL] = i;
    keepL[TR] = j;
    jflag0[TR] = 0;
}

// ---------------------------------------------------------------------------
// Per segment: root piece list from the junctions, the one-cluster check, or
// the tree of merges.  One CTA per large segment.
// ---------------------------------------------------------------------------
constexpr int RNT = 1024;

struct ResolveSmem {
    long long wsum64[RNT / 32];
    int wsum[RNT / 32];
    long long wlo[RNT / 32], whi[RNT / 32];
    int carry_cum;
    i128 carry_off;
    int ok;
};

// exclusive scan of an i128 over the CTA (two 64-bit halves with carry)
__device__ __forceinline__ i128 ws_block_excl_scan_i128(i128 v, ResolveSmem& s, i128* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const i128 inc = ws_warp_incl_scan<i128>(v);
    if (lane == 31) { s.wlo[w] = (long long)(uint64_t)inc; s.whi[w] = (long long)(uint64_t)(inc >> 64); }
    __syncthreads();
    if (w == 0) {
        i128 x = (lane < RNT / 32) ? (i128)(((u128)(uint64_t)s.whi[lane] << 64) | (u128)(uint64_t)s.wlo[lane]) : (i128)0;
        x = ws_warp_incl_scan<i128>(x);
        if (lane < RNT / 32) { s.wlo[lane] = (long long)(uint64_t)x; s.whi[lane] = (long long)(uint64_t)(x >> 64); }
    }
    __syncthreads();
    auto get = [&](int k) { return (i128)(((u128)(uint64_t)s.whi[k] << 64) | (u128)(uint64_t)s.wlo[k]); };
    const i128 base = w > 0 ? get(w - 1) : (i128)0;
    if (total) *total = get(RNT / 32 - 1);
    const i128 r = base + inc - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void __launch_bounds__(RNT) k_resolve(const LargeSeg* __restrict__ lsegs,
                                                 const int32_t* __restrict__ nvert,
                                                 const i128* __restrict__ tile_total,
                                                 const int32_t* __restrict__ keepR, const int32_t* __restrict__ keepL,
                                                 const int32_t* __restrict__ jflag0, Piece* pieces,
                                                 int32_t* npieces, int32_t* seg_mode, i128* tile_base,
                                                 i128* seg_total, int32_t* seg_below) {
    __shared__ ResolveSmem s;
    const int t = threadIdx.x;
    const int lseg = blockIdx.x;
    const LargeSeg ls = lsegs[lseg];
    const int nt = ls.hull_count, h0 = ls.hull_first;
    // does every tile keep >= 2 vertices between its bridges?
    bool ok = true;
    for (int k = t; k < nt; k += RNT) {
        const int a = (k == 0) ? 0 : keepL[h0 + k];
        const int b = (k == nt - 1) ? nvert[h0 + k] - 1 : keepR[h0 + k];
        ok &= a < b;
    }
    const int all_ok = __syncthreads_and(ok);
    // tile bases (X at every tile's first point) and, if every tile keeps its
    // range, the root piece list: tile k keeps [lo, hi) of its hull (a flag-0
    // junction point is kept by the tile on its left)
    if (t == 0) { s.carry_cum = 0; s.carry_off = 0; }
    __syncthreads();
    for (int k0 = 0; k0 < nt; k0 += RNT) {
        const int k = k0 + t;
        int lo = 0, hi = 0;
        i128 tot = 0;
        if (k < nt) {
            tot = tile_total[h0 + k];
            if (all_ok) {
                lo = (k == 0) ? 0 : (jflag0[h0 + k] ? 1 : keepL[h0 + k]);
                hi = ((k == nt - 1) ? nvert[h0 + k] - 1 : keepR[h0 + k]) + 1;
            }
        }
        int csum;
        const int cum = ws_block_excl_scan<RNT, int>(hi - lo, s.wsum, &csum);
        i128 osum;
        const i128 off = ws_block_excl_scan_i128(tot, s, &osum);
        if (k < nt) {
            tile_base[h0 + k] = s.carry_off + off;
            if (all_ok) {
                Piece pc;
                pc.tile = h0 + k;
                pc.lo = (uint16_t)lo;
                pc.hi = (uint16_t)hi;
                pc.cum = s.carry_cum + cum;
                pc.pad = 0;
                pc.off = s.carry_off + off;
                pieces[h0 + k] = pc;
            }
        }
        __syncthreads();
        if (t == 0) { s.carry_cum += csum; s.carry_off += osum; }
        __syncthreads();
    }
    if (t == 0) {
        seg_total[lseg] = s.carry_off;
        seg_below[lseg] = 0;
        if (all_ok) npieces[h0] = nt;
        seg_mode[lseg] = all_ok ? 0 : 3;   // 3: the one-cluster check decides
    }
}

// One cluster iff no vertex of any tile hull lies strictly below the chord
// from the segment's first point to its last (every point is on or above its
// tile's hull).  One warp per hull tile of the segments left undecided.
template <typename T>
__global__ void __launch_bounds__(256) k_chord(const TileDesc* __restrict__ htiles, const LargeSeg* __restrict__ lsegs,
                                               const double* __restrict__ lambdas, const SegRuntime* __restrict__ rt,
                                               const uint16_t* __restrict__ vp, const i128* __restrict__ vx,
                                               const int32_t* __restrict__ nvert, const i128* __restrict__ tile_base,
                                               const i128* __restrict__ seg_total,
                                               const int32_t* __restrict__ seg_mode, int32_t* seg_below,
                                               int n_hull) {
    const int gw = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (gw >= n_hull) return;
    const TileDesc td = htiles[gw];
    if (seg_mode[td.lseg] != 3) return;
    const LargeSeg ls = lsegs[td.lseg];
    double lam = lambdas[ls.seg];
    if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) lam = 0.0;
    const SegConst sc = ws_seg_const<T>(ls.len, lam, rt[td.lseg].emax);
    const i128 base = tile_base[gw], Xd = seg_total[td.lseg];
    const int nv = nvert[gw];
    const size_t b = (size_t)gw * (HT + 1);
    const int64_t p0 = (int64_t)td.tin * HT;
    bool below = false;
    for (int v = lane, it = 0; v < nv; v += 32, ++it) {
        // decided elsewhere?  (an L2 round trip: every eighth step only, so that
        // the two tail tiles' thousands of vertices do not wait on it each step)
        if ((it & 7) == 0 && *(volatile const int32_t*)(seg_below + td.lseg)) break;
        const int64_t pos = p0 + vp[b + v];
        if (pos == 0 || pos == ls.len) continue;
        if (ws_convex((i128)0, base + vx[b + v], Xd, 0, pos, ls.len, sc)) { below = true; break; }
    }
    if (below) atomicExch(seg_below + td.lseg, 1);
}

// Per segment left undecided: one cluster (root list = the first and the last
// point) or the tree of merges.
__global__ void k_decide(const LargeSeg* __restrict__ lsegs, int n_lseg, const int32_t* __restrict__ nvert,
                         const i128* __restrict__ tile_base, int32_t* seg_mode, const int32_t* __restrict__ seg_below,
                         Piece* pieces, int32_t* npieces) {
    const int lseg = blockIdx.x * blockDim.x + threadIdx.x;
    if (lseg >= n_lseg || seg_mode[lseg] != 3) return;
    if (seg_below[lseg]) { seg_mode[lseg] = 2; return; }
    const LargeSeg ls = lsegs[lseg];
    const int h0 = ls.hull_first, kl = ls.hull_count - 1;
    const int nvl = nvert[h0 + kl];
    Piece a;
    a.tile = h0; a.lo = 0; a.hi = 1; a.cum = 0; a.pad = 0; a.off = 0;
    if (kl == 0) {   // one tile: the chord is its hull
        a.hi = (uint16_t)nvl;
        pieces[h0] = a;
        npieces[h0] = 1;
    } else {
        Piece z;
        z.tile = h0 + kl; z.lo = (uint16_t)(nvl - 1); z.hi = (uint16_t)nvl; z.cum = 1; z.pad = 0;
        z.off = tile_base[h0 + kl];
        pieces[h0] = a;
        pieces[h0 + 1] = z;
        npieces[h0] = 2;
    }
    seg_mode[lseg] = 1;
}

}  // namespace

template <typename T>
cudaError_t ws_large_hull_fast(const LargeWork<T>& W, const typename KeyOf<T>::K* sorted, const double* lambdas,
                               uint32_t* status, cudaStream_t st) {
    WS_LAUNCH(W.prof, WSK_MISC, st,
              (k_scales<T><<<W.n_lseg, WS_NSCALE, 0, st>>>(sorted, W.lsegs, lambdas, W.seg_emin, W.rt, W.scales,
                                                           status)));
    const size_t smem = sizeof(FastSmem);
    cudaError_t e = cudaFuncSetAttribute(k_hull_fast<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    e = cudaMemsetAsync(W.gen_count, 0, sizeof(int32_t), st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_TILE_HULL, st,
              (k_hull_fast<T><<<W.n_hull_tiles, NT, smem, st>>>(sorted, W.hull_tiles, W.lsegs, W.rt, W.scales, W.vp,
                                                                W.vx, W.nvert, W.tile_total, W.gen_list, W.gen_count,
                                                                W.tile_rounds, W.ic_cap)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t ws_large_junctions(const LargeWork<T>& W, const double* lambdas, cudaStream_t st) {
    const int warps_per_cta = 8;
    const int grid = (W.n_hull_tiles + warps_per_cta - 1) / warps_per_cta;
    WS_LAUNCH(W.prof, WSK_JUNCTION, st,
              (k_junction<T><<<(W.n_hull_tiles + 127) / 128, 128, 0, st>>>(W.hull_tiles, W.lsegs, lambdas, W.rt, W.vp, W.vx,
                                                                  W.nvert, W.tile_total, W.keepR, W.keepL, W.jflag0,
                                                                  W.n_hull_tiles)));
    WS_LAUNCH(W.prof, WSK_JUNCTION, st,
              (k_resolve<T><<<W.n_lseg, RNT, 0, st>>>(W.lsegs, W.nvert, W.tile_total, W.keepR, W.keepL, W.jflag0,
                                                      W.pieces, W.npieces, W.seg_mode, W.tile_base, W.seg_total,
                                                      W.seg_below)));
    WS_LAUNCH(W.prof, WSK_JUNCTION, st,
              (k_chord<T><<<grid, 32 * warps_per_cta, 0, st>>>(W.hull_tiles, W.lsegs, lambdas, W.rt, W.vp, W.vx,
                                                               W.nvert, W.tile_base, W.seg_total, W.seg_mode,
                                                               W.seg_below, W.n_hull_tiles)));
    WS_LAUNCH(W.prof, WSK_JUNCTION, st,
              (k_decide<<<(W.n_lseg + 255) / 256, 256, 0, st>>>(W.lsegs, W.n_lseg, W.nvert, W.tile_base,
                                                                W.seg_mode, W.seg_below, W.pieces, W.npieces)));
    return cudaGetLastError();
}

#define WS_INST_TILE(T)                                                                                          \
    template cudaError_t ws_large_hull_fast<T>(const LargeWork<T>&, const typename KeyOf<T>::K*, const double*, \
                                               uint32_t*, cudaStream_t);                                         \
    template cudaError_t ws_large_junctions<T>(const LargeWork<T>&, const double*, cudaStream_t);
WS_INST_TILE(float)
WS_INST_TILE(double)
