// ws_large.cu -- the device-wide path for segments longer than one CTA:
//   sorted keys -> per-tile exact hulls -> tree of bridge merges across tiles
//   -> cluster table -> key -> cluster lookup in the caller's order.
//
// The hull of the points P_p = (p, S_p) (see ws_common.cuh) is built tile by
// tile (4096 elements per CTA); adjacent tile hulls are then merged up a
// binary tree.  A merge keeps a prefix of the left hull and a suffix of the
// right one (the bridge is the common lower tangent, Search Collisions'
// Merge step of Sec. 4.3 re-derived on convex chains), so a node's hull is a
// list of "pieces" -- contiguous vertex ranges of tile hulls -- and a merge
// only edits the two lists where they meet.  The root list is the cluster
// partition: its consecutive vertices bound the clusters.
#include "ws_kernels.cuh"

namespace {

constexpr int HT = WS_HULL_TILE;
constexpr int HNT = WS_HULL_NT;
constexpr int HM = WS_HULL_M;

// ---------------------------------------------------------------------------
// 1. per-tile hull
// ---------------------------------------------------------------------------
struct TileHullSmem {
    TilePrefix<HNT, HM> pre;
    HullSmem<HNT, HM> hull;
    SegConst sc;     // global fixed-point scale of the segment
    SegConst sct;    // scale of this tile when it lies in one binade
    float muq, muqt;
    int fast, fastt;
};

template <typename T>
__global__ void __launch_bounds__(HNT) k_tile_hull(const typename KeyOf<T>::K* __restrict__ sorted,
                                                   const TileDesc* __restrict__ htiles,
                                                   const LargeSeg* __restrict__ lsegs,
                                                   const double* __restrict__ lambdas, SegRuntime* rt,
                                                   uint16_t* vp, i128* vx, int32_t* nvert, i128* tile_total,
                                                   Piece* pieces, int32_t* npieces, uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileHullSmem& s = *reinterpret_cast<TileHullSmem*>(smem_raw);
    const int t = threadIdx.x;
    const int tile = blockIdx.x;
    const TileDesc td = htiles[tile];
    const LargeSeg ls = lsegs[td.lseg];
    const double lam = lambdas[ls.seg];
    const bool lam_ok = lam >= 0.0 && lam <= 1.7976931348623157e308;
    const double lamv = lam_ok ? lam : 0.0;
    const int n = td.len;
    const K* kp = sorted + td.kpos;
    const K kfirst = kp[0], klast = kp[n - 1];
    const T xlo = KO::from_key(sorted[ls.kpos]), xhi = KO::from_key(sorted[ls.kpos + ls.len - 1]);
    const int emax = max(ws_eff_exp(xlo), ws_eff_exp(xhi));
    if (t == 0) {
        if (!lam_ok) ws_flag(status, WS_STATUS_BAD_LAMBDA);
        if (td.tin == 0) rt[td.lseg].emax = emax;
        s.sc = ws_seg_const<T>(ls.len, lamv, emax);
        bool f;
        s.muq = ws_muq(lamv, s.sc, f);
        s.fast = f ? 1 : 0;
        const int sh = ws_eff_exp(KO::from_key(kfirst)) - emax + KO::FIX_OFS;
        s.sct = ws_seg_const_L(ls.len, lamv, s.sc.L - (sh > 0 ? sh : 0));
        s.muqt = ws_muq(lamv, s.sct, f);
        s.fastt = f ? 1 : 0;
    }
    // this thread's 16 consecutive sorted keys (vector loads when whole and aligned)
    K kr[HM];
    {
        const int first = t * HM;
        const K* src = kp + first;
        if (first + HM <= n && (((uintptr_t)src) & 15) == 0) {
            constexpr int NV = HM * (int)sizeof(K) / 16;
            const uint4* v4 = reinterpret_cast<const uint4*>(src);
            uint4 buf[NV];
#pragma unroll
            for (int i = 0; i < NV; ++i) buf[i] = v4[i];
            const K* bk = reinterpret_cast<const K*>(buf);
#pragma unroll
            for (int i = 0; i < HM; ++i) kr[i] = bk[i];
        } else {
#pragma unroll
            for (int i = 0; i < HM; ++i) kr[i] = (first + i < n) ? src[i] : (K)0;
        }
    }
    int64_t q0;
    i128 total;
    int bsh;
    const int mode = ws_tile_prefix<T, HNT, HM>(s.pre, kr, kfirst, klast, n, emax, q0, total, bsh);
    int nv;
    if (mode == WS_TILE_BINADE) {
        const TilePtsBinade<HM> P{s.pre.s64, s.muqt, s.fastt != 0};
        ws_cta_hull<HNT, HM>(s.hull, n, P, s.sct, &nv);
    } else if (mode == WS_TILE_NARROW) {
        const TilePts<HM, true> P{s.pre.s64, s.pre.base, q0, s.muq, s.fast != 0};
        ws_cta_hull<HNT, HM>(s.hull, n, P, s.sc, &nv);
    } else {
        const TilePts<HM, false> P{s.pre.s64, s.pre.base, q0, 0.0f, false};
        ws_cta_hull<HNT, HM>(s.hull, n, P, s.sc, &nv);
    }
    {
        const int l = s.hull.lo[t], h = s.hull.hi[t], o = s.hull.cum[t];
        const size_t b = (size_t)tile * (HT + 1);
        for (int i = l; i < h; ++i) {
            const int pnt = s.hull.H[i * HNT + t];
            vp[b + o + (i - l)] = (uint16_t)pnt;
            vx[b + o + (i - l)] = ws_tile_X<HM>(s.pre.s64, s.pre.base, mode, q0, bsh, pnt);
        }
    }
    if (t == 0) {
        nvert[tile] = nv;
        tile_total[tile] = total;
        Piece pc;
        pc.tile = tile; pc.lo = 0; pc.hi = (uint16_t)nv; pc.cum = 0; pc.pad = 0;
        pieces[tile] = pc;
        npieces[tile] = 1;
    }
}

// ---------------------------------------------------------------------------
// 2. exclusive scan of tile totals inside each segment
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tile_scan(const LargeSeg* __restrict__ lsegs, const i128* tile_total,
                                                   i128* tile_offset) {
    __shared__ i128 ws[8];
    const LargeSeg ls = lsegs[blockIdx.x];
    i128 carry = 0;
    for (int b = 0; b < ls.hull_count; b += 256) {
        int i = b + threadIdx.x;
        i128 v = (i < ls.hull_count) ? tile_total[ls.hull_first + i] : (i128)0;
        i128 tot;
        i128 ex = ws_block_excl_scan<256, i128>(v, ws, &tot);
        if (i < ls.hull_count) tile_offset[ls.hull_first + i] = carry + ex;
        carry += tot;
    }
}

// ---------------------------------------------------------------------------
// 3. merge of two adjacent node hulls (one CTA per node)
// ---------------------------------------------------------------------------
struct NodeView {
    const Piece* pc;   // piece list
    int np;            // pieces
    const uint16_t* vp;
    const i128* vx;
    const i128* toff;
    int hull_first;    // global index of the segment's first hull tile
    __device__ __forceinline__ int find(int r) const {   // piece holding rank r
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (pc[mid].cum <= r) lo = mid; else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ void get(int r, int64_t& pt, i128& X) const {
        const Piece p = pc[find(r)];
        size_t v = (size_t)p.tile * (HT + 1) + p.lo + (r - p.cum);
        pt = (int64_t)(p.tile - hull_first) * HT + vp[v];
        X = toff[p.tile] + vx[v];
    }
    __device__ __forceinline__ int count() const {
        if (np == 0) return 0;
        const Piece p = pc[np - 1];
        return p.cum + (p.hi - p.lo);
    }
};

// Bridge between two node hulls by walking outward from their junction
// (the linear merge of two convex chains), stepping through the piece lists
// directly.  Returns false (no result) after too many steps; the caller then
// runs the galloping search.  Same outputs as ws_bridge.
__device__ __forceinline__ void ws_piece_vertex(const Piece* P, int pi, int v, const uint16_t* vp, const i128* vx,
                                                const i128* toff, int hull_first, int64_t& pt, i128& X) {
    const Piece q = P[pi];
    const size_t idx = (size_t)q.tile * (HT + 1) + v;
    pt = (int64_t)(q.tile - hull_first) * HT + vp[idx];
    X = toff[q.tile] + vx[idx];
}

__device__ bool ws_bridge_walk(const Piece* PL, int npL, const Piece* PR, int npR, const uint16_t* vp,
                               const i128* vx, const i128* toff, int hull_first, const SegConst& sc, int& flag,
                               int& istar, int& jstar) {
    // cursors: (piece, vertex index in the tile list)
    int lp = npL - 1, lv = PL[lp].hi - 1;   // L_p = junction
    int rp = 0, rv = PR[0].lo;              // R_0 = junction
    auto prevL = [&](int& p, int& v) -> bool {
        if (v > PL[p].lo) { --v; return true; }
        if (p == 0) return false;
        --p; v = PL[p].hi - 1; return true;
    };
    auto nextR = [&](int& p, int& v) -> bool {
        if (v + 1 < PR[p].hi) { ++v; return true; }
        if (p + 1 >= npR) return false;
        ++p; v = PR[p].lo; return true;
    };
    int64_t pj; i128 Xj;
    ws_piece_vertex(PR, rp, rv, vp, vx, toff, hull_first, pj, Xj);
    if (!prevL(lp, lv) || !nextR(rp, rv)) { flag = 0; return true; }   // a one-vertex side: nothing to merge
    int64_t pl, pr; i128 Xl, Xr;
    ws_piece_vertex(PL, lp, lv, vp, vx, toff, hull_first, pl, Xl);
    ws_piece_vertex(PR, rp, rv, vp, vx, toff, hull_first, pr, Xr);
    if (ws_convex(Xl, Xj, Xr, pl, pj, pr, sc)) { flag = 0; return true; }
    flag = 1;
    int steps = 0;
    constexpr int WALK_MAX = 32;
    while (true) {
        bool moved = false;
        while (true) {
            int p2 = lp, v2 = lv;
            if (!prevL(p2, v2)) break;
            int64_t pm; i128 Xm;
            ws_piece_vertex(PL, p2, v2, vp, vx, toff, hull_first, pm, Xm);
            if (ws_convex(Xm, Xl, Xr, pm, pl, pr, sc)) break;
            lp = p2; lv = v2; pl = pm; Xl = Xm; moved = true;
            if (++steps > WALK_MAX) return false;
        }
        while (true) {
            int p2 = rp, v2 = rv;
            if (!nextR(p2, v2)) break;
            int64_t pn; i128 Xn;
            ws_piece_vertex(PR, p2, v2, vp, vx, toff, hull_first, pn, Xn);
            if (ws_convex(Xl, Xr, Xn, pl, pr, pn, sc)) break;
            rp = p2; rv = v2; pr = pn; Xr = Xn; moved = true;
            if (++steps > WALK_MAX) return false;
        }
        if (!moved) break;
    }
    istar = PL[lp].cum + (lv - PL[lp].lo);
    jstar = PR[rp].cum + (rv - PR[rp].lo);
    return true;
}

template <typename T>
__global__ void __launch_bounds__(256) k_merge(const MergeNode* __restrict__ nodes, const LargeSeg* __restrict__ lsegs,
                                               const double* __restrict__ lambdas, const SegRuntime* __restrict__ rt,
                                               const uint16_t* __restrict__ vp, const i128* __restrict__ vx,
                                               const i128* __restrict__ toff, Piece* pieces, int32_t* npieces,
                                               uint32_t* status) {
    __shared__ int s_is, s_js, s_flag, s_pl, s_pr;
    __shared__ int wsi[8];
    const MergeNode nd = nodes[blockIdx.x];
    const LargeSeg ls = lsegs[nd.lseg];
    const int t = threadIdx.x;
    Piece* PL = pieces + nd.left;
    Piece* PR = pieces + nd.right;
    const int npL = npieces[nd.left], npR = npieces[nd.right];
    if (t == 0) {
        double lam = lambdas[ls.seg];
        if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) lam = 0.0;
        const SegConst sc = ws_seg_const<T>(ls.len, lam, rt[nd.lseg].emax);
        NodeView L{PL, npL, vp, vx, toff, ls.hull_first};
        NodeView R{PR, npR, vp, vx, toff, ls.hull_first};
        int nL = L.count(), nR = R.count();
        int flag = 0, is = nL - 1, js = 0;
        if (nL > 0 && nR > 0) {
            if (!ws_bridge_walk(PL, npL, PR, npR, vp, vx, toff, ls.hull_first, sc, flag, is, js)) {
                auto gl = [&](int r, int64_t& pt, i128& X) { L.get(r, pt, X); };
                auto gr = [&](int r, int64_t& pt, i128& X) { R.get(r, pt, X); };
                ws_bridge(gl, nL - 1, gr, nR - 1, sc, flag, is, js);
            }
            if (flag == 0) { is = nL - 1; js = 1; }
        }
        // pieces holding istar and jstar
        s_pl = (nL > 0) ? L.find(is) : -1;
        s_pr = (nR > 0 && js < nR) ? R.find(js) : npR;
        s_is = is; s_js = js; s_flag = flag;
        // truncate the left list at istar
        if (s_pl >= 0) {
            Piece p = PL[s_pl];
            p.hi = (uint16_t)(p.lo + (is - p.cum) + 1);
            PL[s_pl] = p;
        }
        if (s_pr < npR) {
            Piece p = PR[s_pr];
            int newlo = p.lo + (js - p.cum);
            p.lo = (uint16_t)newlo;
            PR[s_pr] = p;
        }
    }
    __syncthreads();
    const int keepL = s_pl + 1;                // pieces kept from the left list
    const int firstR = s_pr;                   // first piece kept from the right list
    const int keepR = npR - firstR;
    // move the right suffix down behind the left prefix (dst <= src: chunked copy)
    Piece* dst = PL + keepL;
    const Piece* src = PR + firstR;
    for (int b = 0; b < keepR; b += 256) {
        Piece v;
        bool has = b + t < keepR;
        if (has) v = src[b + t];
        __syncthreads();
        if (has) dst[b + t] = v;
        __syncthreads();
    }
    // recompute the ranks of the merged list (drop empty pieces is not needed:
    // a kept piece always holds >= 1 vertex)
    const int np = keepL + keepR;
    int carry = 0;
    for (int b = 0; b < np; b += 256) {
        int i = b + t;
        int c = 0;
        Piece v;
        if (i < np) { v = PL[i]; c = v.hi - v.lo; }
        int tot;
        int ex = ws_block_excl_scan<256, int>(c, wsi, &tot);
        if (i < np) { v.cum = carry + ex; PL[i] = v; }
        carry += tot;
        __syncthreads();
    }
    if (t == 0) npieces[nd.left] = np;
    (void)status;
}

// ---------------------------------------------------------------------------
// 4. root of each segment: cluster count, piece index per tile, bucket map
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_root(const LargeSeg* __restrict__ lsegs,
                                              const typename KeyOf<T>::K* __restrict__ sorted, const Piece* pieces,
                                              const int32_t* npieces, int32_t* tile_piece, SegRuntime* rt,
                                              int64_t* n_clusters_out) {
    typedef KeyOf<T> KO;
    const int lseg = blockIdx.x;
    const LargeSeg ls = lsegs[lseg];
    const Piece* P = pieces + ls.hull_first;
    const int np = npieces[ls.hull_first];
    for (int i = threadIdx.x; i < np; i += 256) tile_piece[P[i].tile] = i;
    if (threadIdx.x == 0) {
        const Piece last = P[np - 1];
        int64_t nvtx = (int64_t)last.cum + (last.hi - last.lo);
        int64_t c = nvtx - 1;
        SegRuntime r = rt[lseg];
        r.n_clusters = c;
        r.table_pos = ls.kpos + lseg;
        int D = 0;
        while (D < ls.dir_cap_log2 && ((int64_t)1 << D) < c) ++D;
        r.dir_log2 = D;
        float lo = (float)KO::from_key(sorted[ls.kpos]);
        float hi = (float)KO::from_key(sorted[ls.kpos + ls.len - 1]);
        float range = hi - lo;
        float scale = (range > 0.0f && range <= 3.0e38f) ? (float)((int64_t)1 << D) / range : 0.0f;
        if (!(scale <= 3.0e38f)) scale = 0.0f;
        r.lo = lo; r.scale = scale;
        rt[lseg] = r;
        if (n_clusters_out) n_clusters_out[ls.seg] = c;
    }
}

__device__ __forceinline__ int ws_bucket(float x, float lo, float scale, int nb) {
    float f = (x - lo) * scale;
    int b = (f >= (float)nb) ? nb - 1 : (f > 0.0f ? (int)f : 0);
    return b > nb - 1 ? nb - 1 : b;
}

// ---------------------------------------------------------------------------
// 5. cluster table + directory fill (one CTA per hull tile)
// ---------------------------------------------------------------------------
constexpr int GAP_INLINE = 64;

struct BigGap { int64_t pos; int32_t count; int32_t value; uint32_t key32; int32_t pad; };

template <typename T>
__global__ void __launch_bounds__(256) k_table(const TileDesc* __restrict__ htiles, const LargeSeg* __restrict__ lsegs,
                                               const double* __restrict__ lambdas, const SegRuntime* __restrict__ rt,
                                               const typename KeyOf<T>::K* __restrict__ sorted,
                                               const uint16_t* __restrict__ vp, const i128* __restrict__ vx,
                                               const i128* __restrict__ toff, const Piece* __restrict__ pieces,
                                               const int32_t* __restrict__ npieces,
                                               const int32_t* __restrict__ tile_piece, CEntry<T>* table,
                                               DirEntry* dir, BigGap* gaps, uint32_t* ngaps, int64_t gap_cap,
                                               int fp64, uint32_t* status) {
    typedef KeyOf<T> KO;
    const int tile = blockIdx.x;
    const int tp = tile_piece[tile];
    if (tp < 0) return;
    const TileDesc td = htiles[tile];
    const LargeSeg ls = lsegs[td.lseg];
    const SegRuntime R = rt[td.lseg];
    double lam = lambdas[ls.seg];
    if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) lam = 0.0;
    const SegConst sc = ws_seg_const<T>(ls.len, lam, R.emax);
    const Piece* P = pieces + ls.hull_first;
    const int np = npieces[ls.hull_first];
    const Piece pc = P[tp];
    const int nb = 1 << R.dir_log2;
    DirEntry* D = dir + ls.dir_pos;
    auto vertex = [&](int piece_idx, int i, int64_t& pt, i128& X) {
        const Piece q = P[piece_idx];
        size_t v = (size_t)q.tile * (HT + 1) + i;
        pt = (int64_t)(q.tile - ls.hull_first) * HT + vp[v];
        X = toff[q.tile] + vx[v];
    };
    for (int i = pc.lo + threadIdx.x; i < pc.hi; i += 256) {
        int64_t r = (int64_t)pc.cum + (i - pc.lo);
        if (r >= R.n_clusters) continue;   // the final vertex (point d) opens no cluster
        int64_t a, b; i128 Xa, Xb;
        vertex(tp, i, a, Xa);
        if (i + 1 < pc.hi) vertex(tp, i + 1, b, Xb);
        else {
            if (tp + 1 >= np) { ws_flag(status, WS_STATUS_INTERNAL); continue; }
            vertex(tp + 1, P[tp + 1].lo, b, Xb);
        }
        typename KO::K k = sorted[ls.kpos + a];
        T xs = KO::from_key(k);
        CEntry<T> ce;
        ce.key = k;
        ce.val = ValueOut<T>::value(Xb - Xa, a, b, xs, sc, fp64 != 0);
        table[R.table_pos + r] = ce;
        // directory: buckets (bucket(prev start), bucket(this start)] -> r
        int bcur = ws_bucket((float)xs, R.lo, R.scale, nb);
        int bprev = -1;
        if (r > 0) {
            int64_t pa; i128 Xp;
            if (i > pc.lo) vertex(tp, i - 1, pa, Xp);
            else {
                const Piece q = P[tp - 1];
                vertex(tp - 1, q.hi - 1, pa, Xp);
            }
            bprev = ws_bucket((float)KO::from_key(sorted[ls.kpos + pa]), R.lo, R.scale, nb);
        }
        const uint32_t k32 = (uint32_t)(k >> (KO::BITS - 32));
        int64_t from = bprev + 1, to = bcur;   // inclusive range of buckets
        int64_t cnt = to - from + 1;
        const DirEntry de{(int32_t)r, k32};
        if (cnt > GAP_INLINE) {
            uint32_t g = atomicAdd(ngaps, 1u);
            if ((int64_t)g < gap_cap) {
                gaps[g].pos = ls.dir_pos + from; gaps[g].count = (int32_t)cnt; gaps[g].value = (int32_t)r;
                gaps[g].key32 = k32;
            } else ws_flag(status, WS_STATUS_INTERNAL);
        } else {
            for (int64_t bb = from; bb <= to; ++bb) D[bb] = de;
        }
        if (r == R.n_clusters - 1) {   // tail: buckets after the last start, plus the sentinel
            int64_t f2 = bcur + 1, c2 = (int64_t)nb - bcur;   // buckets bcur+1 .. nb (nb = sentinel)
            const DirEntry te{(int32_t)R.n_clusters, 0xffffffffu};
            if (c2 > GAP_INLINE) {
                uint32_t g = atomicAdd(ngaps, 1u);
                if ((int64_t)g < gap_cap) {
                    gaps[g].pos = ls.dir_pos + f2; gaps[g].count = (int32_t)c2; gaps[g].value = (int32_t)R.n_clusters;
                    gaps[g].key32 = 0xffffffffu;
                } else ws_flag(status, WS_STATUS_INTERNAL);
            } else {
                for (int64_t bb = f2; bb <= nb; ++bb) D[bb] = te;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_big_gaps(const BigGap* gaps, const uint32_t* ngaps, DirEntry* dir,
                                                  int64_t gap_cap) {
    const int64_t n = min((int64_t)*ngaps, gap_cap);
    for (int64_t g = blockIdx.x; g < n; g += gridDim.x) {
        const BigGap G = gaps[g];
        const DirEntry e{G.value, G.key32};
        for (int i = threadIdx.x; i < G.count; i += 256) dir[G.pos + i] = e;
    }
}

// ---------------------------------------------------------------------------
// 6. lookup: every weight, in the caller's order, finds its cluster by value
// ---------------------------------------------------------------------------
// Last cluster in [lo, hi) whose start key is <= k, else lo - 1; starts from
// the guess g (interpolated on the 32-bit key prefix) and steps, bisecting if
// the guess is far off.
template <typename T>
__device__ __forceinline__ int ws_find_cluster(const CEntry<T>* tab, int lo, int hi, int g, typename KeyOf<T>::K k,
                                               typename KeyOf<T>::K kg) {
    int steps = 0;
    if (kg <= k) {
        while (g + 1 < hi && tab[g + 1].key <= k && ++steps < 8) ++g;
    } else {
        while (g > lo && tab[g].key > k && ++steps < 8) --g;
        if (tab[g].key > k) g = lo - 1;
    }
    if (steps >= 8) {
        int l = lo, h = hi;
        while (l < h) {
            const int mid = (l + h) >> 1;
            if (tab[mid].key <= k) l = mid + 1; else h = mid;
        }
        g = l - 1;
    }
    return g;
}

// Every weight, in the caller's order, finds its cluster by value: bucket ->
// directory (L2-resident) -> interpolated probe of the cluster table.  Each
// thread carries LK elements through every stage so that their independent
// random loads overlap.
template <typename T>
__global__ void __launch_bounds__(256) k_lookup(const T* __restrict__ values, const TileDesc* __restrict__ tiles,
                                                const LargeSeg* __restrict__ lsegs, const SegRuntime* __restrict__ rt,
                                                const CEntry<T>* __restrict__ table, const DirEntry* __restrict__ dir,
                                                T* out, int32_t* ids, uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int LK = 4;
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const SegRuntime R = rt[td.lseg];
    const int nb = 1 << R.dir_log2;
    const DirEntry* D = dir + ls.dir_pos;
    const CEntry<T>* tab = table + R.table_pos;
    const int c = (int)R.n_clusters;
    for (int i0 = threadIdx.x; i0 < td.len; i0 += 256 * LK) {
        T x[LK];
        K k[LK];
        int lo[LK], hi[LK], g[LK];
        DirEntry e0[LK], e1[LK];
        bool in[LK];
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            const int i = i0 + u * 256;
            in[u] = i < td.len;
            x[u] = in[u] ? values[td.vpos + i] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            k[u] = KO::to_key(x[u]);
            const int b = ws_bucket((float)x[u], R.lo, R.scale, nb);
            e0[u] = D[b];
            e1[u] = D[b + 1];
        }
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            const uint32_t k32 = (uint32_t)(k[u] >> (KO::BITS - 32));
            lo[u] = min(max(e0[u].idx, 0), c);
            hi[u] = min(max(e1[u].idx, lo[u]), c);
            if (lo[u] == hi[u] || k32 < e0[u].key32) {
                g[u] = -1;   // precedes every start in the bucket: cluster lo - 1
            } else {
                const uint32_t span = e1[u].key32 - e0[u].key32;
                int gg = lo[u];
                if (span > 0) {
                    const float f = (float)(k32 - e0[u].key32) / (float)span;
                    gg = lo[u] + (int)(f * (float)(hi[u] - lo[u]));
                    gg = min(max(gg, lo[u]), hi[u] - 1);
                }
                g[u] = gg;
            }
        }
        CEntry<T> cg[LK];
#pragma unroll
        for (int u = 0; u < LK; ++u) cg[u] = tab[g[u] >= 0 ? g[u] : max(lo[u] - 1, 0)];
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            int r;
            CEntry<T> ce = cg[u];
            if (g[u] < 0) {
                r = lo[u] - 1;
            } else {
                r = ws_find_cluster<T>(tab, lo[u], hi[u], g[u], k[u], ce.key);
                if (r != g[u] && r >= 0) ce = tab[r];
            }
            if (r < 0 || r >= c) { ws_flag(status, WS_STATUS_INTERNAL); r = 0; ce = tab[0]; }
            if (in[u]) {
                const int i = i0 + u * 256;
                out[td.vpos + i] = ce.val;
                if (ids) ids[td.vpos + i] = r;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// backward: per-cluster mean of grad_out (atomics into the cluster slots)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_bwd_accum(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                   const TileDesc* __restrict__ tiles,
                                                   const LargeSeg* __restrict__ lsegs, T* bsum, int32_t* bcnt,
                                                   uint32_t* status) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    for (int i = threadIdx.x; i < td.len; i += 256) {
        int id = ids[td.vpos + i];
        if (id < 0 || id >= ls.len) { ws_flag(status, WS_STATUS_INTERNAL); continue; }
        atomicAdd(&bsum[slot0 + id], g[td.vpos + i]);
        atomicAdd(&bcnt[slot0 + id], 1);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_bwd_apply(const int32_t* __restrict__ ids, const TileDesc* __restrict__ tiles,
                                                   const LargeSeg* __restrict__ lsegs, const T* __restrict__ bsum,
                                                   const int32_t* __restrict__ bcnt, T* gin) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    for (int i = threadIdx.x; i < td.len; i += 256) {
        int id = ids[td.vpos + i];
        if (id < 0 || id >= ls.len) continue;
        gin[td.vpos + i] = bsum[slot0 + id] / (T)bcnt[slot0 + id];
    }
}

template <typename T>
__global__ void k_copy_sorted(const typename KeyOf<T>::K* __restrict__ sorted, const TileDesc* __restrict__ tiles,
                              T* dst) {
    const TileDesc td = tiles[blockIdx.x];
    for (int i = threadIdx.x; i < td.len; i += 256) dst[td.vpos + i] = KeyOf<T>::from_key(sorted[td.kpos + i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// host-side sequencing of the large path
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t ws_large_prox(const LargeWork<T>& W, const T* values, const double* lambdas, T* out, int32_t* ids,
                          int64_t* n_clusters, int fp64, uint32_t* status, uint64_t spin_limit,
                          const MergeNode* const* level_nodes, const int* level_counts, int n_levels,
                          cudaStream_t st) {
    typedef typename KeyOf<T>::K K;
    if (W.n_lseg == 0) return cudaSuccess;
    K* sorted = nullptr;
    cudaError_t e = ws_large_sort<T>(W, values, status, spin_limit, st, &sorted);
    if (e) return e;
    size_t smem = sizeof(TileHullSmem);
    e = cudaFuncSetAttribute(k_tile_hull<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_TILE_HULL, st,
              (k_tile_hull<T><<<W.n_hull_tiles, HNT, smem, st>>>(sorted, W.hull_tiles, W.lsegs, lambdas, W.rt, W.vp,
                                                                W.vx, W.nvert, W.tile_total, W.pieces, W.npieces,
                                                                status)));
    WS_LAUNCH(W.prof, WSK_TILE_SCAN, st, (k_tile_scan<<<W.n_lseg, 256, 0, st>>>(W.lsegs, W.tile_total, W.tile_offset)));
    for (int l = 0; l < n_levels; ++l)
        if (level_counts[l] > 0)
            WS_LAUNCH(W.prof, WSK_MERGE, st,
                      (k_merge<T><<<level_counts[l], 256, 0, st>>>(level_nodes[l], W.lsegs, lambdas, W.rt, W.vp, W.vx,
                                                                  W.tile_offset, W.pieces, W.npieces, status)));
    e = cudaMemsetAsync(W.tile_piece, 0xff, sizeof(int32_t) * (size_t)W.n_hull_tiles, st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_ROOT, st,
              (k_root<T><<<W.n_lseg, 256, 0, st>>>(W.lsegs, sorted, W.pieces, W.npieces, W.tile_piece, W.rt,
                                                  n_clusters)));
    // big-gap list lives at the tail of the backward sum buffer (unused in the forward)
    uint32_t* ngaps = reinterpret_cast<uint32_t*>(W.bcnt);
    BigGap* gaps = reinterpret_cast<BigGap*>(W.bsum);
    int64_t gap_cap = (int64_t)((W.n_keys + W.n_lseg) * sizeof(T) / sizeof(BigGap));
    e = cudaMemsetAsync(ngaps, 0, sizeof(uint32_t), st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_TABLE, st,
              (k_table<T><<<W.n_hull_tiles, 256, 0, st>>>(W.hull_tiles, W.lsegs, lambdas, W.rt, sorted, W.vp, W.vx,
                                                         W.tile_offset, W.pieces, W.npieces, W.tile_piece, W.table,
                                                         W.dir, gaps, ngaps, gap_cap, fp64, status)));
    WS_LAUNCH(W.prof, WSK_BIG_GAPS, st, (k_big_gaps<<<1024, 256, 0, st>>>(gaps, ngaps, W.dir, gap_cap)));
    WS_LAUNCH(W.prof, WSK_LOOKUP, st,
              (k_lookup<T><<<W.n_sort_tiles, 256, 0, st>>>(values, W.sort_tiles, W.lsegs, W.rt, W.table, W.dir, out,
                                                          ids, status)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t ws_large_backward(const LargeWork<T>& W, const T* g, const int32_t* ids, T* gin, uint32_t* status,
                              cudaStream_t st) {
    if (W.n_lseg == 0) return cudaSuccess;
    size_t slots = (size_t)(W.n_keys + W.n_lseg);
    cudaError_t e = cudaMemsetAsync(W.bsum, 0, sizeof(T) * slots, st);
    if (e) return e;
    e = cudaMemsetAsync(W.bcnt, 0, sizeof(int32_t) * slots, st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_accum<T><<<W.n_sort_tiles, 256, 0, st>>>(g, ids, W.sort_tiles, W.lsegs, W.bsum, W.bcnt, status)));
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_apply<T><<<W.n_sort_tiles, 256, 0, st>>>(ids, W.sort_tiles, W.lsegs, W.bsum, W.bcnt, gin)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t ws_large_copy_sorted(const LargeWork<T>& W, const typename KeyOf<T>::K* sorted, T* dst,
                                 cudaStream_t st) {
    if (W.n_sort_tiles == 0) return cudaSuccess;
    WS_LAUNCH(W.prof, WSK_MISC, st, (k_copy_sorted<T><<<W.n_sort_tiles, 256, 0, st>>>(sorted, W.sort_tiles, dst)));
    return cudaGetLastError();
}

#define WS_INST(T)                                                                                                  \
    template cudaError_t ws_large_prox<T>(const LargeWork<T>&, const T*, const double*, T*, int32_t*, int64_t*, int, \
                                          uint32_t*, uint64_t, const MergeNode* const*, const int*, int,            \
                                          cudaStream_t);                                                            \
    template cudaError_t ws_large_backward<T>(const LargeWork<T>&, const T*, const int32_t*, T*, uint32_t*,         \
                                              cudaStream_t);                                                        \
    template cudaError_t ws_large_copy_sorted<T>(const LargeWork<T>&, const typename KeyOf<T>::K*, T*, cudaStream_t);
WS_INST(float)
WS_INST(double)
