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
// 2. merging two adjacent node hulls (run by the CTA that arrives last)
//
// Piece lists are rewritten in place as the tree climbs, by whichever CTA
// merges a node, so they are read through L2 (ld.global.cg): an SM's L1 may
// still hold a line of a list another SM has since rewritten.
// ---------------------------------------------------------------------------
__device__ __forceinline__ Piece ws_ld_piece(const Piece* p) {
    const uint4* q = reinterpret_cast<const uint4*>(p);
    uint4 a = __ldcg(q), b = __ldcg(q + 1);
    Piece r;
    *reinterpret_cast<uint4*>(&r) = a;
    *(reinterpret_cast<uint4*>(&r) + 1) = b;
    return r;
}
__device__ __forceinline__ void ws_st_piece(Piece* p, const Piece& v) {
    uint4* q = reinterpret_cast<uint4*>(p);
    __stcg(q, *reinterpret_cast<const uint4*>(&v));
    __stcg(q + 1, *(reinterpret_cast<const uint4*>(&v) + 1));
}
__device__ __forceinline__ i128 ws_ld_i128(const i128* p) {
    const uint4 v = __ldcg(reinterpret_cast<const uint4*>(p));
    return *reinterpret_cast<const i128*>(&v);
}

struct NodeView {
    const Piece* pc;   // piece list
    int np;            // pieces
    const uint16_t* vp;
    const i128* vx;
    int hull_first;    // global index of the segment's first hull tile
    i128 base;         // X offset of this node's first point in the merge frame
    __device__ __forceinline__ int find(int r) const {   // piece holding rank r
        int lo = 0, hi = np - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (ws_ld_piece(pc + mid).cum <= r) lo = mid; else hi = mid - 1;
        }
        return lo;
    }
    __device__ __forceinline__ void get(int r, int64_t& pt, i128& X) const {
        const Piece p = ws_ld_piece(pc + find(r));
        size_t v = (size_t)p.tile * (HT + 1) + p.lo + (r - p.cum);
        pt = (int64_t)(p.tile - hull_first) * HT + vp[v];
        X = base + p.off + vx[v];
    }
    __device__ __forceinline__ int count() const {
        if (np == 0) return 0;
        const Piece p = ws_ld_piece(pc + np - 1);
        return p.cum + (p.hi - p.lo);
    }
};

__device__ __forceinline__ void ws_piece_vertex(const Piece& q, int v, const uint16_t* vp, const i128* vx,
                                                int hull_first, i128 base, int64_t& pt, i128& X) {
    const size_t idx = (size_t)q.tile * (HT + 1) + v;
    pt = (int64_t)(q.tile - hull_first) * HT + vp[idx];
    X = base + q.off + vx[idx];
}

// Bridge between two node hulls by walking outward from their junction
// (the linear merge of two convex chains), stepping through the piece lists
// directly.  Returns false (no result) after too many steps; the caller then
// runs the galloping search.  Same outputs as ws_bridge.
__device__ bool ws_bridge_walk(const Piece* PL, int npL, const Piece* PR, int npR, const uint16_t* vp,
                               const i128* vx, int hull_first, i128 baseR, const SegConst& sc, int& flag, int& istar,
                               int& jstar) {
    int lp = npL - 1, rp = 0;
    Piece qL = ws_ld_piece(PL + lp), qR = ws_ld_piece(PR + rp);
    int lv = qL.hi - 1, rv = qR.lo;   // L_p and R_0: the junction
    auto prevL = [&](int& p, Piece& q, int& v) -> bool {
        if (v > q.lo) { --v; return true; }
        if (p == 0) return false;
        --p; q = ws_ld_piece(PL + p); v = q.hi - 1; return true;
    };
    auto nextR = [&](int& p, Piece& q, int& v) -> bool {
        if (v + 1 < q.hi) { ++v; return true; }
        if (p + 1 >= npR) return false;
        ++p; q = ws_ld_piece(PR + p); v = q.lo; return true;
    };
    int64_t pj; i128 Xj;
    ws_piece_vertex(qR, rv, vp, vx, hull_first, baseR, pj, Xj);
    if (!prevL(lp, qL, lv) || !nextR(rp, qR, rv)) { flag = 0; return true; }
    int64_t pl, pr; i128 Xl, Xr;
    ws_piece_vertex(qL, lv, vp, vx, hull_first, 0, pl, Xl);
    ws_piece_vertex(qR, rv, vp, vx, hull_first, baseR, pr, Xr);
    if (ws_convex(Xl, Xj, Xr, pl, pj, pr, sc)) { flag = 0; return true; }
    flag = 1;
    int steps = 0;
    constexpr int WALK_MAX = 32;
    while (true) {
        bool moved = false;
        while (true) {
            int p2 = lp, v2 = lv;
            Piece q2 = qL;
            if (!prevL(p2, q2, v2)) break;
            int64_t pm; i128 Xm;
            ws_piece_vertex(q2, v2, vp, vx, hull_first, 0, pm, Xm);
            if (ws_convex(Xm, Xl, Xr, pm, pl, pr, sc)) break;
            lp = p2; qL = q2; lv = v2; pl = pm; Xl = Xm; moved = true;
            if (++steps > WALK_MAX) return false;
        }
        while (true) {
            int p2 = rp, v2 = rv;
            Piece q2 = qR;
            if (!nextR(p2, q2, v2)) break;
            int64_t pn; i128 Xn;
            ws_piece_vertex(q2, v2, vp, vx, hull_first, baseR, pn, Xn);
            if (ws_convex(Xl, Xr, Xn, pl, pr, pn, sc)) break;
            rp = p2; qR = q2; rv = v2; pr = pn; Xr = Xn; moved = true;
            if (++steps > WALK_MAX) return false;
        }
        if (!moved) break;
    }
    istar = qL.cum + (lv - qL.lo);
    jstar = qR.cum + (rv - qR.lo);
    return true;
}

constexpr int MW = 16;   // vertices of each child prefetched around the junction

struct MergeSmem {
    int is, js, pl, pr, npL, npR;
    i128 totL, totR;
    int wsi[8];
    // window: the last MW vertices of L (index 0 = L_p, the junction, going
    // left) and the first MW of R (index 0 = R_0 = junction, going right)
    Piece wpL[MW], wpR[MW];        // the pieces at the ends of the two lists
    int nwpL, nwpR;
    int wLn, wRn;                  // vertices in each window
    int wLpc[MW], wLv[MW], wRpc[MW], wRv[MW];   // (piece slot in the list, vertex index)
    int64_t wLpt[MW], wRpt[MW];
    i128 wLX[MW], wRX[MW];
    int ok;
    int cand_i[HNT / 32], cand_s[HNT / 32], cand_j[HNT / 32];   // parallel search: one candidate per warp
};

// Vertex of rank r of a node hull whose piece list is cached in shared memory.
__device__ __forceinline__ void ws_cached_vertex(const Piece* c, int np, int r, const uint16_t* vp, const i128* vx,
                                                 int hull_first, i128 base, int64_t& pt, i128& X) {
    int lo = 0, hi = np - 1;   // the last piece whose first rank is <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c[mid].cum <= r) lo = mid; else hi = mid - 1;
    }
    ws_piece_vertex(c[lo], c[lo].lo + (r - c[lo].cum), vp, vx, hull_first, base, pt, X);
}
__device__ __forceinline__ int ws_cached_find(const Piece* c, int np, int r) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (c[mid].cum <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The bridge of two node hulls searched by the whole CTA, for merges whose
// bridge lies beyond the prefetched window (typically near the root, where
// one side loses thousands of vertices).  Same definitions as ws_bridge:
// right(i, j) = R_{j+1} on or below the line (L_i, R_j); tangent(i) = the
// first j with !right(i, j) (right(i, .) is true then false along the convex
// chain R); survives(i) = i == 0 or L_{i-1}, L_i, R_tangent(i) convex
// (survivors are a prefix of L); istar = the last survivor below the
// junction, jstar = tangent(istar).  Each round of the outer search gives
// one candidate i to each warp; a warp finds tangent(i) by a 32-way search
// (every lane tests one j), so a merge costs about log_9(p) * log_33(q)
// rounds instead of a serial gallop through global memory.  Requires the
// junction not to be a vertex and both hulls to have >= 2 vertices.  The
// piece lists are copied into `cache` (capacity >= npL + npR).  All threads
// call it; it ends synchronised with m.is/js/pl/pr set and m.ok = 1.
__device__ void ws_parallel_bridge(Piece* cache, MergeSmem& m, const Piece* PL, const Piece* PR, const uint16_t* vp,
                                   const i128* vx, int hull_first, const SegConst& sc) {
    constexpr int NW = HNT / 32;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int npL = m.npL, npR = m.npR;
    Piece* cL = cache;
    Piece* cR = cache + npL;
    for (int k = t; k < npL + npR; k += HNT) cache[k] = ws_ld_piece(k < npL ? PL + k : PR + (k - npL));
    __syncthreads();
    const int p = cL[npL - 1].cum + (cL[npL - 1].hi - cL[npL - 1].lo) - 1;   // L_p = R_0: the junction
    const int q = cR[npR - 1].cum + (cR[npR - 1].hi - cR[npR - 1].lo) - 1;
    const i128 baseR = m.totL;
    if (p < 1 || q < 1) return;   // (not reached from the window walk) left to the serial search
    if (t == 0) {   // the junction stays a vertex: keep all of L, drop R_0 (as ws_bridge's flag 0)
        int64_t pa, pb, pc;
        i128 Xa, Xb, Xc;
        ws_cached_vertex(cL, npL, p - 1, vp, vx, hull_first, 0, pa, Xa);
        ws_cached_vertex(cL, npL, p, vp, vx, hull_first, 0, pb, Xb);
        ws_cached_vertex(cR, npR, 1, vp, vx, hull_first, baseR, pc, Xc);
        m.cand_s[0] = ws_convex(Xa, Xb, Xc, pa, pb, pc, sc) ? 1 : 0;
        if (m.cand_s[0]) {
            m.is = p; m.js = 1;
            m.pl = ws_cached_find(cL, npL, p);
            m.pr = ws_cached_find(cR, npR, 1);
            m.ok = 1;
        }
    }
    __syncthreads();
    const bool junction_vertex = m.cand_s[0] != 0;
    __syncthreads();   // every thread has read the flag before the search reuses cand_s
    if (junction_vertex) return;   // (m.ok set)
    // first j in [0, q] with !right(i, j), by the whole warp
    auto tangent = [&](int64_t pi, const i128& Xi) -> int {
        int jl = -1, jh = q;   // right(i, jl) (or jl = -1), !right(i, jh) (jh = q: no R_{q+1})
        while (jh - jl > 1) {
            const int span = jh - jl - 1;   // candidates jl + 1 .. jh - 1
            const int j = (span <= 32) ? jl + 1 + lane : jl + 1 + (int)(((long long)span * lane) >> 5);
            const bool valid = j < jh;
            bool rt = false;
            if (valid) {
                int64_t pj, pk;
                i128 Xj, Xk;
                ws_cached_vertex(cR, npR, j, vp, vx, hull_first, baseR, pj, Xj);
                ws_cached_vertex(cR, npR, j + 1, vp, vx, hull_first, baseR, pk, Xk);
                rt = !ws_convex(Xi, Xj, Xk, pi, pj, pk, sc);
            }
            const unsigned bt = __ballot_sync(WS_FULL_MASK, valid && rt);
            const unsigned bf = __ballot_sync(WS_FULL_MASK, valid && !rt);
            if (bt) jl = __shfl_sync(WS_FULL_MASK, j, 31 - __clz((int)bt));
            if (bf) jh = __shfl_sync(WS_FULL_MASK, j, __ffs((int)bf) - 1);
        }
        return jh;
    };
    int good = 0, bad = p, jgood = -1;   // survives(good), !survives(bad) (bad = p: the junction)
    while (bad - good > 1) {
        const int span = bad - good - 1;
        const int c = (span <= NW) ? good + 1 + w : good + 1 + (int)(((long long)span * w) / NW);
        if (c < bad) {
            int64_t pc;
            i128 Xc;
            ws_cached_vertex(cL, npL, c, vp, vx, hull_first, 0, pc, Xc);
            const int jt = tangent(pc, Xc);
            if (lane == 0) {
                int64_t pm, pt;
                i128 Xm, Xt;
                ws_cached_vertex(cL, npL, c - 1, vp, vx, hull_first, 0, pm, Xm);
                ws_cached_vertex(cR, npR, jt, vp, vx, hull_first, baseR, pt, Xt);
                m.cand_i[w] = c;
                m.cand_j[w] = jt;
                m.cand_s[w] = ws_convex(Xm, Xc, Xt, pm, pc, pt, sc) ? 1 : 0;
            }
        } else if (lane == 0) {
            m.cand_i[w] = -1;
        }
        __syncthreads();
        int ng = good, nb = bad, nj = jgood;
        for (int k = 0; k < NW; ++k) {
            const int ci = m.cand_i[k];
            if (ci < 0) continue;
            if (m.cand_s[k]) { if (ci > ng) { ng = ci; nj = m.cand_j[k]; } }
            else if (ci < nb) nb = ci;
        }
        good = ng; bad = nb; jgood = nj;
        __syncthreads();
    }
    if (jgood < 0 && w == 0) {   // istar = 0 was never a candidate: its tangent
        int64_t p0;
        i128 X0;
        ws_cached_vertex(cL, npL, 0, vp, vx, hull_first, 0, p0, X0);
        const int jt = tangent(p0, X0);
        if (lane == 0) m.cand_j[0] = jt;
    }
    __syncthreads();
    if (t == 0) {
        const int js = jgood >= 0 ? jgood : m.cand_j[0];
        m.is = good;
        m.js = js;
        m.pl = ws_cached_find(cL, npL, good);
        m.pr = js <= q ? ws_cached_find(cR, npR, js) : npR;
        m.ok = 1;
    }
    __syncthreads();
}

// Merge the node hulls whose piece lists start at Lg and Rg (global hull-tile
// indices, Rg > Lg adjacent); the result replaces the list at Lg.  All
// threads of the CTA call this.  Warp 0 first gathers, in parallel, the
// vertices next to the junction (usually all the bridge needs); thread 0
// walks them in shared memory and falls back to the global search only if
// the bridge leaves that window.
__device__ __noinline__ void ws_merge_children(MergeSmem& m, Piece* pieces, int32_t* npieces, i128* ntotal, int Lg, int Rg,
                                  const uint16_t* vp, const i128* vx, int hull_first, const SegConst& sc,
                                  Piece* cache, int cache_cap) {
    const int t = threadIdx.x;
    Piece* PL = pieces + Lg;
    Piece* PR = pieces + Rg;
    if (t < 32) {
        const int npL = __ldcg(npieces + Lg), npR = __ldcg(npieces + Rg);
        // the last MW pieces of L (slot 0 = last) and the first MW of R
        if (t < MW) { if (t < npL) m.wpL[t] = ws_ld_piece(PL + npL - 1 - t); }
        else { const int k = t - MW; if (k < npR) m.wpR[k] = ws_ld_piece(PR + k); }
        if (t == 0) {
            m.npL = npL; m.npR = npR;
            m.totL = ws_ld_i128(ntotal + Lg);
            m.totR = ws_ld_i128(ntotal + Rg);
            m.nwpL = min(npL, MW); m.nwpR = min(npR, MW);
        }
        __syncwarp();
        if (t == 0) {   // enumerate the window's vertices
            int n = 0;
            for (int k = 0; k < m.nwpL && n < MW; ++k) {
                const Piece q = m.wpL[k];
                for (int v = q.hi - 1; v >= (int)q.lo && n < MW; --v) { m.wLpc[n] = npL - 1 - k; m.wLv[n] = v; ++n; }
            }
            m.wLn = n;
            n = 0;
            for (int k = 0; k < m.nwpR && n < MW; ++k) {
                const Piece q = m.wpR[k];
                for (int v = q.lo; v < (int)q.hi && n < MW; ++v) { m.wRpc[n] = k; m.wRv[n] = v; ++n; }
            }
            m.wRn = n;
        }
        __syncwarp();
        if (t < MW) {
            if (t < m.wLn) {
                const Piece q = m.wpL[npL - 1 - m.wLpc[t]];
                ws_piece_vertex(q, m.wLv[t], vp, vx, hull_first, 0, m.wLpt[t], m.wLX[t]);
            }
        } else {
            const int k = t - MW;
            if (k < m.wRn) {
                const Piece q = m.wpR[m.wRpc[k]];
                ws_piece_vertex(q, m.wRv[k], vp, vx, hull_first, m.totL, m.wRpt[k], m.wRX[k]);
            }
        }
        __syncwarp();
        if (t == 0) {
            // walk in the window: li indexes wL (0 = junction), rj indexes wR (0 = junction)
            const int nL = m.wLn, nR = m.wRn;
            int flag = 0, li = 0, rj = 0;
            bool ok = true;
            const bool Lmore = nL == MW, Rmore = nR == MW;   // a list may continue past the window
            if (nL >= 2 && nR >= 2) {
                if (!ws_convex(m.wLX[1], m.wLX[0], m.wRX[1], m.wLpt[1], m.wLpt[0], m.wRpt[1], sc)) {
                    flag = 1; li = 1; rj = 1;
                    while (ok) {
                        bool moved = false;
                        while (true) {
                            if (li + 1 >= nL) { if (Lmore) ok = false; break; }
                            if (ws_convex(m.wLX[li + 1], m.wLX[li], m.wRX[rj], m.wLpt[li + 1], m.wLpt[li], m.wRpt[rj], sc))
                                break;
                            ++li; moved = true;
                        }
                        if (!ok) break;
                        while (true) {
                            if (rj + 1 >= nR) { if (Rmore) ok = false; break; }
                            if (ws_convex(m.wLX[li], m.wRX[rj], m.wRX[rj + 1], m.wLpt[li], m.wRpt[rj], m.wRpt[rj + 1], sc))
                                break;
                            ++rj; moved = true;
                        }
                        if (!moved) break;
                    }
                }
            } else if (!(nL == 1 || nR == 1)) {
                ok = false;
            }
            if (ok) {
                // (the pieces named here are in the window: its copies, not global memory)
                if (flag == 0) {   // junction stays: keep all of L, drop R_0
                    m.pl = npL - 1;
                    const Piece qL = m.wpL[0];
                    m.is = qL.cum + (qL.hi - qL.lo) - 1;
                    m.js = 1;
                    if (nR >= 2) { m.pr = m.wRpc[1]; } else { m.pr = npR; }
                } else {
                    m.pl = m.wLpc[li];
                    m.pr = m.wRpc[rj];
                    const Piece qL = m.wpL[npL - 1 - m.pl];
                    const Piece qR = m.wpR[m.pr];
                    m.is = qL.cum + (m.wLv[li] - qL.lo);
                    m.js = qR.cum + (m.wRv[rj] - qR.lo);
                }
                if (nL == 1 || nR == 1) { m.pl = npL - 1; m.is = -1; m.pr = (nR >= 2) ? m.wRpc[1] : npR; m.js = 1; }
            }
            m.ok = ok ? 1 : 0;
        }
        __syncwarp();
    }
    __syncthreads();
    // the bridge reaches beyond the window: the CTA searches it in parallel
    // (the serial walk and gallop below remain for lists too long to cache)
    if (!m.ok && m.npL + m.npR <= cache_cap) ws_parallel_bridge(cache, m, PL, PR, vp, vx, hull_first, sc);
    if (t == 0) {
        const int npL = m.npL, npR = m.npR;
        const i128 totL = m.totL;
        if (!m.ok) {   // the bridge reaches beyond the window: global walk, then the gallop
            NodeView L{PL, npL, vp, vx, hull_first, 0};
            NodeView R{PR, npR, vp, vx, hull_first, totL};
            const int nL = L.count(), nR = R.count();
            int flag = 0, is = nL - 1, js = 0;
            if (nL > 0 && nR > 0) {
                if (!ws_bridge_walk(PL, npL, PR, npR, vp, vx, hull_first, totL, sc, flag, is, js)) {
                    auto gl = [&](int r, int64_t& pt, i128& X) { L.get(r, pt, X); };
                    auto gr = [&](int r, int64_t& pt, i128& X) { R.get(r, pt, X); };
                    ws_bridge(gl, nL - 1, gr, nR - 1, sc, flag, is, js);
                }
                if (flag == 0) { is = nL - 1; js = 1; }
            }
            m.pl = (nL > 0) ? L.find(is) : -1;
            m.pr = (nR > 0 && js < nR) ? R.find(js) : npR;
            m.is = is; m.js = js;
        }
        if (m.pl >= 0 && m.is >= 0) {   // truncate the left list after istar
            const int slot = npL - 1 - m.pl;
            Piece q = slot < m.nwpL ? m.wpL[slot] : ws_ld_piece(PL + m.pl);
            q.hi = (uint16_t)(q.lo + (m.is - q.cum) + 1);
            ws_st_piece(PL + m.pl, q);
        }
        if (m.pr < npR) {  // the right list starts at jstar
            const bool in_window = m.pr < m.nwpR;
            Piece q = in_window ? m.wpR[m.pr] : ws_ld_piece(PR + m.pr);
            q.lo = (uint16_t)(q.lo + (m.js - q.cum));
            ws_st_piece(PR + m.pr, q);
            if (in_window) m.wpR[m.pr] = q;   // the copy below reads the window
        }
    }
    __syncthreads();
    const int keepL = m.pl + 1, firstR = m.pr, keepR = m.npR - m.pr;
    const i128 totL = m.totL;
    // Move the right suffix down behind the left prefix (dst <= src: chunked),
    // rebasing offsets onto the left node's first point.  Ranks of the kept
    // left pieces are unchanged; the right ones shift uniformly: the first
    // kept right piece starts at rank istar + 1.
    const int shift = m.is + 1 - m.js;
    for (int b = 0; b < keepR; b += 256) {
        Piece v;
        const bool has = b + t < keepR;
        if (has) {
            const int k = firstR + b + t;
            v = k < m.nwpR ? m.wpR[k] : ws_ld_piece(PR + k);
            v.off += totL;
            v.cum = (b + t == 0) ? m.is + 1 : v.cum + shift;
        }
        __syncthreads();
        if (has) ws_st_piece(PL + keepL + b + t, v);
        __syncthreads();
    }
    const int np = keepL + keepR;
    if (t == 0) {
        __stcg(npieces + Lg, np);
        const i128 tot = m.totL + m.totR;
        __stcg(reinterpret_cast<uint4*>(ntotal + Lg), *reinterpret_cast<const uint4*>(&tot));
    }
}

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

// The general tile kernel: the exact hull of a tile whose prefix sums need
// 128 bits (or whose bridge walks were too long for the lean kernel of
// ws_tile.cu, which lists such tiles in gen_list).  A small grid walks the
// list.  Four CTAs per SM (64 registers; only the rare merge paths spill).
template <typename T>
__global__ void __launch_bounds__(HNT, 4) k_tile_hull(const typename KeyOf<T>::K* __restrict__ sorted,
                                                   const TileDesc* __restrict__ htiles,
                                                   const LargeSeg* __restrict__ lsegs,
                                                   const double* __restrict__ lambdas, SegRuntime* rt,
                                                   uint16_t* vp, i128* vx, int32_t* nvert, i128* tile_total,
                                                   const int32_t* __restrict__ gen_list,
                                                   const int32_t* __restrict__ gen_count,
                                                   const int32_t* __restrict__ seg_emin, uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileHullSmem& s = *reinterpret_cast<TileHullSmem*>(smem_raw);
    const int t = threadIdx.x;
    const int n_list = *gen_count;
    for (int li = blockIdx.x; li < n_list; li += gridDim.x) {
    __syncthreads();   // (the previous tile's shared memory is dead)
    const int tile = gen_list[li];
    const TileDesc td = htiles[tile];
    const LargeSeg ls = lsegs[td.lseg];
    const double lam = lambdas[ls.seg];
    const bool lam_ok = lam >= 0.0 && lam <= 1.7976931348623157e308;
    const double lamv = lam_ok ? lam : 0.0;
    const int n = td.len;
    const K* kp = sorted + td.kpos;
    const K kfirst = kp[0], klast = kp[n - 1];
    const T xlo = KO::from_key(sorted[ls.kpos]), xhi = KO::from_key(sorted[ls.kpos + ls.len - 1]);
    const int emax = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[td.lseg]);
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
    // this thread's entry of the chain thresholds, at the scale the tile's mode uses
    // (computed while the keys are in flight; stored by the prefix after its first barrier)
    static_assert(HM * HM <= HNT, "one threshold entry per thread");
    int thr_v = 0;
    if (t < HM * HM) {
        int shb;
        const bool tbin = ws_tile_binade<T>(kfirst, klast, n, emax, shb);
        uint64_t mlam;
        int sx;
        ws_thr_consts(lamv, KO::L_BASE - emax - (tbin && shb > 0 ? shb : 0), mlam, sx);
        thr_v = ws_thr_entry<HM>(t, mlam, sx, ls.len > 1 ? (uint64_t)(ls.len - 1) : 1ull);
    }
    int64_t q0;
    i128 total;
    int bsh;
    const int mode = ws_tile_prefix<T, HNT, HM>(s.pre, kr, kfirst, klast, n, emax, q0, total, bsh,
                                                t < HM * HM ? s.hull.thr + t : nullptr, thr_v);
    int nv;
    if (mode == WS_TILE_BINADE) {
        TilePtsDev<HM> P = ws_dev_pts<HM>(s.pre.s64, s.muqt, s.fastt != 0, (uint64_t)(klast - kfirst), n, s.sct);
        P.thr = s.hull.thr;
        ws_cta_hull<HNT, HM>(s.hull, n, P, s.sct, &nv);
    } else if (mode == WS_TILE_NARROW) {
        const uint64_t range = (uint64_t)(ws_fixed<T>(KO::from_key(klast), emax) - q0);
        TilePtsDev<HM> P = ws_dev_pts<HM>(s.pre.s64, s.muq, s.fast != 0, range, n, s.sc);
        P.thr = s.hull.thr;
        ws_cta_hull<HNT, HM>(s.hull, n, P, s.sc, &nv);
    } else {
        const TilePtsWide<HM> P{s.pre.s64, s.pre.base};
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
        __stcg(reinterpret_cast<uint4*>(tile_total + tile), *reinterpret_cast<const uint4*>(&total));
    }
    }
}

// ---------------------------------------------------------------------------
// 3. the tree of bridge merges across tiles, for segments whose junctions do
// not resolve locally (seg_mode 2).  All tile hulls are written.  A CTA takes
// one hull tile after another (a small grid); for each it starts the tile's
// node list, then climbs: at each level the CTA that arrives second merges
// the two children of the parent, the first one goes on to its next tile.
// Nobody waits.
// ---------------------------------------------------------------------------
constexpr int CLIMB_CACHE = 1024;   // piece lists up to this long are searched from shared memory

struct ClimbSmem {
    MergeSmem ms;
    Piece cache[CLIMB_CACHE];
    int go;
    SegConst sc;
};

template <typename T>
__global__ void __launch_bounds__(HNT) k_climb(const TileDesc* __restrict__ htiles, const LargeSeg* __restrict__ lsegs,
                                               const double* __restrict__ lambdas,
                                               const SegRuntime* __restrict__ rt, const uint16_t* vp, const i128* vx,
                                               const int32_t* __restrict__ nvert, i128* tile_total, Piece* pieces,
                                               int32_t* npieces, int32_t* arrive, int n_hull,
                                               const int32_t* __restrict__ seg_mode) {
    __shared__ ClimbSmem s;
    const int t = threadIdx.x;
    // Most calls have no segment left for the tree: all threads check this
    // CTA's tiles at once, instead of one tile per round trip in the loop below.
    bool any = false;
    for (int tile = blockIdx.x + t * gridDim.x; tile < n_hull; tile += HNT * gridDim.x)
        any |= seg_mode[htiles[tile].lseg] == 2;
    if (!__syncthreads_or(any)) return;
    for (int tile = blockIdx.x; tile < n_hull; tile += gridDim.x) {
    const TileDesc td = htiles[tile];
    if (seg_mode[td.lseg] != 2) continue;   // (uniform)
    __syncthreads();   // (the previous tile's shared memory is dead)
    const LargeSeg ls = lsegs[td.lseg];
    if (t == 0) {
        double lam = lambdas[ls.seg];
        if (!(lam >= 0.0) || !(lam <= 1.7976931348623157e308)) lam = 0.0;
        s.sc = ws_seg_const<T>(ls.len, lam, rt[td.lseg].emax);
        Piece pc;
        pc.tile = tile; pc.lo = 0; pc.hi = (uint16_t)nvert[tile]; pc.cum = 0; pc.pad = 0; pc.off = 0;
        ws_st_piece(pieces + tile, pc);
        __stcg(npieces + tile, 1);
    }
    __syncthreads();
    const int nt = ls.hull_count, tin = td.tin;
    for (int level = 0; (1 << level) < nt; ++level) {
        const int span = 1 << level;
        const int parent_base = (tin >> (level + 1)) << (level + 1);
        const int right_base = parent_base + span;
        if (right_base >= nt) continue;   // no right sibling: the parent is this node
        __threadfence();                  // this CTA's writes of the child are visible GPU-wide ...
        __syncthreads();
        if (t == 0) {                     // ... before its arrival is counted
            const int old = atomicAdd(&arrive[(size_t)(level + 1) * n_hull + ls.hull_first + parent_base], 1);
            __threadfence();
            s.go = (old == 1);
        }
        __syncthreads();
        if (!s.go) break;
        ws_merge_children(s.ms, pieces, npieces, tile_total, ls.hull_first + parent_base, ls.hull_first + right_base,
                          vp, vx, ls.hull_first, s.sc, s.cache, CLIMB_CACHE);
    }
    }
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
// 5. cluster table + directory fill (one CTA per hull tile; eight CTAs per
//    SM at 32 registers: its reads are latency bound, so warps beat registers)
// ---------------------------------------------------------------------------
constexpr int GAP_INLINE = 64;

struct BigGap { int64_t pos; int32_t count; int32_t value; uint32_t key32; int32_t pad; };

template <typename T>
__global__ void __launch_bounds__(256, 8) k_table(const TileDesc* __restrict__ htiles, const LargeSeg* __restrict__ lsegs,
                                               const double* __restrict__ lambdas, const SegRuntime* __restrict__ rt,
                                               const typename KeyOf<T>::K* __restrict__ sorted,
                                               const uint16_t* __restrict__ vp, const i128* __restrict__ vx,
                                               const Piece* __restrict__ pieces,
                                               const int32_t* __restrict__ npieces,
                                               const int32_t* __restrict__ tile_piece, CEntry<T>* table,
                                               DirEntry* dir, BigGap* gaps, uint32_t* ngaps, int64_t gap_cap,
                                               int fp64, const WsEpi ep, uint32_t* status) {
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
    const uint64_t pol = ws_policy_evict_last();
    auto vertex = [&](int piece_idx, int i, int64_t& pt, i128& X) {
        const Piece q = P[piece_idx];
        size_t v = (size_t)q.tile * (HT + 1) + i;
        pt = (int64_t)(q.tile - ls.hull_first) * HT + vp[v];
        X = q.off + vx[v];
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
        ce.val = ValueOut<T>::value(Xb - Xa, a, b, xs, sc, fp64 != 0, ep);
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
            for (int64_t bb = from; bb <= to; ++bb) ws_st_u2_last(D + bb, make_uint2((uint32_t)de.idx, de.key32), pol);
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
                for (int64_t bb = f2; bb <= nb; ++bb) ws_st_u2_last(D + bb, make_uint2((uint32_t)te.idx, te.key32), pol);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_big_gaps(const BigGap* gaps, const uint32_t* ngaps, DirEntry* dir,
                                                  int64_t gap_cap) {
    const int64_t n = min((int64_t)*ngaps, gap_cap);
    const uint64_t pol = ws_policy_evict_last();
    for (int64_t g = blockIdx.x; g < n; g += gridDim.x) {
        const BigGap G = gaps[g];
        const DirEntry e{G.value, G.key32};
        for (int i = threadIdx.x; i < G.count; i += 256) ws_st_u2_last(dir + G.pos + i, make_uint2((uint32_t)e.idx, e.key32), pol);
    }
}

// ---------------------------------------------------------------------------
// 6. lookup: every weight, in the caller's order, finds its cluster by value
// ---------------------------------------------------------------------------
// The cluster table is read a whole 32-byte sector at a time (E entries): the
// sector holding the interpolated guess almost always contains the answer,
// so a weight costs about one random sector instead of one per probed entry.
template <typename T>
struct TabSector {
    static constexpr int E = 32 / (int)sizeof(CEntry<T>);
    CEntry<T> e[E];
    __device__ __forceinline__ void load(const CEntry<T>* table, int64_t sb) {
        const uint4* p = reinterpret_cast<const uint4*>(table + sb);
        uint4 v[2];
        v[0] = __ldg(p);
        v[1] = __ldg(p + 1);
        const CEntry<T>* q = reinterpret_cast<const CEntry<T>*>(v);
#pragma unroll
        for (int i = 0; i < E; ++i) e[i] = q[i];
    }
};

// Last cluster j in [jlo, jhi] (segment-local, keys ascending, key[jlo] <= k)
// whose start key is <= k, starting at the sector that holds local index j0
// and walking sector by sector (at most four, then bisection).
template <typename T>
__device__ __forceinline__ int ws_find_cluster(const CEntry<T>* table, int64_t tp, int jlo, int jhi, int j0,
                                               typename KeyOf<T>::K k, CEntry<T>& out) {
    constexpr int E = TabSector<T>::E;
    int j = min(max(j0, jlo), jhi);
    int best = -1, dir = 0;
    for (int it = 0; it < 4; ++it) {
        const int64_t sb = (tp + j) & ~(int64_t)(E - 1);
        const int s0 = (int)(sb - tp);
        TabSector<T> S;
        S.load(table, sb);
        int last_le = -1, top = -1;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int li = s0 + i;
            if (li < jlo || li > jhi) continue;
            top = li;
            if (S.e[i].key <= k) { last_le = li; out = S.e[i]; }
        }
        if (last_le < 0) {              // every entry here is above k
            if (dir > 0) return best;   // ... and the previous sector's last one was not: out holds it
            if (s0 - 1 < jlo) break;    // (cannot happen: key[jlo] <= k)
            dir = -1;                   // the answer lies further left
            j = s0 - 1;
            continue;
        }
        best = last_le;
        // an entry above k follows inside this sector, the range ends here, or
        // the sector to the right was all above k: the answer is here
        if (last_le < top || last_le == jhi || dir < 0) return best;
        dir = 1;
        j = s0 + E;
    }
    int l = jlo, h = jhi + 1;   // bisection fallback
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (table[tp + mid].key <= k) l = mid + 1; else h = mid;
    }
    // key[jlo] <= k keeps l >= jlo + 1; the clamp only guards the read
    out = table[tp + max(l - 1, jlo)];
    return l - 1;
}

// Every weight, in the caller's order, finds its cluster by value: bucket ->
// directory (L2-resident) -> interpolated guess -> the table sector holding
// it.  Each thread carries LK elements through every stage so that their
// independent random loads overlap.
template <typename T>
__global__ void __launch_bounds__(256) k_lookup(const T* __restrict__ values, const TileDesc* __restrict__ tiles,
                                                const LargeSeg* __restrict__ lsegs, const SegRuntime* __restrict__ rt,
                                                const CEntry<T>* __restrict__ table, const DirEntry* __restrict__ dir,
                                                T* out, int32_t* ids, uint32_t* status) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int LK = 2;   // measured: 2 beats 1, 4 and 8 (occupancy against loads in flight)
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const SegRuntime R = rt[td.lseg];
    const int nb = 1 << R.dir_log2;
    const DirEntry* D = dir + ls.dir_pos;
    const int64_t tp = R.table_pos;
    const int c = (int)R.n_clusters;
    if (c == 1) {   // one cluster (large lambda): every weight gets its value, no search
        const T v = table[tp].val;
        for (int i = threadIdx.x; i < td.len; i += 256) {
            __stcs(out + td.vpos + i, v);
            if (ids) __stcs(ids + td.vpos + i, 0);
        }
        return;
    }
    const uint64_t pol = ws_policy_evict_last();
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
            x[u] = in[u] ? __ldcs(values + td.vpos + i) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            k[u] = KO::to_key(x[u]);
            const int b = ws_bucket((float)x[u], R.lo, R.scale, nb);
            const uint2 a0 = ws_ld_u2_last(D + b, pol), a1 = ws_ld_u2_last(D + b + 1, pol);
            e0[u] = DirEntry{(int32_t)a0.x, a0.y};
            e1[u] = DirEntry{(int32_t)a1.x, a1.y};
        }
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            const uint32_t k32 = (uint32_t)(k[u] >> (KO::BITS - 32));
            lo[u] = min(max(e0[u].idx, 0), c);
            hi[u] = min(max(e1[u].idx, lo[u]), c);
            if (lo[u] == hi[u] || k32 < e0[u].key32) {
                g[u] = lo[u] - 1;   // precedes every start in the bucket: cluster lo - 1
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
#pragma unroll
        for (int u = 0; u < LK; ++u) {
            if (!in[u]) continue;   // past the tile's end: no element (its x = 0 may precede every cluster)
            CEntry<T> ce;
            const int jlo = max(lo[u] - 1, 0), jhi = max(hi[u] - 1, jlo);
            int r = jlo;
            if (jhi == jlo) ce = table[tp + jlo];   // one candidate: no search
            else r = ws_find_cluster<T>(table, tp, jlo, jhi, g[u], k[u], ce);
            if (r < 0 || r >= c) { ws_flag(status, WS_STATUS_INTERNAL); r = 0; ce = table[tp]; }
            const int i = i0 + u * 256;
            __stcs(out + td.vpos + i, ce.val);
            if (ids) __stcs(ids + td.vpos + i, r);
        }
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
                          int64_t* n_clusters, int fp64, const WsEpi& ep, uint32_t* status, uint64_t spin_limit,
                          int n_levels, cudaStream_t st) {
    typedef typename KeyOf<T>::K K;
    if (W.n_lseg == 0) return cudaSuccess;
    K* sorted = nullptr;
    cudaError_t e = ws_large_sort<T>(W, values, status, spin_limit, st, &sorted);
    if (e) return e;
    // tile hulls: the lean kernel, then the general one for the tiles it flagged
    e = ws_large_hull_fast<T>(W, sorted, lambdas, status, st);
    if (e) return e;
    size_t smem = sizeof(TileHullSmem);
    e = cudaFuncSetAttribute(k_tile_hull<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const int small_grid = W.n_hull_tiles < 4 * 152 ? W.n_hull_tiles : 4 * 152;
    WS_LAUNCH(W.prof, WSK_TILE_GENERAL, st,
              (k_tile_hull<T><<<small_grid, HNT, smem, st>>>(sorted, W.hull_tiles, W.lsegs, lambdas, W.rt, W.vp, W.vx,
                                                            W.nvert, W.tile_total, W.gen_list, W.gen_count,
                                                            W.seg_emin, status)));
    // across tiles: junction bridges and the per-segment resolution, then the
    // tree of merges for the segments that need it
    e = ws_large_junctions<T>(W, lambdas, st);
    if (e) return e;
    e = cudaMemsetAsync(W.arrive, 0, sizeof(int32_t) * (size_t)n_levels * W.n_hull_tiles, st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_CLIMB, st,
              (k_climb<T><<<small_grid, HNT, 0, st>>>(W.hull_tiles, W.lsegs, lambdas, W.rt, W.vp, W.vx, W.nvert,
                                                          W.tile_total, W.pieces, W.npieces, W.arrive,
                                                          W.n_hull_tiles, W.seg_mode)));
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
                                                         W.pieces, W.npieces, W.tile_piece, W.table,
                                                         W.dir, gaps, ngaps, gap_cap, fp64, ep, status)));
    WS_LAUNCH(W.prof, WSK_BIG_GAPS, st, (k_big_gaps<<<1024, 256, 0, st>>>(gaps, ngaps, W.dir, gap_cap)));
    WS_LAUNCH(W.prof, WSK_LOOKUP, st,
              (k_lookup<T><<<W.n_sort_tiles, 256, 0, st>>>(values, W.sort_tiles, W.lsegs, W.rt, W.table, W.dir, out,
                                                          ids, status)));
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
                                          const WsEpi&, uint32_t*, uint64_t, int, cudaStream_t);                    \
    template cudaError_t ws_large_copy_sorted<T>(const LargeWork<T>&, const typename KeyOf<T>::K*, T*, cudaStream_t);
WS_INST(float)
WS_INST(double)
