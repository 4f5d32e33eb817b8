// ws_bwd.cu -- the backward of the prox with the partition held fixed: every
// element's gradient is the mean of grad_out over its cluster (the Jacobian
// of the cluster means; a cluster moves as one particle, Sec. 3).
//
// The cluster sums are exact and deterministic: every grad_out value is
// converted to a 128-bit integer at a per-segment scale (exact for values
// within SH binades of the segment's largest |g|: 71 for float, 42 for
// double; smaller ones keep their top bits), and the integers are added with
// 64-bit atomics that carry into the high word explicitly.  Integer addition
// is associative, so the sum -- hence the mean -- does not depend on the
// order of the additions, and its error does not grow with the cluster size
// (one rounding when the mean is formed).
//
// Large segments: per-segment scale and largest id (k_bwd_prep), the used
// cluster slots cleared (k_bwd_zero), the sums, the means (k_bwd_mean), the
// gather (k_bwd_apply).  The sums: the cluster slots are cut into buckets of
// 2^s consecutive slots, small enough for L2; k_bwd_scatter writes every
// element as a pair (slot within its bucket, exact fixed-point code) into its
// bucket's region (the regions sized by k_bwd_prep's bucket counts; each
// tile's pairs are grouped by bucket in shared memory first, so every run is
// copied out whole), and the CTAs of k_bwd_pairs take chunks of pairs in
// order from a counter, so the atomics of the chunks in flight fall into one
// or two buckets' slots and stay in L2 instead of each costing a random DRAM
// read and write.  Lanes of a
// warp with the same slot add once, and a sort tile whose elements all share
// one cluster adds once per CTA (no pairs), so a single huge cluster costs
// one atomic per sort tile.  The pairs and the bucket counters borrow the
// forward's sort buffers, which the backward does not otherwise use.
// One-CTA segments: the same arithmetic in shared memory (k_small_backward).
#include "ws_kernels.cuh"

namespace {

constexpr int BNT = 256;
constexpr int BTILE = WS_SORT_TILE;   // elements per CTA (the sort tiles of the plan)

template <typename T> struct BwdFix;
template <> struct BwdFix<float> { static constexpr int SH = 71, BIAS = 127, MANT = 23; };
template <> struct BwdFix<double> { static constexpr int SH = 42, BIAS = 1023, MANT = 52; };

// g * 2^(SH - emax + BIAS + MANT) as an integer (exact unless g is more than
// SH binades below 2^emax; then truncated toward zero).
template <typename T>
__device__ __forceinline__ i128 ws_bwd_fix(T g, int emax) {
    typedef KeyOf<T> KO;
    const uint64_t b = (uint64_t)KO::bits(g);
    int e = (int)((b >> KO::MANT) & KO::EXPMASK);
    uint64_t m = b & ((1ull << KO::MANT) - 1ull);
    if (e == 0) e = 1; else m |= (1ull << KO::MANT);
    const int sh = e - emax + BwdFix<T>::SH;
    u128 mag;
    if (sh >= 0) mag = (u128)m << sh;
    else mag = (sh > -64) ? (u128)(m >> (-sh)) : (u128)0;
    const bool neg = (b >> (KO::BITS - 1)) & 1ull;
    return neg ? -(i128)mag : (i128)mag;
}

// mean = S / cnt * 2^-(SH - emax + BIAS + MANT)
template <typename T>
__device__ __forceinline__ T ws_bwd_mean(i128 S, int cnt, int emax) {
    const int Lg = BwdFix<T>::SH - emax + BwdFix<T>::BIAS + BwdFix<T>::MANT;
    if (sizeof(T) == 4) return (T)ldexpf(ws_i128_to_float_scaled(S, 0) / (float)cnt, -Lg);
    return (T)ldexp(ws_div_i128_n(S, cnt), -Lg);
}

// A ws_bwd_fix value in one word of the key's width: the significand m
// (MANT + 1 bits, implicit bit included), the shift sh + MANT + 1 in 7 bits
// (sh <= SH, and shifts below -(MANT + 1) give 0, stored as m = 0), the sign
// on top.  Decoding gives back ws_bwd_fix(g, emax) exactly, with no segment
// at hand.
template <typename T>
__device__ __forceinline__ typename KeyOf<T>::K ws_bwd_encode(T g, int emax) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int MB = KO::MANT + 1;
    const uint64_t b = (uint64_t)KO::bits(g);
    int e = (int)((b >> KO::MANT) & KO::EXPMASK);
    uint64_t m = b & ((1ull << KO::MANT) - 1ull);
    if (e == 0) e = 1; else m |= (1ull << KO::MANT);
    int sh = e - emax + BwdFix<T>::SH;
    if (sh < -MB) { m = 0; sh = 0; }
    const uint64_t neg = (b >> (KO::BITS - 1)) & 1ull;
    return (K)((neg << (KO::BITS - 1)) | ((uint64_t)(sh + MB) << MB) | m);
}
template <typename T>
__device__ __forceinline__ i128 ws_bwd_decode(typename KeyOf<T>::K c) {
    typedef KeyOf<T> KO;
    constexpr int MB = KO::MANT + 1;
    const uint64_t w = (uint64_t)c;
    const uint64_t m = w & ((1ull << MB) - 1ull);
    const int sh = (int)((w >> MB) & 127u) - MB;
    const u128 mag = sh >= 0 ? (u128)m << sh : (u128)(m >> (-sh));
    return ((w >> (KO::BITS - 1)) & 1ull) ? -(i128)mag : (i128)mag;
}

constexpr int BK_MAX = 256;   // slot buckets at most
constexpr int BL = 8;         // elements per thread whose loads are issued together (prep, scatter)

__device__ __forceinline__ void ws_atomic_add_i128(unsigned long long* lo_hi, i128 v) {
    const unsigned long long lo = (unsigned long long)(uint64_t)v;
    const unsigned long long hi = (unsigned long long)(uint64_t)((u128)v >> 64);
    const unsigned long long old = atomicAdd(lo_hi, lo);
    atomicAdd(lo_hi + 1, hi + (old + lo < old ? 1ull : 0ull));
}

template <typename T> __device__ __forceinline__ int ws_g_exp(T g) { return g != (T)0 ? ws_eff_exp(g) : 0; }

// Sum of v over the lanes in `peers` (every one of them calls with the same
// mask; the groups of a __match_any_sync may call side by side).  |v| < 2^95
// (a ws_bwd_fix value), so v + 2^95 lies in [0, 2^96): its four 24-bit limbs
// are summed separately -- at most 32 * (2^24 - 1) < 2^29 each, no carry is
// lost -- and recombined.  Exact.
__device__ __forceinline__ i128 ws_group_sum_i96(unsigned peers, i128 v) {
    const u128 o = (u128)(v + ((i128)1 << 95));
    const uint32_t lo = (uint32_t)(uint64_t)o, mid = (uint32_t)(uint64_t)(o >> 32),
                   hi = (uint32_t)(uint64_t)(o >> 64);
    const uint32_t s0 = __reduce_add_sync(peers, lo & 0xffffffu);
    const uint32_t s1 = __reduce_add_sync(peers, (lo >> 24) | ((mid & 0xffffu) << 8));
    const uint32_t s2 = __reduce_add_sync(peers, (mid >> 16) | ((hi & 0xffu) << 16));
    const uint32_t s3 = __reduce_add_sync(peers, hi >> 8);
    const u128 S = (u128)s0 + ((u128)s1 << 24) + ((u128)s2 << 48) + ((u128)s3 << 72);
    return (i128)S - (i128)__popc(peers) * ((i128)1 << 95);
}

// 1. per segment: largest exponent of grad_out and largest cluster id
// and, for the tiles that are not one cluster, the number of elements in
// every slot bucket
template <typename T>
__global__ void __launch_bounds__(BNT) k_bwd_prep(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                  const TileDesc* __restrict__ tiles,
                                                  const LargeSeg* __restrict__ lsegs, int32_t* seg_emax,
                                                  int32_t* seg_maxid, int nb, int s, unsigned long long* bk_cnt,
                                                  uint32_t* status) {
    __shared__ int h[BK_MAX];
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    for (int b = threadIdx.x; b < nb; b += BNT) h[b] = 0;
    __syncthreads();
    const int id0 = ids[td.vpos];
    int e = 0, mx = -1;
    bool bad = false, same = true;
    for (int i0 = threadIdx.x; i0 < td.len; i0 += BNT * BL) {
        int idv[BL];
        T gv[BL];
#pragma unroll
        for (int k = 0; k < BL; ++k) {   // (indices clamped into the tile: every load in bounds)
            const int i = min(i0 + k * BNT, td.len - 1);
            idv[k] = ids[td.vpos + i];
            gv[k] = g[td.vpos + i];
        }
#pragma unroll
        for (int k = 0; k < BL; ++k) {
            if (i0 + k * BNT >= td.len) continue;
            e = max(e, ws_g_exp(gv[k]));
            const int id = idv[k];
            same &= id == id0;
            if (id < 0 || (int64_t)id >= ls.len) bad = true;
            else {
                mx = max(mx, id);
                atomicAdd(&h[(int)((slot0 + id) >> s)], 1);
            }
        }
    }
    if (!__syncthreads_and(same))
        for (int b = threadIdx.x; b < nb; b += BNT)
            if (h[b]) atomicAdd(bk_cnt + b, (unsigned long long)h[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(seg_emax + td.lseg, e);
        atomicMax(seg_maxid + td.lseg, mx);
    }
    if (bad) ws_flag(status, WS_STATUS_INTERNAL);
}

// 2. clear the slots of ids 0 .. max id (tile k of a segment clears slots
// [k BTILE, (k + 1) BTILE): a segment has at most len slots)
__global__ void __launch_bounds__(BNT) k_bwd_zero(const TileDesc* __restrict__ tiles, const LargeSeg* __restrict__ lsegs,
                                                  const int32_t* __restrict__ seg_maxid, unsigned long long* acc,
                                                  int32_t* cnt) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    const int64_t r0 = (int64_t)td.tin * BTILE;
    const int64_t r1 = min(r0 + BTILE, (int64_t)seg_maxid[td.lseg] + 1);
    for (int64_t r = r0 + threadIdx.x; r < r1; r += BNT) {
        acc[2 * (slot0 + r)] = 0ull;
        acc[2 * (slot0 + r) + 1] = 0ull;
        cnt[slot0 + r] = 0;
    }
}

// 3a. bucket regions: exclusive prefix of the counts (one thread; at most
// BK_MAX buckets), the scatter cursors and the pairs pass's chunk counter
__global__ void k_bwd_bscan(const unsigned long long* __restrict__ bk_cnt, int nb, unsigned long long* bk_off,
                            unsigned long long* bk_cur) {
    if (threadIdx.x != 0) return;
    bk_cur[nb] = 0ull;
    unsigned long long run = 0;
    for (int b = 0; b < nb; ++b) {
        bk_off[b] = run;
        bk_cur[b] = run;
        run += bk_cnt[b];
    }
    bk_off[nb] = run;
}

// 3b. a tile that is one cluster adds its exact sum once; every other tile
// writes its elements as (slot within bucket, code) pairs into the bucket
// regions: first into shared memory grouped by bucket, then each bucket's
// run copied out to consecutive addresses (whole sectors, not one 4-byte
// store per scattered element)
template <typename T>
size_t ws_bwd_scatter_smem() { return (size_t)BTILE * (sizeof(int32_t) + sizeof(typename KeyOf<T>::K) + 1); }

template <typename T>
__global__ void __launch_bounds__(BNT) k_bwd_scatter(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                     const TileDesc* __restrict__ tiles,
                                                     const LargeSeg* __restrict__ lsegs,
                                                     const int32_t* __restrict__ seg_emax, unsigned long long* acc,
                                                     int32_t* cnt, int nb, int s, unsigned long long* bk_cur,
                                                     int32_t* pslot, typename KeyOf<T>::K* pcode) {
    typedef typename KeyOf<T>::K K;
    __shared__ long long wlo[BNT / 32], whi[BNT / 32];
    __shared__ int h[BK_MAX], lstart[BK_MAX], wsum[BNT / 32];
    __shared__ unsigned long long base[BK_MAX];
    extern __shared__ __align__(16) unsigned char stage_raw[];
    int32_t* st_slot = reinterpret_cast<int32_t*>(stage_raw);               // [BTILE]
    K* st_code = reinterpret_cast<K*>(stage_raw + sizeof(int32_t) * BTILE);  // [BTILE]
    uint8_t* st_b = stage_raw + (sizeof(int32_t) + sizeof(K)) * BTILE;      // [BTILE] bucket (nb <= 256)
    static_assert(BK_MAX <= BNT && BK_MAX <= 256, "one thread per bucket; buckets fit a byte");
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    const int emax = seg_emax[td.lseg];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    auto valid_id = [&](int id) { return id >= 0 && (int64_t)id < ls.len; };
    for (int b = t; b < nb; b += BNT) h[b] = 0;
    __syncthreads();
    const int id0 = ids[td.vpos];
    bool same = true;
    for (int i0 = t; i0 < td.len; i0 += BNT * BL) {
        int idv[BL];
#pragma unroll
        for (int k = 0; k < BL; ++k) idv[k] = ids[td.vpos + min(i0 + k * BNT, td.len - 1)];
#pragma unroll
        for (int k = 0; k < BL; ++k) {
            if (i0 + k * BNT >= td.len) continue;
            same &= idv[k] == id0;
            if (valid_id(idv[k])) atomicAdd(&h[(int)((slot0 + idv[k]) >> s)], 1);
        }
    }
    if (__syncthreads_and(same)) {
        if (!valid_id(id0)) return;
        i128 sum = 0;
        for (int i0 = t; i0 < td.len; i0 += BNT * BL) {
            T gv[BL];
#pragma unroll
            for (int k = 0; k < BL; ++k) gv[k] = g[td.vpos + min(i0 + k * BNT, td.len - 1)];
#pragma unroll
            for (int k = 0; k < BL; ++k)
                if (i0 + k * BNT < td.len) sum += ws_bwd_fix<T>(gv[k], emax);
        }
        sum = ws_warp_reduce_i128(sum);
        if (lane == 0) { wlo[w] = (long long)(uint64_t)sum; whi[w] = (long long)(uint64_t)((u128)sum >> 64); }
        __syncthreads();
        if (t == 0) {
            i128 tot = 0;
            for (int k = 0; k < BNT / 32; ++k) tot += (i128)(((u128)(uint64_t)whi[k] << 64) | (u128)(uint64_t)wlo[k]);
            ws_atomic_add_i128(acc + 2 * (slot0 + id0), tot);
            atomicAdd(cnt + slot0 + id0, td.len);
        }
        return;
    }
    // each bucket's run in the staging area and its region in the pairs
    const int cb = t < nb ? h[t] : 0;
    int total;
    const int lb = ws_block_excl_scan<BNT, int>(cb, wsum, &total);
    if (t < nb) {
        lstart[t] = lb;
        base[t] = cb ? atomicAdd(bk_cur + t, (unsigned long long)cb) : 0ull;
        h[t] = 0;
    }
    __syncthreads();
    const int64_t low = ((int64_t)1 << s) - 1;
    for (int i0 = t; i0 < td.len; i0 += BNT * BL) {
        int idv[BL];
        T gv[BL];
#pragma unroll
        for (int k = 0; k < BL; ++k) {
            const int i = min(i0 + k * BNT, td.len - 1);
            idv[k] = ids[td.vpos + i];
            gv[k] = g[td.vpos + i];
        }
#pragma unroll
        for (int k = 0; k < BL; ++k) {
            if (i0 + k * BNT >= td.len || !valid_id(idv[k])) continue;
            const int64_t slot = slot0 + idv[k];
            const int b = (int)(slot >> s);
            const int lp = lstart[b] + atomicAdd(&h[b], 1);
            st_slot[lp] = (int32_t)(slot & low);
            st_code[lp] = ws_bwd_encode<T>(gv[k], emax);
            st_b[lp] = (uint8_t)b;
        }
    }
    __syncthreads();
    for (int j = t; j < total; j += BNT) {
        const int b = st_b[j];
        const unsigned long long pos = base[b] + (unsigned long long)(j - lstart[b]);
        pslot[pos] = st_slot[j];
        pcode[pos] = st_code[j];
    }
}

// 3c. the pairs, bucket by bucket: the CTAs of a persistent grid take chunks
// in order from a counter (not a fixed stride, which lets CTAs drift apart),
// so the slots that the chunks in flight add into span about one bucket
constexpr int BPER = 8;   // pairs per thread and step

template <typename T>
__global__ void __launch_bounds__(BNT) k_bwd_pairs(const int32_t* __restrict__ pslot,
                                                   const typename KeyOf<T>::K* __restrict__ pcode,
                                                   const unsigned long long* __restrict__ bk_off, int nb, int s,
                                                   unsigned long long* chunk_ctr, unsigned long long* acc,
                                                   int32_t* cnt) {
    typedef typename KeyOf<T>::K K;
    __shared__ unsigned long long off[BK_MAX + 1];
    __shared__ unsigned long long s_c0;
    for (int b = threadIdx.x; b <= nb; b += BNT) off[b] = bk_off[b];
    __syncthreads();
    const unsigned long long total = off[nb];
    const int lane = threadIdx.x & 31;
    constexpr unsigned long long CH = (unsigned long long)BNT * BPER;
    int b = 0;   // bucket of this thread's current pair (pairs only move forward)
    while (true) {
        __syncthreads();   // every thread has read the previous chunk's start
        if (threadIdx.x == 0) s_c0 = atomicAdd(chunk_ctr, 1ull) * CH;
        __syncthreads();
        const unsigned long long c0 = s_c0;
        if (c0 >= total) break;
        int32_t sl[BPER];
        K cd[BPER];
#pragma unroll
        for (int k = 0; k < BPER; ++k) {
            const unsigned long long j = c0 + (unsigned long long)k * BNT + threadIdx.x;
            sl[k] = j < total ? pslot[j] : 0;
            cd[k] = j < total ? pcode[j] : (K)0;
        }
#pragma unroll
        for (int k = 0; k < BPER; ++k) {
            const unsigned long long j = c0 + (unsigned long long)k * BNT + threadIdx.x;
            const bool in = j < total;
            long long slot = -1 - lane;   // distinct for lanes past the end
            i128 v = 0;
            if (in) {
                while (b + 1 < nb && off[b + 1] <= j) ++b;
                slot = ((long long)b << s) | (long long)sl[k];
                v = ws_bwd_decode<T>(cd[k]);
            }
            const unsigned peers = __match_any_sync(0xffffffffu, (unsigned long long)slot);
            const i128 sum = __any_sync(0xffffffffu, __popc(peers) > 1) ? ws_group_sum_i96(peers, v) : v;
            if (in && lane == __ffs((int)peers) - 1) {
                ws_atomic_add_i128(acc + 2 * slot, sum);
                atomicAdd(cnt + slot, __popc(peers));
            }
        }
    }
}

// 4. cluster means (slots 0 .. max id of each segment)
template <typename T>
__global__ void __launch_bounds__(BNT) k_bwd_mean(const TileDesc* __restrict__ tiles, const LargeSeg* __restrict__ lsegs,
                                                  const int32_t* __restrict__ seg_maxid,
                                                  const int32_t* __restrict__ seg_emax,
                                                  const unsigned long long* __restrict__ acc,
                                                  const int32_t* __restrict__ cnt, T* mean) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    const int64_t r0 = (int64_t)td.tin * BTILE;
    const int64_t r1 = min(r0 + BTILE, (int64_t)seg_maxid[td.lseg] + 1);
    const int emax = seg_emax[td.lseg];
    for (int64_t r = r0 + threadIdx.x; r < r1; r += BNT) {
        const int c = cnt[slot0 + r];
        if (c == 0) continue;
        const i128 S = (i128)(((u128)acc[2 * (slot0 + r) + 1] << 64) | (u128)acc[2 * (slot0 + r)]);
        mean[slot0 + r] = ws_bwd_mean<T>(S, c, emax);
    }
}

// 5. every element takes its cluster's mean
template <typename T>
__global__ void __launch_bounds__(BNT) k_bwd_apply(const int32_t* __restrict__ ids, const TileDesc* __restrict__ tiles,
                                                   const LargeSeg* __restrict__ lsegs, const T* __restrict__ mean,
                                                   T* gin) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    for (int i = threadIdx.x; i < td.len; i += BNT) {
        const int id = ids[td.vpos + i];
        if (id < 0 || (int64_t)id >= ls.len) continue;
        gin[td.vpos + i] = mean[slot0 + id];
    }
}

// One-CTA segments: the same exact sums in shared memory.  Every thread keeps
// its CAP / NT elements (grad_out and id) in registers; lanes of a warp with
// the same cluster add once; each used slot forms its mean once, in place.
template <typename T, int NT, int CAP>
__global__ void __launch_bounds__(NT) k_small_backward(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                       const int64_t* __restrict__ offsets,
                                                       const int32_t* __restrict__ seg_list, T* gin,
                                                       uint32_t* status) {
    constexpr int PER = CAP / NT;
    static_assert(CAP % NT == 0, "whole elements per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long* acc = reinterpret_cast<unsigned long long*>(smem_raw);   // [CAP][2]
    int* cnt = reinterpret_cast<int*>(acc + 2 * CAP);                            // [CAP]
    __shared__ int s_emax;
    const int seg = seg_list[blockIdx.x];
    const int64_t a0 = offsets[seg];
    const int n = (int)(offsets[seg + 1] - a0);
    if (n <= 0) return;
    if (n > CAP) { if (threadIdx.x == 0) ws_flag(status, WS_STATUS_INTERNAL); return; }
    const int t = threadIdx.x, lane = t & 31;
    if (t == 0) s_emax = 0;
    T gv[PER];
    int idv[PER];
    int e = 0;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = t + k * NT;
        gv[k] = (T)0;
        idv[k] = -1;
        if (i < n) {
            gv[k] = g[a0 + i];
            const int id = ids[a0 + i];
            if (id >= 0 && id < n) idv[k] = id; else bad = true;
            acc[2 * i] = 0ull;
            acc[2 * i + 1] = 0ull;
            cnt[i] = 0;
        }
        e = max(e, ws_g_exp(gv[k]));
    }
    if (bad) ws_flag(status, WS_STATUS_INTERNAL);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    __syncthreads();
    if (lane == 0) atomicMax(&s_emax, e);
    __syncthreads();
    const int emax = s_emax;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int id = idv[k];
        const i128 q = ws_bwd_fix<T>(gv[k], emax);
        const unsigned peers = __match_any_sync(0xffffffffu, id);
        const i128 s = __any_sync(0xffffffffu, __popc(peers) > 1) ? ws_group_sum_i96(peers, q) : q;
        if (id >= 0 && lane == __ffs((int)peers) - 1) {
            ws_atomic_add_i128(acc + 2 * id, s);
            atomicAdd(cnt + id, __popc(peers));
        }
    }
    __syncthreads();
    // the mean of slot r replaces its low word (only this thread touches slot r)
    for (int r = t; r < n; r += NT) {
        const int c = cnt[r];
        if (c == 0) continue;
        const i128 S = (i128)(((u128)acc[2 * r + 1] << 64) | (u128)acc[2 * r]);
        *reinterpret_cast<T*>(acc + 2 * r) = ws_bwd_mean<T>(S, c, emax);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int i = t + k * NT;
        if (i < n && idv[k] >= 0) gin[a0 + i] = *reinterpret_cast<const T*>(acc + 2 * idv[k]);
    }
}

}  // namespace

template <typename T>
cudaError_t ws_large_backward(const LargeWork<T>& W, const T* g, const int32_t* ids, T* gin, uint32_t* status,
                              cudaStream_t st) {
    if (W.n_lseg == 0) return cudaSuccess;
    // seg_emax / seg_maxid live in the backward's per-segment words
    int32_t* seg_emax = W.bwd_seg;
    int32_t* seg_maxid = W.bwd_seg + W.n_lseg;
    cudaError_t e = cudaMemsetAsync(seg_emax, 0, sizeof(int32_t) * W.n_lseg, st);
    if (e) return e;
    e = cudaMemsetAsync(seg_maxid, 0xff, sizeof(int32_t) * W.n_lseg, st);
    if (e) return e;
    const int nt = W.n_sort_tiles;
    // slot buckets of 2^s slots (2^21 slots of 20 bytes: about 40 MB, well
    // inside L2); their counters live in the sort histogram buffer, which
    // holds at least 3 nb + 2 words for the nb allowed here
    typedef typename KeyOf<T>::K K;
    constexpr int P = KeyOf<T>::BITS / 8;
    const int64_t total_slots = W.n_keys + W.n_lseg;
    const int64_t words = (int64_t)sizeof(uint32_t) * W.n_lseg * P * 256 / sizeof(unsigned long long);
    const int nb_max = (int)std::min<int64_t>(BK_MAX, (words - 2) / 3);
    int s = 21;
    while (((total_slots + ((int64_t)1 << s) - 1) >> s) > nb_max) ++s;
    const int nb = (int)((total_slots + ((int64_t)1 << s) - 1) >> s);
    unsigned long long* bk_cnt = reinterpret_cast<unsigned long long*>(W.hist);
    unsigned long long* bk_off = bk_cnt + nb;
    unsigned long long* bk_cur = bk_off + nb + 1;   // nb cursors, then the chunk counter
    // the pairs borrow the sort's key buffers (n_keys entries each)
    int32_t* pslot = reinterpret_cast<int32_t*>(W.keys_a);
    K* pcode = W.keys_b;
    e = cudaMemsetAsync(bk_cnt, 0, sizeof(unsigned long long) * nb, st);
    if (e) return e;
    static const int pairs_grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bwd_pairs<T>, BNT, 0) != cudaSuccess) {
            cudaGetLastError();
            return 4 * 152;
        }
        return std::max(1, sms * std::max(per_sm, 1));
    }();
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_prep<T><<<nt, BNT, 0, st>>>(g, ids, W.sort_tiles, W.lsegs, seg_emax, seg_maxid, nb, s, bk_cnt,
                                                 status)));
    WS_LAUNCH(W.prof, WSK_BWD, st, (k_bwd_zero<<<nt, BNT, 0, st>>>(W.sort_tiles, W.lsegs, seg_maxid, W.bacc, W.bcnt)));
    WS_LAUNCH(W.prof, WSK_BWD, st, (k_bwd_bscan<<<1, 32, 0, st>>>(bk_cnt, nb, bk_off, bk_cur)));
    const size_t scatter_smem = ws_bwd_scatter_smem<T>();
    e = cudaFuncSetAttribute(k_bwd_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)scatter_smem);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_scatter<T><<<nt, BNT, scatter_smem, st>>>(g, ids, W.sort_tiles, W.lsegs, seg_emax, W.bacc, W.bcnt, nb, s,
                                                    bk_cur, pslot, pcode)));
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_pairs<T><<<pairs_grid, BNT, 0, st>>>(pslot, pcode, bk_off, nb, s, bk_cur + nb, W.bacc,
                                                          W.bcnt)));
    WS_LAUNCH(W.prof, WSK_BWD, st,
              (k_bwd_mean<T><<<nt, BNT, 0, st>>>(W.sort_tiles, W.lsegs, seg_maxid, seg_emax, W.bacc, W.bcnt,
                                                 W.bsum)));
    WS_LAUNCH(W.prof, WSK_BWD, st, (k_bwd_apply<T><<<nt, BNT, 0, st>>>(ids, W.sort_tiles, W.lsegs, W.bsum, gin)));
    return cudaGetLastError();
}

template <typename T>
cudaError_t ws_launch_small_backward(const T* g, const int32_t* ids, const int64_t* offsets, const int32_t* seg_list,
                                     int n_list, T* gin, uint32_t* status, cudaStream_t st, WsProf* prof) {
    constexpr int NT = 256;
    constexpr int CAP = SmallCfg<T>::CAP;
    if (n_list <= 0) return cudaSuccess;
    const size_t smem = (size_t)CAP * (2 * sizeof(unsigned long long) + sizeof(int));
    auto k = k_small_backward<T, NT, CAP>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    WS_LAUNCH(prof, WSK_BWD, st, (k<<<n_list, NT, smem, st>>>(g, ids, offsets, seg_list, gin, status)));
    return cudaGetLastError();
}

template cudaError_t ws_large_backward<float>(const LargeWork<float>&, const float*, const int32_t*, float*,
                                              uint32_t*, cudaStream_t);
template cudaError_t ws_large_backward<double>(const LargeWork<double>&, const double*, const int32_t*, double*,
                                               uint32_t*, cudaStream_t);
template cudaError_t ws_launch_small_backward<float>(const float*, const int32_t*, const int64_t*, const int32_t*,
                                                     int, float*, uint32_t*, cudaStream_t, WsProf*);
template cudaError_t ws_launch_small_backward<double>(const double*, const int32_t*, const int64_t*,
                                                      const int32_t*, int, double*, uint32_t*, cudaStream_t,
                                                      WsProf*);
