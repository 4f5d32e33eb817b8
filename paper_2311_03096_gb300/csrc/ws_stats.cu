// ws_stats.cu -- R(w) and the weight-sharing measure of a vector, on the
// sorted keys of the device-wide path.
//
// R(w) = 1/(d-1) sum_{i>j} |w_i - w_j| (Eq. (1)) is evaluated the way the
// appendix "Computing R" does it: sort, then R = 1/(d-1) sum_k (2k - d - 1) x_k
// (k = 1..d, x sorted ascending), an O(d) reduction after the sort.  The sum
// is accumulated exactly in 128-bit fixed point (q = x 2^L as in the hull:
// |q| <= 2^58, |2k - d - 1| < 2^31, so every term and the total fit) and
// rounded once at the end.  The weight-sharing measure of the CIFAR10
// experiment is #distinct nonzero weights / #nonzero weights (0 when every
// weight is zero); on sorted keys a distinct value is a key that differs
// from its predecessor.
#include "ws_kernels.cuh"

namespace {

struct RPartial {
    i128 s;             // sum of (2k - d - 1) q_k over the tile
    long long distinct; // nonzero keys that differ from their predecessor
    long long nonzero;
};

template <typename T>
__global__ void __launch_bounds__(256) k_R_tiles(const typename KeyOf<T>::K* __restrict__ sorted,
                                                 const TileDesc* __restrict__ tiles,
                                                 const LargeSeg* __restrict__ lsegs,
                                                 const int32_t* __restrict__ seg_emin, RPartial* part) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    __shared__ i128 ws128[8];
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const K* seg = sorted + ls.kpos;
    const T xlo = KO::from_key(seg[0]), xhi = KO::from_key(seg[ls.len - 1]);
    const int E = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[td.lseg]);
    const K kz = KO::to_key((T)0), knz = KO::to_key(-(T)0);
    const int64_t j0 = (int64_t)td.tin * WS_SORT_TILE;
    i128 acc = 0;
    long long dis = 0, nz = 0;
    for (int i = threadIdx.x; i < td.len; i += 256) {
        const int64_t j = j0 + i;
        const K k = seg[j];
        const bool nonzero = k != kz && k != knz;
        nz += nonzero;
        dis += nonzero && (j == 0 || seg[j - 1] != k);
        const int64_t coef = 2 * j - ls.len + 1;   // 2k - d - 1 with k = j + 1
        acc += (i128)coef * (i128)ws_fixed<T>(KO::from_key(k), E);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long packed[2] = {dis, nz};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += (i128)__shfl_xor_sync(0xffffffffu, (long long)(acc >> 64), o) * ((i128)1 << 64) +
               (i128)(unsigned long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)acc, o);
        packed[0] += __shfl_xor_sync(0xffffffffu, packed[0], o);
        packed[1] += __shfl_xor_sync(0xffffffffu, packed[1], o);
    }
    __shared__ long long wsd[8], wsn[8];
    if (lane == 0) { ws128[w] = acc; wsd[w] = packed[0]; wsn[w] = packed[1]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        RPartial p;
        p.s = 0; p.distinct = 0; p.nonzero = 0;
        for (int k = 0; k < 8; ++k) { p.s += ws128[k]; p.distinct += wsd[k]; p.nonzero += wsn[k]; }
        part[blockIdx.x] = p;
    }
}

template <typename T>
__global__ void __launch_bounds__(32) k_R_final(const LargeSeg* __restrict__ lsegs, const TileDesc* __restrict__ tiles,
                                                const typename KeyOf<T>::K* __restrict__ sorted,
                                                const int32_t* __restrict__ seg_emin, const RPartial* part,
                                                double* R_out, double* metric_out, uint32_t* status) {
    typedef KeyOf<T> KO;
    if (threadIdx.x != 0) return;
    const LargeSeg ls = lsegs[blockIdx.x];
    i128 s = 0;
    long long dis = 0, nz = 0;
    for (int t = 0; t < ls.sort_count; ++t) {
        const RPartial p = part[ls.sort_first + t];
        s += p.s; dis += p.distinct; nz += p.nonzero;
    }
    const T xlo = KO::from_key(sorted[ls.kpos]), xhi = KO::from_key(sorted[ls.kpos + ls.len - 1]);
    const int E = ws_fix_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[blockIdx.x]);
    ws_note_scale<T>(max(ws_eff_exp(xlo), ws_eff_exp(xhi)), seg_emin[blockIdx.x], status);
    const int L = KO::L_BASE - E;
    if (R_out) R_out[ls.seg] = ls.len > 1 ? ldexp(ws_i128_to_double(s), -L) / (double)(ls.len - 1) : 0.0;
    if (metric_out) metric_out[ls.seg] = nz > 0 ? (double)dis / (double)nz : 0.0;
}

}  // namespace

template <typename T>
cudaError_t ws_large_R(const LargeWork<T>& W, const T* values, double* R_out, double* metric_out, uint32_t* status,
                       uint64_t spin_limit, void* partial, cudaStream_t st) {
    typedef typename KeyOf<T>::K K;
    if (W.n_lseg == 0) return cudaSuccess;
    K* sorted = nullptr;
    cudaError_t e = ws_large_sort<T>(W, values, status, spin_limit, st, &sorted);
    if (e) return e;
    RPartial* part = reinterpret_cast<RPartial*>(partial);
    WS_LAUNCH(W.prof, WSK_MISC, st,
              (k_R_tiles<T><<<W.n_sort_tiles, 256, 0, st>>>(sorted, W.sort_tiles, W.lsegs, W.seg_emin, part)));
    WS_LAUNCH(W.prof, WSK_MISC, st,
              (k_R_final<T><<<W.n_lseg, 32, 0, st>>>(W.lsegs, W.sort_tiles, sorted, W.seg_emin, part, R_out,
                                                     metric_out, status)));
    return cudaGetLastError();
}

namespace {
template <typename T>
__global__ void k_R_tiny(const T* values, int64_t d, double* R_out, double* metric_out) {
    if (R_out) *R_out = 0.0;   // d <= 1: no pairs
    if (metric_out) *metric_out = (d == 1 && values[0] != (T)0) ? 1.0 : 0.0;
}
}  // namespace

template <typename T>
cudaError_t ws_tiny_R(const T* values, int64_t d, double* R_out, double* metric_out, WsProf* prof, cudaStream_t st) {
    WS_LAUNCH(prof, WSK_MISC, st, (k_R_tiny<T><<<1, 1, 0, st>>>(values, d, R_out, metric_out)));
    return cudaGetLastError();
}
template cudaError_t ws_tiny_R<float>(const float*, int64_t, double*, double*, WsProf*, cudaStream_t);
template cudaError_t ws_tiny_R<double>(const double*, int64_t, double*, double*, WsProf*, cudaStream_t);

size_t ws_R_partial_bytes(int n_sort_tiles) { return sizeof(RPartial) * (size_t)(n_sort_tiles > 0 ? n_sort_tiles : 1); }

template cudaError_t ws_large_R<float>(const LargeWork<float>&, const float*, double*, double*, uint32_t*, uint64_t,
                                       void*, cudaStream_t);
template cudaError_t ws_large_R<double>(const LargeWork<double>&, const double*, double*, double*, uint32_t*,
                                        uint64_t, void*, cudaStream_t);

// ---------------------------------------------------------------------------
// d out / d lambda with the partition held fixed (Sec. 3: a cluster moves
// with the mean velocity of its particles).  A cluster on sorted positions
// a..b (1-based) has d out / d lambda = (d + 1 - a - b)/(d - 1); with 0-based
// start s and size m that is (d - 2s - m)/(d - 1).  Starts follow from the
// cluster sizes because cluster ids are ranked by value.  The result per
// segment is sum_i grad_out[i] * d out_i / d lambda (FP64, atomics: the
// summation order is not fixed).
// ---------------------------------------------------------------------------
namespace {

template <typename T, int NT, int CAP>
__global__ void __launch_bounds__(NT) k_dlam_small(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                   const int64_t* __restrict__ offsets,
                                                   const int32_t* __restrict__ seg_list, double* out,
                                                   uint32_t* status) {
    __shared__ int cnt[CAP];
    __shared__ int start[CAP];
    __shared__ int wsum[NT / 32];
    __shared__ double wacc[NT / 32];
    constexpr int PER = CAP / NT;
    const int seg = seg_list[blockIdx.x];
    const int64_t a0 = offsets[seg];
    const int n = (int)(offsets[seg + 1] - a0);
    if (n <= 1) return;   // d <= 1: no shift
    if (n > CAP) { if (threadIdx.x == 0) ws_flag(status, WS_STATUS_INTERNAL); return; }
    const int t = threadIdx.x;
    for (int i = t; i < CAP; i += NT) cnt[i] = 0;
    __syncthreads();
    for (int i = t; i < n; i += NT) {
        const int id = ids[a0 + i];
        if (id < 0 || id >= n) { ws_flag(status, WS_STATUS_INTERNAL); continue; }
        atomicAdd(&cnt[id], 1);
    }
    __syncthreads();
    int run = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) run += cnt[t * PER + k];
    int tot;
    int ex = ws_block_excl_scan<NT, int>(run, wsum, &tot);
#pragma unroll
    for (int k = 0; k < PER; ++k) { start[t * PER + k] = ex; ex += cnt[t * PER + k]; }
    __syncthreads();
    double acc = 0.0;
    for (int i = t; i < n; i += NT) {
        const int id = ids[a0 + i];
        if (id < 0 || id >= n) continue;
        acc += (double)g[a0 + i] * (double)(n - 2 * start[id] - cnt[id]) / (double)(n - 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) wacc[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int w = 0; w < NT / 32; ++w) s += wacc[w];
        atomicAdd(&out[seg], s);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dlam_count(const int32_t* __restrict__ ids, const TileDesc* __restrict__ tiles,
                                                    const LargeSeg* __restrict__ lsegs, int32_t* cnt,
                                                    uint32_t* status) {
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    for (int i = threadIdx.x; i < td.len; i += 256) {
        const int id = ids[td.vpos + i];
        if (id < 0 || id >= ls.len) { ws_flag(status, WS_STATUS_INTERNAL); continue; }
        atomicAdd(&cnt[slot0 + id], 1);
    }
}

// exclusive scan of cnt[0..S) in chunks of 4096: pos = chunk-local prefix,
// csum[b] = total of chunk b
constexpr int DL_CHUNK = 4096;
__global__ void __launch_bounds__(256) k_dlam_scan_chunks(const int32_t* __restrict__ cnt, int64_t S, int32_t* pos,
                                                          int32_t* csum) {
    __shared__ int wsum[8];
    const int64_t b0 = (int64_t)blockIdx.x * DL_CHUNK;
    const int t = threadIdx.x;
    constexpr int PER = DL_CHUNK / 256;
    int v[PER];
    int run = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int64_t s = b0 + t * PER + k;
        v[k] = s < S ? cnt[s] : 0;
        run += v[k];
    }
    int tot;
    int ex = ws_block_excl_scan<256, int>(run, wsum, &tot);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int64_t s = b0 + t * PER + k;
        if (s < S) pos[s] = ex;
        ex += v[k];
    }
    if (t == 0) csum[blockIdx.x] = tot;
}

// exclusive scan of the chunk totals, in place (one CTA, carried across rounds)
__global__ void __launch_bounds__(1024) k_dlam_scan_totals(int32_t* csum, int nb) {
    __shared__ int wsum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        const int b = b0 + (int)threadIdx.x;
        const int v = b < nb ? csum[b] : 0;
        int tot;
        const int ex = ws_block_excl_scan<1024, int>(v, wsum, &tot);
        if (b < nb) csum[b] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_dlam_apply(const T* __restrict__ g, const int32_t* __restrict__ ids,
                                                    const TileDesc* __restrict__ tiles,
                                                    const LargeSeg* __restrict__ lsegs,
                                                    const int32_t* __restrict__ cnt, const int32_t* __restrict__ pos,
                                                    const int32_t* __restrict__ csum, double* out) {
    __shared__ double wacc[8];
    const TileDesc td = tiles[blockIdx.x];
    const LargeSeg ls = lsegs[td.lseg];
    const int64_t slot0 = ls.kpos + td.lseg;
    const int64_t base = (int64_t)pos[slot0] + csum[slot0 / DL_CHUNK];
    const double inv = 1.0 / (double)(ls.len - 1);
    double acc = 0.0;
    for (int i = threadIdx.x; i < td.len; i += 256) {
        const int id = ids[td.vpos + i];
        if (id < 0 || id >= ls.len) continue;
        const int64_t s = slot0 + id;
        const int64_t start = (int64_t)pos[s] + csum[s / DL_CHUNK] - base;
        acc += (double)g[td.vpos + i] * (double)(ls.len - 2 * start - cnt[s]) * inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) wacc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += wacc[w];
        atomicAdd(&out[ls.seg], s);
    }
}

}  // namespace

template <typename T>
cudaError_t ws_dlambda(const T* g, const int32_t* ids, const int64_t* d_offsets, const int32_t* d_small, int n_small,
                       int64_t n_seg, const LargeWork<T>& W, double* out, uint32_t* status, void* partial,
                       cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)n_seg, st);
    if (e) return e;
    if (n_small > 0) {
        WS_LAUNCH(W.prof, WSK_BWD, st,
                  (k_dlam_small<T, 256, SmallCfg<T>::CAP><<<n_small, 256, 0, st>>>(g, ids, d_offsets, d_small, out,
                                                                                   status)));
    }
    if (W.n_lseg > 0) {
        const int64_t S = W.n_keys + W.n_lseg;
        int32_t* cnt = W.bcnt;
        int32_t* pos = reinterpret_cast<int32_t*>(W.bsum);
        int32_t* csum = reinterpret_cast<int32_t*>(partial);
        const int nb = (int)((S + DL_CHUNK - 1) / DL_CHUNK);
        e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)S, st);
        if (e) return e;
        WS_LAUNCH(W.prof, WSK_BWD, st,
                  (k_dlam_count<T><<<W.n_sort_tiles, 256, 0, st>>>(ids, W.sort_tiles, W.lsegs, cnt, status)));
        WS_LAUNCH(W.prof, WSK_BWD, st, (k_dlam_scan_chunks<<<nb, 256, 0, st>>>(cnt, S, pos, csum)));
        WS_LAUNCH(W.prof, WSK_BWD, st, (k_dlam_scan_totals<<<1, 1024, 0, st>>>(csum, nb)));
        WS_LAUNCH(W.prof, WSK_BWD, st,
                  (k_dlam_apply<T><<<W.n_sort_tiles, 256, 0, st>>>(g, ids, W.sort_tiles, W.lsegs, cnt, pos, csum,
                                                                   out)));
    }
    return cudaGetLastError();
}

template cudaError_t ws_dlambda<float>(const float*, const int32_t*, const int64_t*, const int32_t*, int, int64_t,
                                       const LargeWork<float>&, double*, uint32_t*, void*, cudaStream_t);
template cudaError_t ws_dlambda<double>(const double*, const int32_t*, const int64_t*, const int32_t*, int, int64_t,
                                        const LargeWork<double>&, double*, uint32_t*, void*, cudaStream_t);
