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
                                                double* R_out, double* metric_out) {
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
                                                     metric_out)));
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
