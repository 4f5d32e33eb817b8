// ws_sort.cu -- segmented LSD radix sort of the keys of the large segments
// (the pre-processing every prox algorithm of Sec. 4 assumes).
//
// Only keys move: because equal weights always share a cluster, the result of
// the prox never depends on the order of ties, so no index payload is sorted
// and no unpermute scatter is needed later (the values are recovered by a
// key -> cluster lookup in the caller's order).
//
// One histogram pass computes every digit histogram of every large segment;
// then each 8-bit digit pass is a single "onesweep" kernel: a CTA ranks its
// 8192 keys by digit in shared memory, publishes its per-digit counts, gets
// the counts of the earlier tiles of the same segment through a decoupled
// look-back (bounded waits), and writes its keys as per-digit contiguous runs.
#include "ws_kernels.cuh"

namespace {

constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_CNT = (1ull << 62) - 1ull;

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

template <typename T>
__global__ void __launch_bounds__(WS_SORT_NT) k_hist(const T* __restrict__ values, const TileDesc* __restrict__ tiles,
                                                     uint32_t* hist, uint32_t* status) {
    typedef KeyOf<T> KO;
    constexpr int P = KO::BITS / 8;
    __shared__ uint32_t h[P * 256];
    for (int i = threadIdx.x; i < P * 256; i += WS_SORT_NT) h[i] = 0;
    __syncthreads();
    const TileDesc td = tiles[blockIdx.x];
    bool bad = false;
    for (int i = threadIdx.x; i < td.len; i += WS_SORT_NT) {
        T v = values[td.vpos + i];
        bad |= !ws_isfinite(v);
        typename KO::K k = KO::to_key(v);
#pragma unroll
        for (int p = 0; p < P; ++p) atomicAdd(&h[p * 256 + (int)((k >> (8 * p)) & 0xff)], 1u);
    }
    if (bad) ws_flag(status, WS_STATUS_NONFINITE);
    __syncthreads();
    uint32_t* gh = hist + (size_t)td.lseg * P * 256;
    for (int i = threadIdx.x; i < P * 256; i += WS_SORT_NT)
        if (h[i]) atomicAdd(&gh[i], h[i]);
}

// exclusive scan of every (segment, pass) histogram, in place
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t* hist) {
    __shared__ uint32_t ws[8];
    uint32_t* h = hist + (size_t)blockIdx.x * 256;
    uint32_t v = h[threadIdx.x];
    uint32_t tot;
    uint32_t ex = ws_block_excl_scan<256, int>((int)v, (int*)ws, (int*)&tot);
    h[threadIdx.x] = ex;
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(WS_SORT_NT) k_onesweep(const T* __restrict__ values,
                                                         const typename KeyOf<T>::K* __restrict__ keys_in,
                                                         typename KeyOf<T>::K* __restrict__ keys_out,
                                                         const TileDesc* __restrict__ tiles,
                                                         const LargeSeg* __restrict__ lsegs,
                                                         const uint32_t* __restrict__ hist, uint64_t* lookback,
                                                         uint32_t* counter, int pass, uint32_t* status,
                                                         uint64_t spin_limit) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int P = KO::BITS / 8;
    constexpr int NT = WS_SORT_NT, ITEMS = WS_SORT_ITEMS, TILE = WS_SORT_TILE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* skeys = reinterpret_cast<K*>(smem_raw);
    uint32_t* whist = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * TILE);
    uint32_t* dcount = whist + (NT / 32) * 256;
    uint32_t* dstart = dcount + 256;
    uint32_t* excl = dstart + 256;
    __shared__ int s_tile;
    __shared__ int s_timeout;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) { s_tile = (int)atomicAdd(counter, 1u); s_timeout = 0; }
    __syncthreads();
    const int tile = s_tile;
    const TileDesc td = tiles[tile];
    const int64_t seg_k = lsegs[td.lseg].kpos;
    const uint32_t* dbase = hist + ((size_t)td.lseg * P + pass) * 256;

    K key[ITEMS];
    uint32_t dg[ITEMS];
    bool valid[ITEMS];
    int pos[ITEMS];
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        int p = w * 32 * ITEMS + k * 32 + lane;
        valid[k] = p < td.len;
        if (FIRST) key[k] = valid[k] ? KO::to_key(values[td.vpos + p]) : (K)0;
        else key[k] = valid[k] ? keys_in[td.kpos + p] : (K)0;
        dg[k] = (uint32_t)((key[k] >> (8 * pass)) & 0xff);
    }
    ws_rank_digits<NT, ITEMS>(dg, valid, pos, whist, dcount, dstart, nullptr);

    // publish this tile's per-digit counts, then look back over earlier tiles
    uint64_t* my_lb = lookback + (size_t)tile * 256;
    if (t < 256) {
        uint64_t c = dcount[t];
        if (td.tin == 0) {
            st_relaxed_u64(&my_lb[t], LB_INC | c);
            excl[t] = 0;
        } else {
            st_relaxed_u64(&my_lb[t], LB_AGG | c);
            uint64_t run = 0;
            int j = tile - 1;
            uint64_t it = 0;
            while (true) {
                uint64_t v = ld_relaxed_u64(&lookback[(size_t)j * 256 + t]);
                uint64_t f = v & ~LB_CNT;
                if (f == 0) {
                    if (++it > spin_limit) { s_timeout = 1; break; }
                    ws_backoff((int)min(it, (uint64_t)1 << 20));
                    continue;
                }
                run += v & LB_CNT;
                if (f == LB_INC || j <= td.first) break;
                --j;
            }
            excl[t] = (uint32_t)run;
            st_relaxed_u64(&my_lb[t], LB_INC | (run + c));
        }
    }
    // stage the tile in digit order
#pragma unroll
    for (int k = 0; k < ITEMS; ++k)
        if (valid[k]) skeys[pos[k]] = key[k];
    __syncthreads();
    if (t == 0 && s_timeout) ws_flag(status, WS_STATUS_TIMEOUT);
    for (int j = t; j < td.len; j += NT) {
        K kk = skeys[j];
        uint32_t d = (uint32_t)((kk >> (8 * pass)) & 0xff);
        int64_t dst = seg_k + (int64_t)dbase[d] + (int64_t)excl[d] + (int64_t)(j - (int)dstart[d]);
        keys_out[dst] = kk;
    }
}

}  // namespace

template <typename T>
size_t ws_onesweep_smem() {
    typedef typename KeyOf<T>::K K;
    return sizeof(K) * WS_SORT_TILE + sizeof(uint32_t) * ((WS_SORT_NT / 32) * 256 + 3 * 256);
}

template <typename T>
cudaError_t ws_large_sort(const LargeWork<T>& W, const T* values, uint32_t* status, uint64_t spin_limit,
                          cudaStream_t st, typename KeyOf<T>::K** sorted) {
    typedef typename KeyOf<T>::K K;
    constexpr int P = KeyOf<T>::BITS / 8;
    cudaError_t e;
    *sorted = nullptr;
    if (W.n_sort_tiles == 0) return cudaSuccess;
    e = cudaMemsetAsync(W.hist, 0, sizeof(uint32_t) * (size_t)W.n_lseg * P * 256, st);
    if (e) return e;
    e = cudaMemsetAsync(W.lookback, 0, sizeof(uint64_t) * (size_t)P * W.n_sort_tiles * 256, st);
    if (e) return e;
    e = cudaMemsetAsync(W.tile_counter, 0, sizeof(uint32_t) * P, st);
    if (e) return e;
    WS_LAUNCH(W.prof, WSK_HIST, st, (k_hist<T><<<W.n_sort_tiles, WS_SORT_NT, 0, st>>>(values, W.sort_tiles, W.hist, status)));
    WS_LAUNCH(W.prof, WSK_HIST_SCAN, st, (k_hist_scan<<<W.n_lseg * P, 256, 0, st>>>(W.hist)));
    size_t smem = ws_onesweep_smem<T>();
    e = cudaFuncSetAttribute(k_onesweep<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    e = cudaFuncSetAttribute(k_onesweep<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    K* src = W.keys_b;
    K* dst = W.keys_a;
    for (int p = 0; p < P; ++p) {
        uint64_t* lb = W.lookback + (size_t)p * W.n_sort_tiles * 256;
        if (p == 0)
            WS_LAUNCH(W.prof, WSK_ONESWEEP, st, (k_onesweep<T, true><<<W.n_sort_tiles, WS_SORT_NT, smem, st>>>(
                values, nullptr, dst, W.sort_tiles, W.lsegs, W.hist, lb, W.tile_counter + p, p, status, spin_limit)));
        else
            WS_LAUNCH(W.prof, WSK_ONESWEEP, st, (k_onesweep<T, false><<<W.n_sort_tiles, WS_SORT_NT, smem, st>>>(
                values, src, dst, W.sort_tiles, W.lsegs, W.hist, lb, W.tile_counter + p, p, status, spin_limit)));
        K* tmp = src; src = dst; dst = tmp;
    }
    *sorted = src;   // the buffer written last
    return cudaGetLastError();
}

template cudaError_t ws_large_sort<float>(const LargeWork<float>&, const float*, uint32_t*, uint64_t, cudaStream_t,
                                          uint32_t**);
template cudaError_t ws_large_sort<double>(const LargeWork<double>&, const double*, uint32_t*, uint64_t,
                                           cudaStream_t, uint64_t**);
