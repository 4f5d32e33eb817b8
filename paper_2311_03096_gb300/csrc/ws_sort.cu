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
// 6144 keys by digit in shared memory, publishes its per-digit counts, gets
// the counts of the earlier tiles of the same segment through a decoupled
// look-back (bounded waits), and writes its keys as per-digit contiguous runs.
#include <algorithm>

#include "ws_kernels.cuh"

namespace {

// Look-back word: [63:62] status (1 = tile aggregate, 2 = inclusive prefix),
// [61:40] epoch of the call that wrote it, [39:0] count.  Every call uses a
// new epoch (incremented on the device, so CUDA-graph replays also advance
// it), which makes the words of the previous call read as "not ready"
// without clearing the array.
constexpr uint64_t LB_AGG = 1ull << 62;
constexpr uint64_t LB_INC = 2ull << 62;
constexpr uint64_t LB_STATUS = 3ull << 62;
constexpr int LB_EPOCH_SHIFT = 40;
constexpr uint64_t LB_EPOCH_MASK = ((1ull << 22) - 1ull) << LB_EPOCH_SHIFT;
constexpr uint64_t LB_CNT = (1ull << LB_EPOCH_SHIFT) - 1ull;

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Also the smallest effective exponent of a nonzero value of each segment
// (seg_emin, reduced with atomicMin; cleared to INT_MAX before the launch),
// which fixes the segment's fixed-point scale.  A persistent grid: each CTA
// walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (increasing, so it
// meets each segment in one run) and adds its shared-memory counts to the
// segment's global histogram once per segment, not once per tile.
template <typename T>
__global__ void __launch_bounds__(WS_SORT_NT) k_hist(const T* __restrict__ values, const TileDesc* __restrict__ tiles,
                                                     int n_tiles, uint32_t* hist, int32_t* seg_emin,
                                                     uint32_t* status) {
    typedef KeyOf<T> KO;
    constexpr int P = KO::BITS / 8;
    __shared__ uint32_t h[P * 256];
    __shared__ int s_emin;
    for (int i = threadIdx.x; i < P * 256; i += WS_SORT_NT) h[i] = 0;
    if (threadIdx.x == 0) s_emin = 0x7fffffff;
    __syncthreads();
    bool bad = false;
    int emin = 0x7fffffff;
    auto count = [&](T v) {
        bad |= !ws_isfinite(v);
        if (v != (T)0) emin = min(emin, ws_eff_exp(v));
        const typename KO::K k = KO::to_key(v);
#pragma unroll
        for (int p = 0; p < P; ++p) atomicAdd(&h[p * 256 + (int)((k >> (8 * p)) & 0xff)], 1u);
    };
    auto flush = [&](int lseg) {   // (all threads; ends with zero counts)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        if ((threadIdx.x & 31) == 0 && emin != 0x7fffffff) atomicMin(&s_emin, emin);
        emin = 0x7fffffff;
        __syncthreads();
        if (threadIdx.x == 0 && s_emin != 0x7fffffff) atomicMin(&seg_emin[lseg], s_emin);
        uint32_t* gh = hist + (size_t)lseg * P * 256;
        for (int i = threadIdx.x; i < P * 256; i += WS_SORT_NT) {
            if (h[i]) atomicAdd(&gh[i], h[i]);
            h[i] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_emin = 0x7fffffff;
        __syncthreads();
    };
    constexpr int VEC = 16 / (int)sizeof(T);                  // values per 16-byte load
    constexpr int NV = WS_SORT_TILE / (WS_SORT_NT * VEC);     // 16-byte loads per thread
    int cur = -1;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const TileDesc td = tiles[tile];
        if (td.lseg != cur) {
            if (cur >= 0) flush(cur);
            cur = td.lseg;
        }
        const T* src = values + td.vpos;
        if (td.len == WS_SORT_TILE && (((uintptr_t)src) & 15) == 0) {
            // whole, aligned tile: every load issued before the first count
            uint4 buf[NV];
#pragma unroll
            for (int j = 0; j < NV; ++j) buf[j] = __ldcs(reinterpret_cast<const uint4*>(src) + j * WS_SORT_NT + threadIdx.x);
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                const T* e = reinterpret_cast<const T*>(&buf[j]);
#pragma unroll
                for (int u = 0; u < VEC; ++u) count(e[u]);
            }
        } else {
            for (int i = threadIdx.x; i < td.len; i += WS_SORT_NT) count(src[i]);
        }
    }
    if (cur >= 0) flush(cur);
    if (bad) ws_flag(status, WS_STATUS_NONFINITE);
}

// exclusive scan of every (segment, pass) histogram, in place
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t* hist, uint32_t* epoch) {
    __shared__ uint32_t ws[8];
    if (blockIdx.x == 0 && threadIdx.x == 0) *epoch = (*epoch + 1u) & ((1u << 22) - 1u);
    uint32_t* h = hist + (size_t)blockIdx.x * 256;
    uint32_t v = h[threadIdx.x];
    uint32_t tot;
    uint32_t ex = ws_block_excl_scan<256, int>((int)v, (int*)ws, (int*)&tot);
    h[threadIdx.x] = ex;
}

template <typename T, bool FIRST>
__global__ void __launch_bounds__(WS_SORT_NT, sizeof(T) == 4 ? 3 : 2) k_onesweep(const T* __restrict__ values,
                                                            const typename KeyOf<T>::K* __restrict__ keys_in,
                                                            typename KeyOf<T>::K* __restrict__ keys_out,
                                                            const TileDesc* __restrict__ tiles,
                                                            const LargeSeg* __restrict__ lsegs,
                                                            const uint32_t* __restrict__ hist, uint64_t* lookback,
                                                            uint32_t* counter, const uint32_t* __restrict__ epoch_p,
                                                            int pass, uint32_t* status, uint64_t spin_limit) {
    typedef KeyOf<T> KO;
    typedef typename KO::K K;
    constexpr int P = KO::BITS / 8;
    constexpr int NT = WS_SORT_NT, ITEMS = WS_SORT_ITEMS, TILE = WS_SORT_TILE, NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* skeys = reinterpret_cast<K*>(smem_raw);
    uint32_t* whist = reinterpret_cast<uint32_t*>(smem_raw + sizeof(K) * TILE);   // [NW][256] per-warp counts
    uint32_t* mbins = whist + NW * 256;                                             // [NW][256] peer masks
    uint32_t* dstart = mbins + NW * 256;
    int64_t* gbase = reinterpret_cast<int64_t*>(dstart + 256);
    __shared__ int s_tile;
    __shared__ int s_timeout;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t* my = whist + w * 256;
    uint32_t* mb = mbins + w * 256;
    for (int i = lane; i < 256; i += 32) { my[i] = 0; mb[i] = 0; }
    if (t == 0) { s_tile = (int)atomicAdd(counter, 1u); s_timeout = 0; }
    __syncthreads();
    const int tile = s_tile;
    const TileDesc td = tiles[tile];
    const int64_t seg_k = lsegs[td.lseg].kpos;
    const uint32_t* dbase = hist + ((size_t)td.lseg * P + pass) * 256;
    const uint64_t ep = (uint64_t)(*epoch_p) << LB_EPOCH_SHIFT;
    const int shift = 8 * pass;
    uint64_t* my_lb = lookback + (size_t)tile * 256;

    // Warp w holds keys [w*32*ITEMS, (w+1)*32*ITEMS) of the tile, item k of
    // lane l being key w*32*ITEMS + 32k + l, so ranking items in order k and
    // lanes in order l is stable.
    K key[ITEMS];
    static_assert(ITEMS % 2 == 0 && TILE <= 65536, "ranks are packed two per word");
    uint32_t pos2[ITEMS / 2];   // warp-local rank of item k in half k % 2 of word k / 2 (fewer registers)
    const int base = w * 32 * ITEMS + lane;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const int p = base + k * 32;
        const bool v = p < td.len;
        if (FIRST) key[k] = v ? KO::to_key(values[td.vpos + p]) : (K)0;
        else key[k] = v ? keys_in[td.kpos + p] : (K)0;
    }
    // Rank within the warp: the lanes holding the same digit find each other
    // by OR-ing their lane bits into the digit's shared-memory word; the
    // lowest of them advances the warp's count of that digit.
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        const bool v = base + k * 32 < td.len;
        const uint32_t dg = (uint32_t)(key[k] >> shift) & 0xffu;
        if (v) atomicOr(&mb[dg], 1u << lane);
        __syncwarp();
        const unsigned peers = v ? mb[dg] : 0u;
        const int before = v ? (int)my[dg] : 0;
        __syncwarp();
        const int r = __popc(peers & lt);
        const uint32_t rk = (uint32_t)(before + r);
        if (k % 2 == 0) pos2[k / 2] = rk; else pos2[k / 2] |= rk << 16;
        if (v && r == 0) { my[dg] = (uint32_t)(before + __popc(peers)); mb[dg] = 0u; }
        __syncwarp();
    }
    __syncthreads();
    // Per digit: exclusive scan over the warps, and the tile's count, which is
    // published at once so that later tiles' look-backs can pass this one.
    uint32_t cnt = 0;
    if (t < 256) {
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
            const uint32_t c = whist[ww * 256 + t];
            whist[ww * 256 + t] = cnt;
            cnt += c;
        }
        st_relaxed_u64(&my_lb[t], (td.tin == 0 ? LB_INC : LB_AGG) | ep | (uint64_t)cnt);
    }
    // exclusive scan of the counts over the 256 digits
    {
        uint32_t tot;
        const uint32_t ex = ws_block_excl_scan<NT, int>((int)cnt, (int*)mbins, (int*)&tot);
        if (t < 256) dstart[t] = ex;
    }
    __syncthreads();
    // stage the tile in digit order (frees the key registers before the
    // look-back)
#pragma unroll
    for (int k = 0; k < ITEMS; ++k) {
        if (base + k * 32 < td.len) {
            const uint32_t dg = (uint32_t)(key[k] >> shift) & 0xffu;
            const int rk = (int)((pos2[k / 2] >> (16 * (k % 2))) & 0xffffu);
            skeys[rk + (int)(dstart[dg] + my[dg])] = key[k];
        }
    }

    // look back over earlier tiles of the segment (windows of 4 predecessors
    // per round trip)
    if (t < 256) {
        int64_t gb;   // global position of this digit's first key of the tile, minus its local start
        if (td.tin == 0) {
            gb = 0;
        } else {
            uint64_t run = 0;
            int j = tile - 1;
            uint64_t it = 0;
            bool done = false;
            while (!done) {
                constexpr int WIN = 4;
                uint64_t v[WIN];
                const int nwin = min(WIN, j - td.first + 1);
#pragma unroll
                for (int u = 0; u < WIN; ++u)
                    if (u < nwin) v[u] = ld_relaxed_u64(&lookback[(size_t)(j - u) * 256 + t]);
                int u = 0;
                for (; u < nwin; ++u) {
                    uint64_t x = v[u];
                    while ((x & LB_STATUS) == 0 || (x & LB_EPOCH_MASK) != ep) {
                        if (++it > spin_limit) { s_timeout = 1; break; }
                        ws_backoff((int)min(it, (uint64_t)1 << 20));
                        x = ld_relaxed_u64(&lookback[(size_t)(j - u) * 256 + t]);
                    }
                    if ((x & LB_STATUS) == 0 || (x & LB_EPOCH_MASK) != ep) { done = true; break; }   // gave up
                    run += x & LB_CNT;
                    if ((x & LB_STATUS) == LB_INC || j - u <= td.first) { done = true; break; }
                }
                if (!done) j -= nwin;
            }
            st_relaxed_u64(&my_lb[t], LB_INC | ep | (run + cnt));
            gb = (int64_t)run;
        }
        gbase[t] = seg_k + (int64_t)dbase[t] + gb - (int64_t)dstart[t];
    }
    __syncthreads();
    if (t == 0 && s_timeout) ws_flag(status, WS_STATUS_TIMEOUT);
#pragma unroll 4
    for (int k = 0; k < ITEMS; ++k) {
        const int j = t + k * NT;
        if (j < td.len) {
            const K kk = skeys[j];
            const uint32_t dg = (uint32_t)(kk >> shift) & 0xffu;
            keys_out[gbase[dg] + j] = kk;
        }
    }
}

}  // namespace

template <typename T>
size_t ws_onesweep_smem() {
    typedef typename KeyOf<T>::K K;
    return sizeof(K) * WS_SORT_TILE + sizeof(uint32_t) * (2 * (WS_SORT_NT / 32) * 256 + 256) +
           sizeof(int64_t) * 256;
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
    e = cudaMemsetAsync(W.tile_counter, 0, sizeof(uint32_t) * P, st);
    if (e) return e;
    e = cudaMemsetAsync(W.seg_emin, 0x7f, sizeof(int32_t) * (size_t)W.n_lseg, st);
    if (e) return e;
    // the histogram's persistent grid: every CTA resident at once
    static const int hist_grid = [] {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hist<T>, WS_SORT_NT, 0) != cudaSuccess) {
            cudaGetLastError();
            return 2 * 152;
        }
        return std::max(1, sms * std::max(per_sm, 1));
    }();
    WS_LAUNCH(W.prof, WSK_HIST, st,
              (k_hist<T><<<W.n_sort_tiles < hist_grid ? W.n_sort_tiles : hist_grid, WS_SORT_NT, 0, st>>>(
                  values, W.sort_tiles, W.n_sort_tiles, W.hist, W.seg_emin, status)));
    WS_LAUNCH(W.prof, WSK_HIST_SCAN, st, (k_hist_scan<<<W.n_lseg * P, 256, 0, st>>>(W.hist, W.epoch)));
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
                values, nullptr, dst, W.sort_tiles, W.lsegs, W.hist, lb, W.tile_counter + p, W.epoch, p, status,
                spin_limit)));
        else
            WS_LAUNCH(W.prof, WSK_ONESWEEP, st, (k_onesweep<T, false><<<W.n_sort_tiles, WS_SORT_NT, smem, st>>>(
                values, src, dst, W.sort_tiles, W.lsegs, W.hist, lb, W.tile_counter + p, W.epoch, p, status,
                spin_limit)));
        K* tmp = src; src = dst; dst = tmp;
    }
    *sorted = src;   // the buffer written last
    return cudaGetLastError();
}

template cudaError_t ws_large_sort<float>(const LargeWork<float>&, const float*, uint32_t*, uint64_t, cudaStream_t,
                                          uint32_t**);
template cudaError_t ws_large_sort<double>(const LargeWork<double>&, const double*, uint32_t*, uint64_t,
                                           cudaStream_t, uint64_t**);
