// ws_noalloc.cu -- a backward entry point that never allocates device memory.
//
// Who needs it: code that must not call cudaMalloc/cudaFree at the point where
// it runs the backward -- for example a training step whose framework has
// already reserved all device memory in its own pool, or a loop that cannot
// afford the implicit device-wide synchronisation cudaMalloc and cudaFree
// perform.  The regular ws_prox_backward gets its per-cluster scratch from a
// plan, which allocates on first use of a shape.
//
// Here the scratch (one sum and one count per cluster) lives in a
// file-scope __device__ array that every GPU loading the library holds until
// the process exits.  Host code cannot use the array's name as a device
// address, so the address is looked up with cudaGetSymbolAddress once per
// device, with that device current, the first time the entry point runs on
// it; later calls reuse the cached address.  That first call on a device
// should therefore come before any stream capture begins, and the cached
// address does not survive a device reset (cudaDeviceReset): the entry point
// must not be used across one.
#include <mutex>

#include "../../include/ws_prox.h"
#include "ws_common.cuh"

namespace {

constexpr int64_t kMaxElems = WS_NOALLOC_MAX_ELEMS;
constexpr size_t kSumBytes = (size_t)kMaxElems * sizeof(double);   // room for double sums
constexpr size_t kScratchBytes = kSumBytes + (size_t)kMaxElems * sizeof(int32_t);
constexpr int kMaxDevices = 64;

}  // namespace

// Shared by every call on a device; contents persist between calls.
static __device__ __align__(256) unsigned char g_ws_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Address of the scratch array on the current device (set-up on first use).
ws_status scratch_for_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return WS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_ws_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return WS_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return WS_OK;
}

template <typename T>
__global__ void k_na_clear(T* sum, int32_t* cnt, int64_t d) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
        sum[i] = (T)0;
        cnt[i] = 0;
    }
}

template <typename T>
__global__ void k_na_accum(const T* __restrict__ g, const int32_t* __restrict__ ids, int64_t d, T* sum,
                           int32_t* cnt) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t id = ids[i];
        if (id < 0 || (int64_t)id >= d) continue;   // out-of-range ids are skipped
        atomicAdd(&sum[id], g[i]);
        atomicAdd(&cnt[id], 1);
    }
}

template <typename T>
__global__ void k_na_apply(const int32_t* __restrict__ ids, int64_t d, const T* __restrict__ sum,
                           const int32_t* __restrict__ cnt, T* gin) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t id = ids[i];
        if (id < 0 || (int64_t)id >= d) continue;
        gin[i] = sum[id] / (T)cnt[id];
    }
}

template <typename T>
ws_status run(const void* grad_out, const int32_t* ids, int64_t d, void* grad_in, cudaStream_t st, void* scratch) {
    T* sum = reinterpret_cast<T*>(scratch);
    int32_t* cnt = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(scratch) + kSumBytes);
    const int nt = 256;
    const int nb = (int)((d + nt - 1) / nt < 4096 ? (d + nt - 1) / nt : 4096);
    // each launch is checked on its own (the caller's stale errors were
    // cleared on entry), so a failure is reported by the call that caused it
    k_na_clear<T><<<nb, nt, 0, st>>>(sum, cnt, d);
    if (cudaGetLastError() != cudaSuccess) return WS_ERR_CUDA;
    k_na_accum<T><<<nb, nt, 0, st>>>((const T*)grad_out, ids, d, sum, cnt);
    if (cudaGetLastError() != cudaSuccess) return WS_ERR_CUDA;
    k_na_apply<T><<<nb, nt, 0, st>>>(ids, d, sum, cnt, (T*)grad_in);
    if (cudaGetLastError() != cudaSuccess) return WS_ERR_CUDA;
    return WS_OK;
}

}  // namespace

extern "C" ws_status ws_prox_backward_noalloc(const void* grad_out, const int32_t* cluster_ids, int64_t d,
                                              void* grad_in, ws_dtype dtype, void* stream) {
    if (d < 0 || d > kMaxElems) return WS_ERR_INVALID;
    if (dtype != WS_F32 && dtype != WS_F64) return WS_ERR_INVALID;
    if (d == 0) return WS_OK;
    if (!grad_out || !cluster_ids || !grad_in) return WS_ERR_INVALID;
    cudaGetLastError();   // a launch error left by earlier, unrelated code is not this call's
    void* scratch = nullptr;
    ws_status s = scratch_for_current_device(&scratch);
    if (s != WS_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == WS_F64 ? run<double>(grad_out, cluster_ids, d, grad_in, st, scratch)
                           : run<float>(grad_out, cluster_ids, d, grad_in, st, scratch);
}
