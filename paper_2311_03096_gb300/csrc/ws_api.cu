// ws_api.cu -- the C ABI (include/ws_prox.h): contexts, plans and launches.
// Host code only sequences launches; every step of the prox runs in the
// kernels of ws_small.cu, ws_sort.cu and ws_large.cu.
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/ws_prox.h"
#include "ws_kernels.cuh"

namespace {

constexpr uint64_t WS_DEFAULT_SPIN = 1ull << 24;

struct PlanCacheEntry {
    int64_t d;
    ws_dtype dtype;
    int sort_only;   // every segment on the device-wide path (R and the measure need its sorted keys)
    ws_plan* plan;
};

}  // namespace

struct ws_ctx {
    int device = 0;
    uint32_t* status = nullptr;   // device status word
    uint64_t spin_limit = WS_DEFAULT_SPIN;
    int64_t small_max_override = -1;
    int ic_cap = 32;   // in-tile Imminent Collisions round cap
    bool inexact = false;   // WS_STATUS_INEXACT seen by ws_get_status, not yet reported
    std::vector<PlanCacheEntry> cache;
    std::mutex mu;
    WsProf prof;
    double prof_ms[WSK_COUNT] = {};
    long long prof_cnt[WSK_COUNT] = {};
};

struct ws_plan {
    ws_ctx* ctx = nullptr;
    ws_dtype dtype = WS_F32;
    int64_t n = 0, n_seg = 0;
    int64_t small_max = 0;
    bool sort_only = false;   // no one-CTA segments: everything takes the device-wide path
    int64_t small_force = -1; // >= 0: this plan's one-CTA length threshold (autotuned plans)
    int ic_cap = -1;          // >= 0: this plan's round cap (autotuned plans), else the context's
    std::vector<int64_t> h_offsets;
    int64_t* d_offsets = nullptr;
    int32_t* d_small = nullptr;
    int n_small = 0;
    int32_t* small_gen = nullptr;     // one-CTA segments passed to the general kernel
    int32_t* small_gen_count = nullptr;
    double* d_lambda1 = nullptr;   // lambda slot for single-vector calls
    // large path
    int n_lseg = 0, n_sort_tiles = 0, n_hull_tiles = 0;
    int64_t n_keys = 0;
    LargeSeg* d_lsegs = nullptr;
    TileDesc* d_sort_tiles = nullptr;
    TileDesc* d_hull_tiles = nullptr;
    int n_levels = 0;
    std::vector<void*> allocs;
    void* keys_a = nullptr;
    void* keys_b = nullptr;
    uint32_t* hist = nullptr;
    uint64_t* lookback = nullptr;
    uint32_t* tile_counter = nullptr;
    uint32_t* epoch = nullptr;
    int32_t* seg_emin = nullptr;
    uint16_t* vp = nullptr;
    i128* vx = nullptr;
    int32_t* nvert = nullptr;
    i128* tile_total = nullptr;
    int32_t* arrive = nullptr;
    Piece* pieces = nullptr;
    int32_t* npieces = nullptr;
    int32_t* tile_piece = nullptr;
    int32_t* gen_list = nullptr;
    int32_t* gen_count = nullptr;
    int32_t* keepR = nullptr;
    int32_t* keepL = nullptr;
    int32_t* jflag0 = nullptr;
    int32_t* seg_mode = nullptr;
    i128* tile_base = nullptr;
    TileScale* scales = nullptr;
    int32_t* tile_rounds = nullptr;
    i128* seg_total = nullptr;
    int32_t* seg_below = nullptr;
    SegRuntime* rt = nullptr;
    void* table = nullptr;
    DirEntry* dir = nullptr;
    void* stat_partial = nullptr;
    void* bsum = nullptr;
    int32_t* bcnt = nullptr;
    unsigned long long* bacc = nullptr;
    int32_t* bwd_seg = nullptr;
    // plans with both one-CTA and device-wide segments: the one-CTA kernel
    // runs on this stream, forked from and joined back into the caller's
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

template <typename T>
LargeWork<T> make_work(const ws_plan* p) {
    typedef typename KeyOf<T>::K K;
    LargeWork<T> W;
    W.n_lseg = p->n_lseg;
    W.n_sort_tiles = p->n_sort_tiles;
    W.n_hull_tiles = p->n_hull_tiles;
    W.n_keys = p->n_keys;
    W.lsegs = p->d_lsegs;
    W.sort_tiles = p->d_sort_tiles;
    W.hull_tiles = p->d_hull_tiles;
    W.keys_a = (K*)p->keys_a;
    W.keys_b = (K*)p->keys_b;
    W.hist = p->hist;
    W.lookback = p->lookback;
    W.tile_counter = p->tile_counter;
    W.epoch = p->epoch;
    W.seg_emin = p->seg_emin;
    W.vp = p->vp;
    W.vx = p->vx;
    W.nvert = p->nvert;
    W.tile_total = p->tile_total;
    W.arrive = p->arrive;
    W.pieces = p->pieces;
    W.npieces = p->npieces;
    W.tile_piece = p->tile_piece;
    W.gen_list = p->gen_list;
    W.gen_count = p->gen_count;
    W.keepR = p->keepR;
    W.keepL = p->keepL;
    W.jflag0 = p->jflag0;
    W.seg_mode = p->seg_mode;
    W.tile_base = p->tile_base;
    W.scales = p->scales;
    W.tile_rounds = p->tile_rounds;
    W.ic_cap = p->ic_cap >= 0 ? p->ic_cap : p->ctx->ic_cap;
    W.seg_total = p->seg_total;
    W.seg_below = p->seg_below;
    W.rt = p->rt;
    W.table = (CEntry<T>*)p->table;
    W.dir = p->dir;
    W.bsum = (T*)p->bsum;
    W.bcnt = p->bcnt;
    W.bacc = p->bacc;
    W.bwd_seg = p->bwd_seg;
    W.prof = &p->ctx->prof;
    return W;
}

ws_status plan_alloc(ws_plan* p, void** dst, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return WS_ERR_NOMEM;
    }
    p->allocs.push_back(ptr);
    *dst = ptr;
    return WS_OK;
}

template <typename X>
ws_status plan_upload(ws_plan* p, X** dst, const std::vector<X>& src) {
    ws_status s = plan_alloc(p, (void**)dst, sizeof(X) * src.size());
    if (s) return s;
    if (!src.empty() && cudaMemcpy(*dst, src.data(), sizeof(X) * src.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return WS_ERR_CUDA;
    return WS_OK;
}

int ceil_log2(int64_t v) {
    int k = 0;
    while (((int64_t)1 << k) < v) ++k;
    return k;
}

ws_status build_plan(ws_plan* p) {
    const bool f64 = p->dtype == WS_F64;
    const int64_t small_cap = f64 ? SmallCfg<double>::CAP : SmallCfg<float>::CAP;
    p->small_max = p->ctx->small_max_override >= 0 ? std::min<int64_t>(p->ctx->small_max_override, small_cap)
                                                     : small_cap;
    if (p->small_force >= 0) p->small_max = std::min<int64_t>(p->small_force, small_cap);
    if (p->sort_only) p->small_max = 0;
    const size_t vsize = f64 ? 8 : 4, ksize = vsize;
    std::vector<int32_t> small;
    std::vector<LargeSeg> lsegs;
    std::vector<TileDesc> stiles, htiles;
    int64_t kpos = 0, dir_pos = 0;
    for (int64_t s = 0; s < p->n_seg; ++s) {
        int64_t a = p->h_offsets[s], len = p->h_offsets[s + 1] - a;
        if (len <= p->small_max || len <= 1) { small.push_back((int32_t)s); continue; }
        LargeSeg ls;
        memset(&ls, 0, sizeof ls);
        ls.vpos = a; ls.kpos = kpos; ls.len = len; ls.seg = (int32_t)s;
        int lseg = (int)lsegs.size();
        ls.sort_first = (int32_t)stiles.size();
        for (int64_t o = 0, i = 0; o < len; o += WS_SORT_TILE, ++i) {
            TileDesc td;
            td.kpos = kpos + o; td.vpos = a + o; td.len = (int32_t)std::min<int64_t>(WS_SORT_TILE, len - o);
            td.lseg = lseg; td.first = ls.sort_first; td.tin = (int32_t)i;
            stiles.push_back(td);
        }
        ls.sort_count = (int32_t)stiles.size() - ls.sort_first;
        ls.hull_first = (int32_t)htiles.size();
        for (int64_t o = 0, i = 0; o < len; o += WS_HULL_TILE, ++i) {
            TileDesc td;
            td.kpos = kpos + o; td.vpos = a + o; td.len = (int32_t)std::min<int64_t>(WS_HULL_TILE, len - o);
            td.lseg = lseg; td.first = ls.hull_first; td.tin = (int32_t)i;
            htiles.push_back(td);
        }
        ls.hull_count = (int32_t)htiles.size() - ls.hull_first;
        ls.dir_cap_log2 = std::min(ceil_log2(len), WS_DIR_MAX_LOG2);
        ls.dir_pos = dir_pos;
        dir_pos += ((int64_t)1 << ls.dir_cap_log2) + 1;
        kpos += (len + 3) & ~(int64_t)3;   // keep every segment's keys 16-byte aligned
        lsegs.push_back(ls);
    }
    p->n_small = (int)small.size();
    p->n_lseg = (int)lsegs.size();
    if (p->n_small > 0 && p->n_lseg > 0) {
        if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return WS_ERR_CUDA;
        }
    }
    p->n_sort_tiles = (int)stiles.size();
    p->n_hull_tiles = (int)htiles.size();
    p->n_keys = kpos;
    // merge-tree depth: levels above the tiles of the longest segment
    p->n_levels = 0;
    for (const LargeSeg& ls : lsegs) p->n_levels = std::max(p->n_levels, ceil_log2(ls.hull_count) + 1);
    ws_status st;
    std::vector<int64_t> offs(p->h_offsets);
    if ((st = plan_upload(p, &p->d_offsets, offs))) return st;
    if ((st = plan_upload(p, &p->d_small, small))) return st;
    if ((st = plan_alloc(p, (void**)&p->small_gen, sizeof(int32_t) * std::max<size_t>(small.size(), 1)))) return st;
    if ((st = plan_alloc(p, (void**)&p->small_gen_count, sizeof(int32_t)))) return st;
    if ((st = plan_alloc(p, (void**)&p->d_lambda1, sizeof(double)))) return st;
    if (p->n_lseg == 0) return WS_OK;
    if ((st = plan_upload(p, &p->d_lsegs, lsegs))) return st;
    if ((st = plan_upload(p, &p->d_sort_tiles, stiles))) return st;
    if ((st = plan_upload(p, &p->d_hull_tiles, htiles))) return st;
    const int P = f64 ? 8 : 4;
    const size_t nk = (size_t)p->n_keys, nh = (size_t)p->n_hull_tiles, slots = nk + (size_t)p->n_lseg;
    if ((st = plan_alloc(p, &p->keys_a, ksize * nk))) return st;
    if ((st = plan_alloc(p, &p->keys_b, ksize * nk))) return st;
    if ((st = plan_alloc(p, (void**)&p->hist, sizeof(uint32_t) * p->n_lseg * P * 256))) return st;
    if ((st = plan_alloc(p, (void**)&p->lookback, sizeof(uint64_t) * (size_t)P * p->n_sort_tiles * 256))) return st;
    if ((st = plan_alloc(p, (void**)&p->tile_counter, sizeof(uint32_t) * P))) return st;
    if ((st = plan_alloc(p, (void**)&p->epoch, sizeof(uint32_t)))) return st;
    if ((st = plan_alloc(p, (void**)&p->seg_emin, sizeof(int32_t) * p->n_lseg))) return st;
    if ((st = plan_alloc(p, &p->stat_partial, ws_R_partial_bytes(p->n_sort_tiles)))) return st;
    if (cudaMemset(p->epoch, 0, sizeof(uint32_t)) != cudaSuccess) return WS_ERR_CUDA;
    if (cudaMemset(p->lookback, 0, sizeof(uint64_t) * (size_t)P * p->n_sort_tiles * 256) != cudaSuccess)
        return WS_ERR_CUDA;
    if ((st = plan_alloc(p, (void**)&p->vp, sizeof(uint16_t) * nh * (WS_HULL_TILE + 1)))) return st;
    if ((st = plan_alloc(p, (void**)&p->vx, sizeof(i128) * nh * (WS_HULL_TILE + 1)))) return st;
    if ((st = plan_alloc(p, (void**)&p->nvert, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->tile_total, sizeof(i128) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->arrive, sizeof(int32_t) * (size_t)p->n_levels * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->pieces, sizeof(Piece) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->npieces, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->tile_piece, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->gen_list, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->gen_count, sizeof(int32_t)))) return st;
    if ((st = plan_alloc(p, (void**)&p->keepR, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->keepL, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->jflag0, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->seg_mode, sizeof(int32_t) * p->n_lseg))) return st;
    if ((st = plan_alloc(p, (void**)&p->tile_base, sizeof(i128) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->scales, sizeof(TileScale) * WS_NSCALE * p->n_lseg))) return st;
    if ((st = plan_alloc(p, (void**)&p->tile_rounds, sizeof(int32_t) * nh))) return st;
    if ((st = plan_alloc(p, (void**)&p->seg_total, sizeof(i128) * p->n_lseg))) return st;
    if ((st = plan_alloc(p, (void**)&p->seg_below, sizeof(int32_t) * p->n_lseg))) return st;
    if ((st = plan_alloc(p, (void**)&p->rt, sizeof(SegRuntime) * p->n_lseg))) return st;
    // (+4 entries: the lookup reads whole 32-byte sectors of the table)
    if ((st = plan_alloc(p, &p->table, (f64 ? sizeof(CEntry<double>) : sizeof(CEntry<float>)) * (slots + 4)))) return st;
    if ((st = plan_alloc(p, (void**)&p->dir, sizeof(DirEntry) * (size_t)dir_pos))) return st;
    if ((st = plan_alloc(p, &p->bsum, vsize * slots))) return st;
    if ((st = plan_alloc(p, (void**)&p->bcnt, sizeof(int32_t) * slots))) return st;
    if ((st = plan_alloc(p, (void**)&p->bacc, 2 * sizeof(unsigned long long) * slots))) return st;
    if ((st = plan_alloc(p, (void**)&p->bwd_seg, 2 * sizeof(int32_t) * p->n_lseg))) return st;
    if (cudaMemset(p->rt, 0, sizeof(SegRuntime) * p->n_lseg) != cudaSuccess) return WS_ERR_CUDA;
    return WS_OK;
}

__global__ void k_set_lambda(double* dst, double v) { *dst = v; }

ws_status map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return WS_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? WS_ERR_NOMEM : WS_ERR_CUDA;
}

// The one-CTA segments and the device-wide chain touch disjoint elements, so
// with both present the one-CTA kernel runs on the plan's side stream, after
// everything already queued on the caller's stream (fork) and before anything
// queued there after this call (join).  Event record/wait pairs: capturable.
// *ss: the stream for the one-CTA kernel (st itself without a side stream);
// false on a CUDA error.
bool fork(ws_plan* p, cudaStream_t st, cudaStream_t* ss) {
    *ss = st;
    if (!p->side) return true;
    if (cudaEventRecord(p->ev_fork, st) != cudaSuccess || cudaStreamWaitEvent(p->side, p->ev_fork, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    *ss = p->side;
    return true;
}

bool join(ws_plan* p, cudaStream_t st) {
    if (!p->side) return true;
    if (cudaEventRecord(p->ev_join, p->side) != cudaSuccess || cudaStreamWaitEvent(st, p->ev_join, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

template <typename T>
ws_status run_forward(ws_plan* p, const void* values, const double* lambdas, void* out, int32_t* ids,
                      int64_t* n_clusters, ws_prec prec, const WsEpi& ep, cudaStream_t st,
                      const int32_t* ids_prev = nullptr) {
    const int fp64 = prec == WS_PREC_FP64 ? 1 : 0;
    cudaStream_t ss;
    if (!fork(p, st, &ss)) return WS_ERR_CUDA;
    cudaError_t e = ws_launch_small<T>((const T*)values, p->d_offsets, p->d_small, p->n_small, lambdas, (T*)out, ids,
                                       n_clusters, fp64, ep, p->ctx->status, ss, &p->ctx->prof, p->small_gen,
                                       p->small_gen_count, p->ic_cap >= 0 ? p->ic_cap : p->ctx->ic_cap, ids_prev);
    if (e) { join(p, st); return map_cuda(e); }
    if (p->n_lseg > 0) {
        LargeWork<T> W = make_work<T>(p);
        e = ws_large_prox<T>(W, (const T*)values, lambdas, (T*)out, ids, n_clusters, fp64, ep, p->ctx->status,
                             p->ctx->spin_limit, p->n_levels, st);
    }
    if (!join(p, st)) return WS_ERR_CUDA;
    return e ? map_cuda(e) : WS_OK;
}

template <typename T>
ws_status run_backward(ws_plan* p, const void* g, const int32_t* ids, void* gin, cudaStream_t st) {
    cudaStream_t ss;
    if (!fork(p, st, &ss)) return WS_ERR_CUDA;
    cudaError_t e = ws_launch_small_backward<T>((const T*)g, ids, p->d_offsets, p->d_small, p->n_small, (T*)gin,
                                                p->ctx->status, ss, &p->ctx->prof);
    if (e) { join(p, st); return map_cuda(e); }
    if (p->n_lseg > 0) {
        LargeWork<T> W = make_work<T>(p);
        e = ws_large_backward<T>(W, (const T*)g, ids, (T*)gin, p->ctx->status, st);
    }
    if (!join(p, st)) return WS_ERR_CUDA;
    return e ? map_cuda(e) : WS_OK;
}

ws_status plan_create_impl(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg, ws_dtype dtype,
                           bool sort_only, int64_t small_force = -1);

ws_plan* cached_plan(ws_ctx* ctx, int64_t d, ws_dtype dtype, ws_status* st, int sort_only = 0) {
    std::lock_guard<std::mutex> g(ctx->mu);
    for (auto& c : ctx->cache)
        if (c.d == d && c.dtype == dtype && c.sort_only == sort_only) { *st = WS_OK; return c.plan; }
    int64_t offs[2] = {0, d};
    ws_plan* p = nullptr;
    *st = plan_create_impl(ctx, &p, offs, 1, dtype, sort_only != 0);
    if (*st) return nullptr;
    if (ctx->cache.size() >= 8) {   // keep at most 8 cached shapes
        ws_plan_destroy(ctx->cache.front().plan);
        ctx->cache.erase(ctx->cache.begin());
    }
    ctx->cache.push_back({d, dtype, sort_only, p});
    return p;
}

ws_status plan_create_impl(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg, ws_dtype dtype,
                           bool sort_only, int64_t small_force) {
    if (!ctx || !plan || n_seg < 0 || (n_seg > 0 && !offsets) || (dtype != WS_F32 && dtype != WS_F64))
        return WS_ERR_INVALID;
    *plan = nullptr;
    if (n_seg > 0 && offsets[0] != 0) return WS_ERR_INVALID;
    if (n_seg >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    for (int64_t s = 0; s < n_seg; ++s) {
        int64_t len = offsets[s + 1] - offsets[s];
        if (len < 0 || len >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return WS_ERR_CUDA;
    ws_plan* p = new (std::nothrow) ws_plan();
    if (!p) return WS_ERR_NOMEM;
    p->ctx = ctx;
    p->dtype = dtype;
    p->sort_only = sort_only;
    p->small_force = small_force;
    p->n_seg = n_seg;
    p->h_offsets.assign(offsets ? offsets : nullptr, offsets ? offsets + n_seg + 1 : nullptr);
    if (n_seg == 0) p->h_offsets.assign(1, 0);
    p->n = p->h_offsets.back();
    ws_status st = build_plan(p);
    if (st) { ws_plan_destroy(p); return st; }
    *plan = p;
    return WS_OK;
}

}  // namespace



extern "C" {

const char* ws_status_string(ws_status s) {
    switch (s) {
        case WS_OK: return "ok";
        case WS_ERR_INVALID: return "invalid argument";
        case WS_ERR_NONFINITE: return "non-finite input value";
        case WS_ERR_CUDA: return "CUDA runtime error";
        case WS_ERR_NOMEM: return "device allocation failed";
        case WS_ERR_TIMEOUT: return "device-side wait gave up";
        case WS_ERR_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

ws_status ws_ctx_create(ws_ctx** ctx, int device) {
    if (!ctx) return WS_ERR_INVALID;
    *ctx = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) { cudaGetLastError(); return WS_ERR_INVALID; }
    if (cudaSetDevice(device) != cudaSuccess) return WS_ERR_CUDA;
    ws_ctx* c = new (std::nothrow) ws_ctx();
    if (!c) return WS_ERR_NOMEM;
    c->device = device;
    if (cudaMalloc(&c->status, sizeof(uint32_t)) != cudaSuccess) { delete c; cudaGetLastError(); return WS_ERR_NOMEM; }
    if (cudaMemset(c->status, 0, sizeof(uint32_t)) != cudaSuccess) { cudaFree(c->status); delete c; return WS_ERR_CUDA; }
    *ctx = c;
    return WS_OK;
}

void ws_ctx_destroy(ws_ctx* ctx) {
    if (!ctx) return;
    if (ctx->prof.ev) {
        for (int i = 0; i < 2 * ctx->prof.cap; ++i) cudaEventDestroy(ctx->prof.ev[i]);
        delete[] ctx->prof.ev;
        delete[] ctx->prof.kind;
    }
    for (auto& c : ctx->cache) ws_plan_destroy(c.plan);
    ctx->cache.clear();
    if (ctx->status) cudaFree(ctx->status);
    delete ctx;
}

ws_status ws_plan_create(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg, ws_dtype dtype) {
    return plan_create_impl(ctx, plan, offsets, n_seg, dtype, false);
}

void ws_plan_destroy(ws_plan* plan) {
    if (!plan) return;
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    if (plan->side) cudaStreamDestroy(plan->side);
    for (void* a : plan->allocs) cudaFree(a);
    delete plan;
}

// Epilogue constants (all-off when epi is null); WS_ERR_INVALID on bad values.
static ws_status make_epi(const ws_l1_rewind* epi, WsEpi* ep) {
    ep->on = 0; ep->beta = 0.0; ep->gamma = 1.0; ep->beta_f = 0.0f; ep->gamma_f = 1.0f;
    if (!epi) return WS_OK;
    const double big = 1.7976931348623157e308;
    if (!(epi->beta >= 0.0) || !(epi->beta <= big) || !(epi->rho >= 0.0) || !(epi->rho <= 1.0) ||
        !(epi->v_scale >= 0.0) || !(epi->v_scale <= big))
        return WS_ERR_INVALID;
    ep->on = 1;
    ep->beta = epi->beta;
    ep->gamma = epi->v_scale * (1.0 - epi->rho);
    ep->beta_f = (float)ep->beta;
    ep->gamma_f = (float)ep->gamma;
    return WS_OK;
}

static ws_status batched_impl(ws_plan* plan, const void* values, const double* lambdas, const ws_l1_rewind* epi, void* out,
                       int32_t* cluster_ids, int64_t* n_clusters, ws_prec prec, void* stream,
                       const int32_t* ids_prev = nullptr) {
    if (!plan || (prec != WS_PREC_FP32_COMP && prec != WS_PREC_FP64)) return WS_ERR_INVALID;
    if (plan->n > 0 && (!values || !out)) return WS_ERR_INVALID;
    if (plan->n_seg > 0 && !lambdas) return WS_ERR_INVALID;
    WsEpi ep;
    if (make_epi(epi, &ep) != WS_OK) return WS_ERR_INVALID;
    if (plan->n_seg == 0) return WS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return plan->dtype == WS_F64
               ? run_forward<double>(plan, values, lambdas, out, cluster_ids, n_clusters, prec, ep, st, ids_prev)
               : run_forward<float>(plan, values, lambdas, out, cluster_ids, n_clusters, prec, ep, st, ids_prev);
}

static ws_status single_impl(ws_ctx* ctx, const void* w, int64_t d, double lambda, const ws_l1_rewind* epi, void* out,
                      int32_t* cluster_ids, int64_t* n_clusters, ws_dtype dtype, ws_prec prec, void* stream) {
    if (!ctx || d < 0 || !(lambda >= 0.0) || !(lambda <= 1.7976931348623157e308)) return WS_ERR_INVALID;
    if (dtype != WS_F32 && dtype != WS_F64) return WS_ERR_INVALID;
    if (d > 0 && (!w || !out)) return WS_ERR_INVALID;
    if (d >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    WsEpi ep;
    if (make_epi(epi, &ep) != WS_OK) return WS_ERR_INVALID;
    ws_status st;
    ws_plan* p = cached_plan(ctx, d, dtype, &st);
    if (!p) return st;
    cudaStream_t s = (cudaStream_t)stream;
    WS_LAUNCH(&ctx->prof, WSK_MISC, s, (k_set_lambda<<<1, 1, 0, s>>>(p->d_lambda1, lambda)));
    if (cudaGetLastError() != cudaSuccess) return WS_ERR_CUDA;
    return batched_impl(p, w, p->d_lambda1, epi, out, cluster_ids, n_clusters, prec, stream);
}

ws_status ws_prox_batched(ws_plan* plan, const void* values, const double* lambdas, void* out, int32_t* cluster_ids,
                          int64_t* n_clusters, ws_prec prec, void* stream) {
    return batched_impl(plan, values, lambdas, nullptr, out, cluster_ids, n_clusters, prec, stream);
}

ws_status ws_prox_batched_warm(ws_plan* plan, const void* values, const double* lambdas, const int32_t* ids_prev,
                               void* out, int32_t* cluster_ids, int64_t* n_clusters, ws_prec prec, void* stream) {
    if (plan && plan->n > 0 && !ids_prev) return WS_ERR_INVALID;
    return batched_impl(plan, values, lambdas, nullptr, out, cluster_ids, n_clusters, prec, stream, ids_prev);
}

ws_status ws_prox_batched_l1(ws_plan* plan, const void* values, const double* lambdas, const ws_l1_rewind* epi,
                             void* out, int32_t* cluster_ids, int64_t* n_clusters, ws_prec prec, void* stream) {
    if (!epi) return WS_ERR_INVALID;
    return batched_impl(plan, values, lambdas, epi, out, cluster_ids, n_clusters, prec, stream);
}

ws_status ws_prox(ws_ctx* ctx, const void* w, int64_t d, double lambda, void* out, int32_t* cluster_ids,
                  int64_t* n_clusters, ws_dtype dtype, ws_prec prec, void* stream) {
    return single_impl(ctx, w, d, lambda, nullptr, out, cluster_ids, n_clusters, dtype, prec, stream);
}

ws_status ws_prox_l1(ws_ctx* ctx, const void* w, int64_t d, double lambda, const ws_l1_rewind* epi, void* out,
                     int32_t* cluster_ids, int64_t* n_clusters, ws_dtype dtype, ws_prec prec, void* stream) {
    if (!epi) return WS_ERR_INVALID;
    return single_impl(ctx, w, d, lambda, epi, out, cluster_ids, n_clusters, dtype, prec, stream);
}

ws_status ws_prox_backward_batched(ws_plan* plan, const void* grad_out, const int32_t* cluster_ids, void* grad_in,
                                   void* stream) {
    if (!plan) return WS_ERR_INVALID;
    if (plan->n > 0 && (!grad_out || !cluster_ids || !grad_in)) return WS_ERR_INVALID;
    if (plan->n_seg == 0) return WS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return plan->dtype == WS_F64 ? run_backward<double>(plan, grad_out, cluster_ids, grad_in, st)
                                 : run_backward<float>(plan, grad_out, cluster_ids, grad_in, st);
}

ws_status ws_prox_backward(ws_ctx* ctx, const void* grad_out, const int32_t* cluster_ids, int64_t d, void* grad_in,
                           ws_dtype dtype, void* stream) {
    if (!ctx || d < 0 || (dtype != WS_F32 && dtype != WS_F64)) return WS_ERR_INVALID;
    if (d >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    ws_status st;
    ws_plan* p = cached_plan(ctx, d, dtype, &st);
    if (!p) return st;
    return ws_prox_backward_batched(p, grad_out, cluster_ids, grad_in, stream);
}

ws_status ws_prox_dlambda_batched(ws_plan* plan, const void* grad_out, const int32_t* cluster_ids,
                                  double* grad_lambda, void* stream) {
    if (!plan || !grad_lambda) return WS_ERR_INVALID;
    if (plan->n > 0 && (!grad_out || !cluster_ids)) return WS_ERR_INVALID;
    if (plan->n_keys + plan->n_lseg >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    if (plan->n_seg == 0) return WS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (plan->dtype == WS_F64) {
        LargeWork<double> W = make_work<double>(plan);
        e = ws_dlambda<double>((const double*)grad_out, cluster_ids, plan->d_offsets, plan->d_small, plan->n_small,
                               plan->n_seg, W, grad_lambda, plan->ctx->status, plan->stat_partial, st);
    } else {
        LargeWork<float> W = make_work<float>(plan);
        e = ws_dlambda<float>((const float*)grad_out, cluster_ids, plan->d_offsets, plan->d_small, plan->n_small,
                              plan->n_seg, W, grad_lambda, plan->ctx->status, plan->stat_partial, st);
    }
    return map_cuda(e);
}

ws_status ws_prox_dlambda(ws_ctx* ctx, const void* grad_out, const int32_t* cluster_ids, int64_t d,
                          double* grad_lambda, ws_dtype dtype, void* stream) {
    if (!ctx || d < 0 || (dtype != WS_F32 && dtype != WS_F64)) return WS_ERR_INVALID;
    if (d >= ((int64_t)1 << 31)) return WS_ERR_INVALID;
    ws_status st;
    ws_plan* p = cached_plan(ctx, d, dtype, &st);
    if (!p) return st;
    return ws_prox_dlambda_batched(p, grad_out, cluster_ids, grad_lambda, stream);
}

ws_status ws_plan_autotune(ws_ctx* ctx, ws_plan** plan, const int64_t* offsets, int64_t n_seg, ws_dtype dtype,
                           const void* values, const double* lambdas, void* out, int32_t* cluster_ids, ws_prec prec,
                           const int64_t* thresholds, int n_cand, int reps, int64_t* chosen, double* times_ms,
                           void* stream) {
    static const int64_t kDefault[] = {0, 512, 1024, 2048, 4096};
    if (!ctx || !plan || reps < 1) return WS_ERR_INVALID;
    if (!thresholds) { thresholds = kDefault; n_cand = 5; }
    if (n_cand < 1) return WS_ERR_INVALID;
    *plan = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) { cudaGetLastError(); return WS_ERR_CUDA; }
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); cudaGetLastError(); return WS_ERR_CUDA; }
    ws_plan* best = nullptr;
    float best_ms = 0.0f;
    int64_t best_t = -1;
    ws_status rc = WS_OK;
    for (int c = 0; c < n_cand && rc == WS_OK; ++c) {
        if (thresholds[c] < 0) { rc = WS_ERR_INVALID; break; }
        ws_plan* p = nullptr;
        rc = plan_create_impl(ctx, &p, offsets, n_seg, dtype, false, thresholds[c]);
        if (rc) break;
        rc = ws_prox_batched(p, values, lambdas, out, cluster_ids, nullptr, prec, stream);   // warm-up
        float ms = 0.0f;
        if (rc == WS_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = WS_ERR_CUDA;
        for (int r = 0; r < reps && rc == WS_OK; ++r)
            rc = ws_prox_batched(p, values, lambdas, out, cluster_ids, nullptr, prec, stream);
        if (rc == WS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = WS_ERR_CUDA;
        if (rc) { ws_plan_destroy(p); break; }
        ms /= (float)reps;
        if (times_ms) times_ms[c] = ms;
        if (!best || ms < best_ms) {
            if (best) ws_plan_destroy(best);
            best = p; best_ms = ms; best_t = p->small_max;
        } else {
            ws_plan_destroy(p);
        }
    }
    // second stage: the round cap of the Imminent Collisions rounds, on the
    // chosen plan (a runtime parameter of the tile and one-CTA kernels)
    static const int kCaps[] = {8, 16, 32, 64};
    if (rc == WS_OK && best) {
        int best_cap = -1;
        float cap_ms = best_ms;
        for (int c = 0; c < 4 && rc == WS_OK; ++c) {
            best->ic_cap = kCaps[c];
            rc = ws_prox_batched(best, values, lambdas, out, cluster_ids, nullptr, prec, stream);   // warm-up
            float ms = 0.0f;
            if (rc == WS_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = WS_ERR_CUDA;
            for (int r = 0; r < reps && rc == WS_OK; ++r)
                rc = ws_prox_batched(best, values, lambdas, out, cluster_ids, nullptr, prec, stream);
            if (rc == WS_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = WS_ERR_CUDA;
            ms /= (float)reps;
            if (rc == WS_OK && ms < cap_ms) { cap_ms = ms; best_cap = kCaps[c]; }
        }
        best->ic_cap = best_cap;   // -1: the context's cap was at least as fast
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) { cudaGetLastError(); if (best) ws_plan_destroy(best); return rc; }
    *plan = best;
    if (chosen) *chosen = best_t;
    return WS_OK;
}

ws_status ws_plan_params(const ws_plan* plan, int64_t* small_max, int* ic_cap) {
    if (!plan) return WS_ERR_INVALID;
    if (small_max) *small_max = plan->small_max;
    if (ic_cap) *ic_cap = plan->ic_cap >= 0 ? plan->ic_cap : plan->ctx->ic_cap;
    return WS_OK;
}

ws_status ws_R(ws_ctx* ctx, const void* w, int64_t d, ws_dtype dtype, double* R_out, double* metric_out,
               void* stream) {
    if (!ctx || d < 0 || (dtype != WS_F32 && dtype != WS_F64)) return WS_ERR_INVALID;
    if (d >= ((int64_t)1 << 31) || (d > 0 && !w)) return WS_ERR_INVALID;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return WS_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (d <= 1) {
        e = dtype == WS_F64 ? ws_tiny_R<double>((const double*)w, d, R_out, metric_out, &ctx->prof, st)
                            : ws_tiny_R<float>((const float*)w, d, R_out, metric_out, &ctx->prof, st);
        return map_cuda(e);
    }
    ws_status s;
    ws_plan* p = cached_plan(ctx, d, dtype, &s, 1);
    if (!p) return s;
    if (dtype == WS_F64) {
        LargeWork<double> W = make_work<double>(p);
        e = ws_large_R<double>(W, (const double*)w, R_out, metric_out, ctx->status, ctx->spin_limit, p->stat_partial,
                               st);
    } else {
        LargeWork<float> W = make_work<float>(p);
        e = ws_large_R<float>(W, (const float*)w, R_out, metric_out, ctx->status, ctx->spin_limit, p->stat_partial,
                              st);
    }
    return map_cuda(e);
}

ws_status ws_get_status(ws_ctx* ctx, void* stream) {
    if (!ctx) return WS_ERR_INVALID;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) { cudaGetLastError(); return WS_ERR_CUDA; }
    uint32_t h = 0;
    if (cudaMemcpy(&h, ctx->status, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return WS_ERR_CUDA;
    if (h && cudaMemset(ctx->status, 0, sizeof(uint32_t)) != cudaSuccess) return WS_ERR_CUDA;
    if (h & WS_STATUS_INEXACT) ctx->inexact = true;   // (information for ws_get_inexact)
    if (h & WS_STATUS_NONFINITE) return WS_ERR_NONFINITE;
    if (h & WS_STATUS_BAD_LAMBDA) return WS_ERR_INVALID;
    if (h & WS_STATUS_TIMEOUT) return WS_ERR_TIMEOUT;
    if (h & WS_STATUS_INTERNAL) return WS_ERR_INTERNAL;
    return WS_OK;
}

ws_status ws_get_inexact(ws_ctx* ctx, int* inexact, void* stream) {
    if (!ctx || !inexact) return WS_ERR_INVALID;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) { cudaGetLastError(); return WS_ERR_CUDA; }
    uint32_t h = 0;
    if (cudaMemcpy(&h, ctx->status, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return WS_ERR_CUDA;
    if (h & WS_STATUS_INEXACT) {   // clear the bit, keep the error bits for ws_get_status
        const uint32_t rest = h & ~(uint32_t)WS_STATUS_INEXACT;
        if (cudaMemcpy(ctx->status, &rest, sizeof rest, cudaMemcpyHostToDevice) != cudaSuccess) return WS_ERR_CUDA;
    }
    *inexact = ((h & WS_STATUS_INEXACT) || ctx->inexact) ? 1 : 0;
    ctx->inexact = false;
    return WS_OK;
}

void ws_debug_set_spin_limit(ws_ctx* ctx, int64_t limit) {
    if (ctx) ctx->spin_limit = limit > 0 ? (uint64_t)limit : WS_DEFAULT_SPIN;
}

void ws_debug_set_ic_cap(ws_ctx* ctx, int cap) {
    if (!ctx) return;
    ctx->ic_cap = cap < 0 ? 32 : cap;
}

ws_status ws_debug_hull_stats(ws_ctx* ctx, int64_t d, ws_dtype dtype, int64_t* counts, int n_counts) {
    if (!ctx || !counts || n_counts < 3 || d < 0) return WS_ERR_INVALID;
    ws_plan* p = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        for (auto& c : ctx->cache)
            if (c.d == d && c.dtype == dtype && c.sort_only == 0) p = c.plan;
    }
    for (int i = 0; i < n_counts; ++i) counts[i] = 0;
    if (!p || p->n_hull_tiles == 0) return WS_OK;
    std::vector<int32_t> r((size_t)p->n_hull_tiles);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(r.data(), p->tile_rounds, sizeof(int32_t) * r.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return WS_ERR_CUDA;
    }
    for (int32_t v : r) {
        if (v == -2) ++counts[0];
        else if (v == -1) ++counts[1];
        else ++counts[v + 1 < n_counts ? v + 1 : n_counts - 1];
    }
    return WS_OK;
}

void ws_debug_set_small_max(ws_ctx* ctx, int64_t small_max) {
    if (!ctx) return;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->small_max_override = small_max;
    for (auto& c : ctx->cache) ws_plan_destroy(c.plan);
    ctx->cache.clear();
}

ws_status ws_debug_sort(ws_plan* plan, const void* values, void* sorted_out, void* stream) {
    if (!plan || (plan->n > 0 && (!values || !sorted_out))) return WS_ERR_INVALID;
    if (plan->n_lseg == 0) return WS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (plan->dtype == WS_F64) {
        LargeWork<double> W = make_work<double>(plan);
        uint64_t* sorted = nullptr;
        e = ws_large_sort<double>(W, (const double*)values, plan->ctx->status, plan->ctx->spin_limit, st, &sorted);
        if (!e) e = ws_large_copy_sorted<double>(W, sorted, (double*)sorted_out, st);
    } else {
        LargeWork<float> W = make_work<float>(plan);
        uint32_t* sorted = nullptr;
        e = ws_large_sort<float>(W, (const float*)values, plan->ctx->status, plan->ctx->spin_limit, st, &sorted);
        if (!e) e = ws_large_copy_sorted<float>(W, sorted, (float*)sorted_out, st);
    }
    return map_cuda(e);
}

static const char* const kKernelNames[WSK_COUNT] = {"small", "hist", "hist_scan", "onesweep", "tile_hull",
                                                     "root", "table", "big_gaps", "lookup", "backward", "misc",
                                                     "tile_general", "junction", "climb"};

const char* ws_debug_kernel_name(int kind) {
    return (kind >= 0 && kind < WSK_COUNT) ? kKernelNames[kind] : nullptr;
}

ws_status ws_debug_profile(ws_ctx* ctx, int enable) {
    if (!ctx) return WS_ERR_INVALID;
    WsProf& P = ctx->prof;
    if (enable && !P.ev) {
        P.cap = 1 << 14;
        P.ev = new (std::nothrow) cudaEvent_t[2 * P.cap];
        P.kind = new (std::nothrow) int[P.cap];
        if (!P.ev || !P.kind) return WS_ERR_NOMEM;
        for (int i = 0; i < 2 * P.cap; ++i)
            if (cudaEventCreate(&P.ev[i]) != cudaSuccess) return WS_ERR_CUDA;
    }
    P.enabled = enable != 0;
    P.n = 0;
    for (int k = 0; k < WSK_COUNT; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_cnt[k] = 0; }
    return WS_OK;
}

ws_status ws_debug_profile_read(ws_ctx* ctx, int kind, double* total_ms, int64_t* count) {
    if (!ctx || kind < 0 || kind >= WSK_COUNT) return WS_ERR_INVALID;
    WsProf& P = ctx->prof;
    if (P.n > 0) {   // fold the recorded event pairs into the per-kind totals
        if (cudaEventSynchronize(P.ev[2 * P.n - 1]) != cudaSuccess) return WS_ERR_CUDA;
        for (int i = 0; i < P.n; ++i) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]) != cudaSuccess) return WS_ERR_CUDA;
            ctx->prof_ms[P.kind[i]] += ms;
            ctx->prof_cnt[P.kind[i]] += 1;
        }
        P.n = 0;
    }
    if (total_ms) *total_ms = ctx->prof_ms[kind];
    if (count) *count = ctx->prof_cnt[kind];
    return WS_OK;
}

int64_t ws_debug_launch_count(ws_ctx* ctx) { return ctx ? (int64_t)ctx->prof.launches : 0; }

}  // extern "C"
