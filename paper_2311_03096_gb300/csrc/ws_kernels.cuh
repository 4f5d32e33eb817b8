// ws_kernels.cuh -- launch interface between the C ABI (ws_api.cu) and the
// kernels.  Internal; not installed.
#pragma once
#include "ws_block.cuh"

template <typename T> struct SmallCfg;
template <> struct SmallCfg<float> { static constexpr int M = 16; static constexpr int CAP = 256 * 16; };
template <> struct SmallCfg<double> { static constexpr int M = 16; static constexpr int CAP = 256 * 16; };

// Opt-in per-launch timing (CUDA events recorded on the launching stream
// around every kernel) and a launch counter.  Host-side only.
enum WsKernelKind {
    WSK_SMALL = 0, WSK_HIST, WSK_HIST_SCAN, WSK_ONESWEEP, WSK_TILE_HULL, WSK_ROOT,
    WSK_TABLE, WSK_BIG_GAPS, WSK_LOOKUP, WSK_BWD, WSK_MISC, WSK_TILE_GENERAL, WSK_JUNCTION, WSK_CLIMB, WSK_COUNT
};
struct WsProf {
    bool enabled = false;
    int cap = 0, n = 0;
    cudaEvent_t* ev = nullptr;   // 2 * cap events
    int* kind = nullptr;         // cap
    long long launches = 0;
    void begin(cudaStream_t st, int k) {
        ++launches;
        if (!enabled || n >= cap) return;
        cudaEventRecord(ev[2 * n], st);
        kind[n] = k;
    }
    void end(cudaStream_t st) {
        if (!enabled || n >= cap) return;
        cudaEventRecord(ev[2 * n + 1], st);
        ++n;
    }
};
#define WS_LAUNCH(PROF, KIND, ST, ...) \
    do { (PROF)->begin((ST), (KIND)); __VA_ARGS__; (PROF)->end((ST)); } while (0)

// Large-path tile geometry.
constexpr int WS_SORT_NT = 512;              // threads per onesweep CTA
constexpr int WS_SORT_ITEMS = 12;            // keys per thread (a multiple of 4: 16-byte loads in k_hist)
constexpr int WS_SORT_CHAINS = 1;            // independent ranking chains per warp
constexpr int WS_SORT_TILE = WS_SORT_NT * WS_SORT_ITEMS;   // 6144 keys per sort tile
constexpr int WS_HULL_NT = 256;              // threads per hull-tile CTA
constexpr int WS_HULL_M = 16;                // points per thread chunk
constexpr int WS_HULL_TILE = WS_HULL_NT * WS_HULL_M;       // 4096 elements per hull tile
constexpr int WS_MAX_LEVELS = 32;           // merge-tree levels (segments < 2^31 elements)

// One tile of a large segment (sort tiles and hull tiles use the same record).
struct TileDesc {
    int64_t kpos;      // first element in the compact key buffer
    int64_t vpos;      // first element in the caller's value array
    int32_t len;       // elements in the tile
    int32_t lseg;      // large-segment index
    int32_t first;     // global index of the segment's first tile (of this kind)
    int32_t tin;       // index of the tile inside its segment
};

// One large segment.
struct LargeSeg {
    int64_t vpos;      // first element in the caller's arrays
    int64_t kpos;      // first element in the compact key buffer
    int64_t len;
    int32_t seg;       // index in the caller's segment list
    int32_t sort_first, sort_count;   // sort tiles
    int32_t hull_first, hull_count;   // hull tiles
    int64_t dir_pos;   // directory slice start
    int32_t dir_cap_log2;             // directory slice holds 2^dir_cap_log2 + 1 entries
    int32_t pad;
};

// A piece of a node hull: vertices [lo, hi) of hull tile `tile`; cum = rank of
// its first vertex within the node hull; off = fixed-point prefix X at the
// tile's first point, relative to the node's first point.
struct __align__(16) Piece {
    int32_t tile;
    uint16_t lo, hi;
    int32_t cum;
    int32_t pad;
    i128 off;
};

// Cluster table entry (sorted by key within a segment).
template <typename T> struct CEntry;
template <> struct CEntry<float> { uint32_t key; float val; };
template <> struct CEntry<double> { uint64_t key; double val; };

// Directory entry: first cluster whose start falls in the bucket (or in a
// later one) and the top 32 bits of that cluster's start key.
struct DirEntry {
    int32_t idx;
    uint32_t key32;
};
constexpr int WS_DIR_MAX_LOG2 = 22;   // <= 2^22 buckets per segment (32 MiB: stays in L2)

// Constants of the exact hull test at one fixed-point unit scale of a
// segment: the units of a one-binade hull tile (ulps of its binade) or the
// segment's own scale.  Computed once per segment (k_scales) so that tiles do
// no FP64 or wide-integer set-up work.
struct TileScale {
    SegConst sc;      // hull-test constants at this scale
    float muq;        // lambda 2^L / (d - 1) in units, for the FP32 filter
    int fast;         // muq usable by the filter
    uint64_t modd;    // odd part of lambda 2^L (0 when lambda = 0) and its exponent
    int sodd;
    int pad;
    int64_t t11;      // floor(2 lambda 2^L / (d - 1)), saturated at 2^62: two adjacent
                      // elements collide at once (IC round 1) iff their gap <= t11 units
};
constexpr int WS_NSCALE = 64;   // per segment: binade shifts 0 .. FIX_OFS, then the segment scale last

// Per-segment run-time values computed on the device.
struct SegRuntime {
    int64_t n_clusters;
    int64_t table_pos;  // first cluster-table entry of the segment
    int32_t emax;
    int32_t dir_log2;   // directory holds 2^dir_log2 buckets (+1 sentinel)
    float lo, scale;    // bucket map: floor((x - lo) * scale)
};

template <typename T>
cudaError_t ws_launch_small(const T* values, const int64_t* offsets, const int32_t* seg_list, int n_list,
                            const double* lambdas, T* out, int32_t* ids, int64_t* n_clusters, int fp64,
                            const WsEpi& ep, uint32_t* status, cudaStream_t st, WsProf* prof, int32_t* gen_list,
                            int32_t* gen_count, int ic_cap, const int32_t* ids_prev);
template <typename T>
cudaError_t ws_launch_small_backward(const T* g, const int32_t* ids, const int64_t* offsets, const int32_t* seg_list,
                                     int n_list, T* gin, uint32_t* status, cudaStream_t st, WsProf* prof);

// Large path workspace pointers (all device).
template <typename T>
struct LargeWork {
    typedef typename KeyOf<T>::K K;
    int n_lseg, n_sort_tiles, n_hull_tiles;
    int64_t n_keys;
    const LargeSeg* lsegs;
    const TileDesc* sort_tiles;
    const TileDesc* hull_tiles;
    K* keys_a;
    K* keys_b;
    uint32_t* hist;          // [n_lseg][passes][256]
    uint64_t* lookback;      // [passes][n_sort_tiles][256]
    uint32_t* tile_counter;  // [passes]
    uint32_t* epoch;         // [1] look-back epoch, advanced by every sort
    int32_t* seg_emin;       // [n_lseg] smallest effective exponent of a nonzero value
    // hull
    uint16_t* vp;            // [n_hull_tiles][WS_HULL_TILE + 1] vertex points (tile-local)
    i128* vx;                // [n_hull_tiles][WS_HULL_TILE + 1] X at vertices (tile-local)
    int32_t* nvert;          // [n_hull_tiles]
    i128* tile_total;        // [n_hull_tiles] node total X, stored at the node's first tile
    int32_t* arrive;         // [WS_MAX_LEVELS][n_hull_tiles] merge-tree arrival counters
    Piece* pieces;           // [n_hull_tiles]
    int32_t* npieces;        // [n_hull_tiles] pieces of the node whose first tile is this index
    int32_t* tile_piece;     // [n_hull_tiles] piece index in the root list or -1
    int32_t* gen_list;       // [n_hull_tiles] tiles whose hull the general kernel builds
    int32_t* gen_count;      // [1] their number
    int32_t* keepR;          // [n_hull_tiles] junction results (ws_tile.cu)
    int32_t* keepL;          // [n_hull_tiles]
    int32_t* jflag0;         // [n_hull_tiles]
    int32_t* seg_mode;       // [n_lseg] 0: junctions resolved, 1: one cluster, 2: tree of merges
    i128* tile_base;         // [n_hull_tiles] X at every hull tile's first point (segment frame)
    TileScale* scales;       // [n_lseg][WS_NSCALE]
    int32_t* tile_rounds;    // [n_hull_tiles] in-tile IC rounds to converge, -1 chain + trees, -2 general kernel
    int ic_cap;              // in-tile IC round cap (0: chain + trees only)
    i128* seg_total;         // [n_lseg] X of the whole segment
    int32_t* seg_below;      // [n_lseg] a tile-hull vertex lies below the segment's chord
    SegRuntime* rt;          // [n_lseg]
    CEntry<T>* table;        // [n_keys + n_lseg]
    DirEntry* dir;           // directory slices
    // backward
    T* bsum;                 // [n_keys + n_lseg] cluster means
    int32_t* bcnt;           // [n_keys + n_lseg] cluster sizes
    unsigned long long* bacc;   // [n_keys + n_lseg][2] exact cluster sums (128-bit, low word first)
    int32_t* bwd_seg;        // [2 n_lseg] per segment: largest grad exponent, largest cluster id
    WsProf* prof;            // host-side launch accounting
};

template <typename T>
cudaError_t ws_large_sort(const LargeWork<T>& W, const T* values, uint32_t* status, uint64_t spin_limit,
                          cudaStream_t st, typename KeyOf<T>::K** sorted);
// Lean tile hulls and the junction resolution (ws_tile.cu).
template <typename T>
cudaError_t ws_large_hull_fast(const LargeWork<T>& W, const typename KeyOf<T>::K* sorted, const double* lambdas,
                               uint32_t* status, cudaStream_t st);
template <typename T>
cudaError_t ws_large_junctions(const LargeWork<T>& W, const double* lambdas, cudaStream_t st);
template <typename T>
cudaError_t ws_large_prox(const LargeWork<T>& W, const T* values, const double* lambdas, T* out, int32_t* ids,
                          int64_t* n_clusters, int fp64, const WsEpi& ep, uint32_t* status, uint64_t spin_limit,
                          int n_levels, cudaStream_t st);
template <typename T>
cudaError_t ws_large_backward(const LargeWork<T>& W, const T* g, const int32_t* ids, T* gin, uint32_t* status,
                              cudaStream_t st);
template <typename T>
cudaError_t ws_large_copy_sorted(const LargeWork<T>& W, const typename KeyOf<T>::K* sorted, T* dst, cudaStream_t st);
// R(w) and the weight-sharing measure per large segment (ws_stats.cu);
// `partial` holds ws_R_partial_bytes(n_sort_tiles) bytes of device scratch.
template <typename T>
cudaError_t ws_large_R(const LargeWork<T>& W, const T* values, double* R_out, double* metric_out, uint32_t* status,
                       uint64_t spin_limit, void* partial, cudaStream_t st);
size_t ws_R_partial_bytes(int n_sort_tiles);
template <typename T>
cudaError_t ws_tiny_R(const T* values, int64_t d, double* R_out, double* metric_out, WsProf* prof, cudaStream_t st);
// d <grad_out, out> / d lambda per segment, partition held fixed (ws_stats.cu);
// `partial` as for ws_large_R.
template <typename T>
cudaError_t ws_dlambda(const T* g, const int32_t* ids, const int64_t* d_offsets, const int32_t* d_small, int n_small,
                       int64_t n_seg, const LargeWork<T>& W, double* out, uint32_t* status, void* partial,
                       cudaStream_t st);
