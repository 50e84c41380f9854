// ann_internal.cuh -- shared declarations of libann's host code and kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ann.h"

namespace ann {

// Packed queue / candidate entry: (order-preserving key bits << 32) | id,
// with bit 31 of the id word holding the "checked" flag of Algorithm 1. Two
// entries compare in (key, id) order once the flag is masked off.
typedef unsigned long long entry_t;
static constexpr entry_t kChecked = 1ull << 31;
static constexpr entry_t kMask = ~kChecked;
static constexpr entry_t kEmptyEntry = ~0ull;
static constexpr uint32_t kEmptySlot = 0xFFFFFFFFu;

struct IndexData {
    int device = 0;
    int64_t n = 0;
    int32_t d = 0, d_pad = 0, R = 0;
    int32_t storage = ANN_STORE_F32, metric = ANN_METRIC_L2;
    int64_t entry = 0;
    void *base = nullptr;       // n x d_pad, storage type, zero padded
    float *scales = nullptr;    // n, E4M3 only
    float *base32 = nullptr;    // n x d_pad32 FP32 rows for re-rank (aliases base for F32)
    int32_t d_pad32 = 0;
    int32_t *adj = nullptr;     // n x R
    bool owns_base32 = false;
    int64_t device_bytes = 0;
    // staging for ann_search_host
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // neighbour groups (Sec. 4.4): base (and scales) hold n_hot * R more rows after the n vertices' rows,
    // the neighbours of each hot vertex in adjacency order; hot_slot[v] = v's group or -1
    int32_t *hot_slot = nullptr;
    int64_t n_hot = 0;
    int32_t group_prefetch = 0;  // 0 = one bulk prefetch of a hot vertex's block; 1 = the fresh rows only
    // device work counters of persistent grids: one slot (its own 128-byte line) per stream that
    // searches the index, so persistent searches on different streams never share a counter
    int *work_counter = nullptr;
};

static constexpr int kCounterSlots = 1024;
static constexpr int kCounterStride = 32;  // ints between slots (one 128-byte line each)

// Byte offsets of the dynamic shared-memory segments (16-byte aligned).
struct SmemLayout {
    int q_off, q0_off, q1_off, cand_off, cand2_off, dup_off, hash_off, act_off, total;
};

__host__ __device__ inline int align16(int x) { return (x + 15) & ~15; }

// Shared memory of the one-CTA sync kernel with nw warps. The cand segment
// holds each warp's fresh (id, row) pairs during a step (nw * ceil(Mcap * R /
// nw) of them, one per 8-byte entry; the host makes Ccap at least that) and
// sort output after it; act holds the step's selected vertices and their
// queue positions.
__host__ __device__ inline SmemLayout sync_layout(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap,
                                                  int slot_bytes, int nw) {
    SmemLayout s;
    int o = 0;
    s.q_off = o;    o += align16(qfloats * 4);
    s.q0_off = o;   o += align16(Lcap * 8);
    s.q1_off = o;   o += align16(Lcap * 8);
    s.cand_off = o; o += align16(Ccap * 8);
    s.cand2_off = o; o += align16(Ccap * 8);
    s.dup_off = o;  o += align16(Ccap);
    s.hash_off = o; o += align16((1 << hash_bits) * slot_bytes);
    s.act_off = o;  o += align16(2 * Mcap * 4);
    s.total = o;
    return s;
}

// Everything a search launch needs, passed by value.
struct SearchArgs {
    const void *base;
    const float *scales;
    const float *base32;
    const int32_t *adj;
    int64_t n;
    int32_t d, d_pad, d_pad32, R;
    int64_t entry;
    int32_t metric;
    const float *queries;
    int64_t nq;
    int32_t k, L, M;  // maxima (uniform values when no per-query arrays)
    const int32_t *k_arr, *L_arr, *M_arr;
    int32_t M0, t;
    float R_ratio;
    int32_t merge_rule;    // async: 0 = Algorithm 2; 1 = stall count against `patience`
    float patience;
    int32_t rerank;
    int32_t hash_bits;
    int32_t visited_mode;  // 0 = open addressing, reset when half full; 1 = direct-mapped, forgets on collision
    int32_t slot_bytes;    // direct-mapped slot: 4 = a full id; 1 or 2 = a tag (the hashed id's bits below the index)
    int32_t tag_bits;      // bits of the tag when slot_bytes < 4 or ways > 0
    int32_t ways;          // set-associative cache: tags per 32-bit set word (2 or 3); 0 = another form
    int32_t l2_prefetch;   // 1 = L2 prefetch of each candidate row once it passes the visited filter
    const int32_t *hot_slot; // neighbour groups: n entries, the group of a hot vertex or -1 (nullptr: none)
    int32_t group_prefetch;  // 0 = one bulk prefetch per hot vertex's block; 1 = the fresh rows only
    int32_t block_gather;    // one-CTA sync kernel: 1 = the CTA's fresh rows in one list gathered by all warps
    int32_t team_lanes;    // distance gather: log2 of the lanes that share one candidate row
    int32_t team_lanes32;  // the same for the FP32 rows of the re-rank
    int64_t *out_ids;
    float *out_dists;
    ann_query_stats *stats;
    int *work_counter;
    int32_t persistent;
    const int32_t *order;  // work list: item i is query order[i] (nullptr: item i is query i)
    long long *phase_cycles; // nq x 4 SM cycles per phase (select, expand, distance, sort+merge) or nullptr
    // shared-memory layout
    int32_t Lcap;        // queue capacity
    int32_t Ccap;        // candidate / sort buffer, power of two >= 32
    int32_t qfloats;     // query buffer length
    SmemLayout sync_lay; // one-CTA sync kernel: segment offsets (kernel parameters, so no register holds them)
};

inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

inline int storage_bytes(int storage) {
    switch (storage) {
        case ANN_STORE_F32: return 4;
        case ANN_STORE_BF16: return 2;
        case ANN_STORE_F16: return 2;
        case ANN_STORE_E4M3: return 1;
    }
    return 0;
}

// kernels/launchers (search_sync.cu)
cudaError_t launch_sync_search(const SearchArgs &a, int storage, int threads, int smem_bytes,
                               int grid, cudaStream_t stream);
cudaError_t sync_search_occupancy(int storage, int metric, int threads, int smem_bytes, int *blocks_per_sm);

// search_async.cu
cudaError_t launch_async_search(const SearchArgs &a, int storage, int threads, int smem_bytes, int grid,
                                cudaStream_t stream);
cudaError_t async_search_occupancy(int storage, int threads, int smem_bytes, int *blocks_per_sm);
int async_smem_size(int qfloats, int Lcap, int walkers, int hash_bits);

// ann_api.cu: sets the calling thread's ann_last_error() text
void set_error(const char *msg);

// ann_api.cu: raise a kernel's dynamic shared-memory limit to at least smem
// bytes on the current device; the attribute is set only when a launch needs
// more than any earlier one (the call costs microseconds on a latency path).
cudaError_t ensure_dyn_smem(const void *kernel, int smem);

// ann_api.cu: argument checks and launch configuration of one search
struct Plan {
    SearchArgs a;
    int threads;
    int smem;
    int grid;
    int mode;
    int storage;
    int cluster;  // CTAs per query (1 = no cluster)
};
int plan_search(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L, int32_t M,
                int64_t *out_ids, float *out_dists, const ann_search_params *p, Plan *plan);
cudaError_t launch(const Plan &plan, cudaStream_t s);
int index_device(const ann_index *index);

// search_cluster.cu
cudaError_t launch_cluster_search(const SearchArgs &a, int storage, int threads, int smem_bytes, int cluster,
                                  cudaStream_t stream);
int cluster_smem_size(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap);

// encode.cu
cudaError_t launch_encode(const float *src, int64_t n, int32_t d, int storage, void *dst, int32_t d_pad,
                          float *scales, cudaStream_t stream);
cudaError_t launch_count_bad_adj(const int32_t *adj, int64_t count, int64_t n, unsigned long long *bad,
                                 cudaStream_t stream);
cudaError_t launch_count_in_degree(const int32_t *adj, int64_t count, int32_t *deg, cudaStream_t stream);

// knn.cu: brute-force k-NN over BF16 rows (graph construction). norms holds
// knn_norms_rows(n) floats for l2 (unused for inner product); err is a
// device int set to 1 if a CTA's merge rounds ran out.
int64_t knn_norms_rows(int64_t n);
cudaError_t launch_knn_bf16(const void *base, int64_t n, int d, const void *queries, int64_t nq, int64_t self0,
                            int metric, int k, int32_t *ids, float *dists, float *norms, int *err,
                            cudaStream_t stream);
cudaError_t launch_fill_groups(unsigned char *rows, float *scales, const int32_t *adj, const int32_t *hot,
                               int64_t n_hot, int32_t R, int64_t n, int32_t row_bytes, cudaStream_t stream);

}  // namespace ann
