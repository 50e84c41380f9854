// ann_api.cu -- host side of the C ABI declared in include/ann.h: argument
// checks, index memory, kernel selection and launch.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>
#include <algorithm>

#include "ann_internal.cuh"

struct ann_index {
    ann::IndexData d;
    // stream -> work-counter slot (see IndexData::work_counter)
    std::mutex slot_mu;
    std::unordered_map<std::string, int> slot_of;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ANN_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(ANN_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ANN_CUDA(call)                                         \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);    \
    } while (0)

void free_index_data(ann::IndexData &x) {
    cudaFree(x.base);
    cudaFree(x.scales);
    if (x.owns_base32) cudaFree(x.base32);
    cudaFree(x.adj);
    cudaFree(x.stage);
    cudaFree(x.work_counter);
    cudaFree(x.hot_slot);
    x = ann::IndexData();
}

// Device properties that a search plan reads, cached per device.
constexpr int kMaxDevices = 64;
std::atomic<int> g_sms[kMaxDevices], g_smem_optin[kMaxDevices];

int device_attr(std::atomic<int> *cache, cudaDeviceAttr attr) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) {
        int v = 0;
        cudaDeviceGetAttribute(&v, attr, dev);
        return v;
    }
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
        cudaDeviceGetAttribute(&v, attr, dev);
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

int sm_count() {
    const int sms = device_attr(g_sms, cudaDevAttrMultiProcessorCount);
    return sms > 0 ? sms : 1;
}

int max_dyn_smem() { return device_attr(g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin); }

int create_impl(const float *base, int64_t n, int32_t d, int32_t storage, const int32_t *adj, int32_t R,
                int64_t entry, int32_t metric, int32_t flags, ann_index **out) {
    if (!out) return fail(ANN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!base || !adj) return fail(ANN_ERR_ARG, "base and adj must not be NULL");
    if (n < 1 || n >= (1ll << 31) - 1) return fail(ANN_ERR_ARG, "n=%lld outside [1, 2^31-1)", (long long)n);
    if (d < 1 || d > 4096) return fail(ANN_ERR_ARG, "d=%d outside [1, 4096]", d);
    if (R < 1 || R > 256) return fail(ANN_ERR_ARG, "R=%d outside [1, 256]", R);
    if (entry < 0 || entry >= n) return fail(ANN_ERR_ARG, "entry=%lld outside [0, n)", (long long)entry);
    if (storage < ANN_STORE_F32 || storage > ANN_STORE_E4M3) return fail(ANN_ERR_ARG, "unknown storage %d", storage);
    if (metric != ANN_METRIC_L2 && metric != ANN_METRIC_IP) return fail(ANN_ERR_ARG, "unknown metric %d", metric);
    if (flags & ~(ANN_INDEX_DEVICE_INPUT | ANN_INDEX_KEEP_F32)) return fail(ANN_ERR_ARG, "unknown flags 0x%x", flags);
    const bool dev_in = flags & ANN_INDEX_DEVICE_INPUT;
    if (!dev_in) {
        for (int64_t i = 0; i < n * (int64_t)R; ++i)
            if (adj[i] < -1 || (int64_t)adj[i] >= n)
                return fail(ANN_ERR_ARG, "adj[%lld]=%d outside [-1, n)", (long long)i, adj[i]);
    }

    ann::IndexData x;
    cudaGetDevice(&x.device);
    x.n = n;
    x.d = d;
    x.R = R;
    x.storage = storage;
    x.metric = metric;
    x.entry = entry;
    const int es = ann::storage_bytes(storage);
    const int per16 = 16 / es;
    x.d_pad = (d + per16 - 1) / per16 * per16;
    x.d_pad32 = (d + 3) / 4 * 4;

    auto cleanup_fail = [&](int code) {
        free_index_data(x);
        return code;
    };
    cudaError_t e;
    const size_t base_bytes = (size_t)n * x.d_pad * es;
    if ((e = cudaMalloc(&x.base, base_bytes)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc(base)"));
    if ((e = cudaMalloc(&x.adj, (size_t)n * R * 4)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc(adj)"));
    if ((e = cudaMalloc(&x.work_counter, (size_t)ann::kCounterSlots * ann::kCounterStride * sizeof(int))) !=
        cudaSuccess)
        return cleanup_fail(cuda_fail(e, "cudaMalloc(counters)"));
    x.device_bytes = base_bytes + (size_t)n * R * 4;
    if (storage == ANN_STORE_E4M3) {
        if ((e = cudaMalloc(&x.scales, (size_t)n * 4)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc(scales)"));
        x.device_bytes += (size_t)n * 4;
    }
    const bool keep32 = storage != ANN_STORE_F32 && (flags & ANN_INDEX_KEEP_F32);
    if (keep32) {
        if ((e = cudaMalloc(&x.base32, (size_t)n * x.d_pad32 * 4)) != cudaSuccess)
            return cleanup_fail(cuda_fail(e, "cudaMalloc(base32)"));
        x.owns_base32 = true;
        x.device_bytes += (size_t)n * x.d_pad32 * 4;
    } else if (storage == ANN_STORE_F32) {
        x.base32 = reinterpret_cast<float *>(x.base);
    }

    // stage FP32 input on the device if it is on the host
    const float *src = base;
    float *tmp = nullptr;
    if (!dev_in) {
        if ((e = cudaMalloc(&tmp, (size_t)n * d * 4)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc(tmp)"));
        if ((e = cudaMemcpy(tmp, base, (size_t)n * d * 4, cudaMemcpyHostToDevice)) != cudaSuccess) {
            cudaFree(tmp);
            return cleanup_fail(cuda_fail(e, "cudaMemcpy(base)"));
        }
        src = tmp;
        if ((e = cudaMemcpy(x.adj, adj, (size_t)n * R * 4, cudaMemcpyHostToDevice)) != cudaSuccess) {
            cudaFree(tmp);
            return cleanup_fail(cuda_fail(e, "cudaMemcpy(adj)"));
        }
    } else {
        if ((e = cudaMemcpy(x.adj, adj, (size_t)n * R * 4, cudaMemcpyDeviceToDevice)) != cudaSuccess)
            return cleanup_fail(cuda_fail(e, "cudaMemcpy(adj)"));
        unsigned long long *bad = nullptr;
        if ((e = cudaMalloc(&bad, 8)) != cudaSuccess) return cleanup_fail(cuda_fail(e, "cudaMalloc(bad)"));
        unsigned long long hbad = 0;
        e = cudaMemset(bad, 0, 8);
        if (e == cudaSuccess) e = ann::launch_count_bad_adj(x.adj, n * (int64_t)R, n, bad, 0);
        if (e == cudaSuccess) e = cudaMemcpy(&hbad, bad, 8, cudaMemcpyDeviceToHost);
        cudaFree(bad);
        if (e != cudaSuccess) return cleanup_fail(cuda_fail(e, "adjacency check"));
        if (hbad) return cleanup_fail(fail(ANN_ERR_ARG, "%llu adjacency ids outside [-1, n)", hbad));
    }
    e = ann::launch_encode(src, n, d, storage, x.base, x.d_pad, x.scales, 0);
    if (e == cudaSuccess && keep32) e = ann::launch_encode(src, n, d, ANN_STORE_F32, x.base32, x.d_pad32, nullptr, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(tmp);
    if (e != cudaSuccess) return cleanup_fail(cuda_fail(e, "encode"));

    ann_index *ix = new (std::nothrow) ann_index;
    if (!ix) return cleanup_fail(fail(ANN_ERR_OOM, "host allocation"));
    ix->d = x;
    *out = ix;
    return ANN_OK;
}

}  // namespace

namespace ann {

int plan_search(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L, int32_t M,
                int64_t *out_ids, float *out_dists, const ann_search_params *p, Plan *plan) {
    if (!index) return fail(ANN_ERR_ARG, "index is NULL");
    const ann::IndexData &x = index->d;
    if (nq < 0 || nq > 0x7fffffffll) return fail(ANN_ERR_ARG, "nq=%lld outside [0, 2^31)", (long long)nq);
    if (nq > 0 && (!queries || !out_ids || !out_dists)) return fail(ANN_ERR_ARG, "queries/out pointers must not be NULL");
    if (L < 1 || L > 2048) return fail(ANN_ERR_ARG, "L=%d outside [1, 2048]", L);
    if (k < 1 || k > L) return fail(ANN_ERR_ARG, "k=%d outside [1, L=%d]", k, L);
    if (M < 1 || M > 64) return fail(ANN_ERR_ARG, "M=%d outside [1, 64]", M);
    ann_search_params def;
    memset(&def, 0, sizeof(def));
    if (!p) p = &def;
    if (p->mode != ANN_MODE_SYNC && p->mode != ANN_MODE_ASYNC) return fail(ANN_ERR_ARG, "unknown mode %d", p->mode);
    const bool async = p->mode == ANN_MODE_ASYNC;
    const int M0 = p->M0 ? p->M0 : 1;
    const int t = p->t ? p->t : 1;
    if (M0 < 1 || t < 1) return fail(ANN_ERR_ARG, "M0=%d and t=%d must be >= 1", M0, t);
    if (p->rerank && !x.base32) return fail(ANN_ERR_ARG, "rerank needs an FP32 copy (ANN_INDEX_KEEP_F32)");
    if (async && !(p->R_ratio >= 0.f)) return fail(ANN_ERR_ARG, "R_ratio must be >= 0 (or INFINITY)");
    if (p->merge_rule != 0 && p->merge_rule != 1) return fail(ANN_ERR_ARG, "merge_rule=%d not in {0, 1}", p->merge_rule);
    if (p->merge_rule == 1 && !(p->patience >= 0.f))
        return fail(ANN_ERR_ARG, "patience must be >= 0 (or INFINITY) with merge_rule 1");
    if (async && M > 32) return fail(ANN_ERR_ARG, "async mode runs one warp per walker: M=%d > 32", M);
    // cluster = 0 and at most 8 queries: each query on a cluster of 8 CTAs (4, 2 if fewer SMs), which the
    // one-query latency measurements favour at every (L, M), when the cluster kernel runs the search as asked
    // (sync, not persistent, no phase counters, no neighbour groups, a set-associative visited set); the
    // results are those of one CTA per query. If that plan does not fit, one CTA per query.
    if (p->cluster == 0 && nq >= 1 && nq <= 8 && !async && !p->persistent && !p->phase_cycles &&
        (p->visited_mode == 0 || p->visited_mode == 4) && x.n_hot == 0) {
        for (int c = 8; c >= 2; c >>= 1) {
            if ((int64_t)nq * c > sm_count()) continue;
            ann_search_params pc = *p;
            pc.cluster = c;
            const std::string saved = g_err;
            if (plan_search(index, queries, nq, k, L, M, out_ids, out_dists, &pc, plan) == ANN_OK) return ANN_OK;
            g_err = saved;
            break;
        }
    }
    const int csize = p->cluster > 1 ? p->cluster : 1;
    if (csize != 1 && csize != 2 && csize != 4 && csize != 8)
        return fail(ANN_ERR_ARG, "cluster=%d not in {0, 1, 2, 4, 8}", p->cluster);
    if (csize > 1 && async) return fail(ANN_ERR_ARG, "clusters are for sync mode only");
    int threads = p->threads;
    // Automatic launch shape, from (threads, visited bits) sweeps on the 1M x 128 (10,000 queries)
    // and 1M x 960 (1,000 queries) workloads. With at least 32 queries per SM the one-CTA sync
    // kernel is fastest with small CTAs (more queries in flight per SM) and a 2^12-slot visited
    // cache at every (L, M). With fewer queries each query's own latency counts: long queues or
    // heavy steps (M * R rows of at least 256 KB) take 512 threads and 2^14 slots.
    const bool many = !async && csize == 1 && nq >= 32LL * sm_count();
    const bool heavy = L >= 384 || (int64_t)M * x.R * x.d_pad * ann::storage_bytes(x.storage) >= (256 << 10);
    if (async) {
        // one warp per walker: T = M walkers, at least two warps
        int walkers = 2;
        while (walkers < M) walkers <<= 1;
        if (threads == 0) threads = 32 * walkers;
        if (threads != 64 && threads != 128 && threads != 256 && threads != 512 && threads != 1024)
            return fail(ANN_ERR_ARG, "threads=%d not in {64,...,1024}", threads);
        if (threads / 32 < M) return fail(ANN_ERR_ARG, "async mode needs threads >= 32*M");
    } else {
        if (threads == 0) threads = many ? (M * x.R >= 1024 ? 256 : 128) : (heavy ? 512 : (M * x.R >= 1024 ? 256 : 128));
        if (threads != 64 && threads != 128 && threads != 256 && threads != 512)
            return fail(ANN_ERR_ARG, "threads=%d not in {64,128,256,512}", threads);
        if (csize > 1 && threads == 64) threads = 128;
    }
    // visited set: 1 = open addressing; 2 = direct-mapped cache of tags; 3 = direct-mapped cache of ids;
    // 4 = set-associative cache of tags (2 or 3 ways per 32-bit set word)
    if (p->visited_mode < 0 || p->visited_mode > 4)
        return fail(ANN_ERR_ARG, "visited_mode=%d not in {0, 1, 2, 3, 4}", p->visited_mode);
    if ((p->visited_mode == 2 || p->visited_mode == 3) && (async || csize > 1))
        return fail(ANN_ERR_ARG, "the direct-mapped visited caches 2 and 3 are for the one-CTA sync kernel");
    if (csize > 1 && p->visited_mode != 0 && p->visited_mode != 4)
        return fail(ANN_ERR_ARG, "clusters keep their visited sets in the set-associative cache (visited_mode 0 or 4)");
    int idbits = 1;  // bits of the largest vertex id
    while (idbits < 31 && (int64_t(1) << idbits) < x.n) ++idbits;
    // tags per set word of the set-associative cache with 2^bits sets (0 if not even two fit)
    auto ways_for = [&](int bits) {
        const int fw = (idbits > bits ? idbits - bits : 0) + 1;
        return fw <= 10 ? 3 : (fw <= 16 ? 2 : 0);
    };
    // auto: a set-associative cache of tags for queues of 128 or more (thousands of vertices visited:
    // capacity and associativity pay; in the same 16 KB three ways repeat a few percent of the distances
    // that one way repeats), full ids below (a 2^12-id cache already holds what a short search visits, and
    // its exchange is cheaper than a CAS)
    // (the asynchronous walkers take it at every L: a set that forgets lets a walker queue, expand and
    // count again what another walker already saw, which changes when Algorithm 2 merges)
    int vmode = p->visited_mode == 0 ? ((csize > 1 || async || L >= 128) ? 4 : 3) : p->visited_mode;
    if (vmode == 4 && ways_for(15) < 2) {
        if (p->visited_mode == 4 || csize > 1)
            return fail(ANN_ERR_ARG, "visited_mode=4: ids of %d bits leave no room for two tags per set word", idbits);
        vmode = async ? 1 : 2;
    }
    auto slot_bytes_for = [&](int bits) {
        if (vmode != 2) return 4;
        const int tb = idbits > bits ? idbits - bits : 0;
        return tb <= 7 ? 1 : (tb <= 15 ? 2 : 4);
    };
    int hb = p->hash_bits;
    if (hb == 0) {
        if (many) {  // the most slots that fit in 16 KB (2^12 full ids or set words; 2^14 one-byte tags)
            hb = 12;
            for (int b = 14; b > 12; --b)
                if ((1 << b) * slot_bytes_for(b) <= (16 << 10)) {
                    hb = b;
                    break;
                }
            while (vmode == 4 && ways_for(hb) < 2) ++hb;  // more sets leave more bits per tag
        } else if (vmode == 4) {  // 2^13 sets hold 24,576 tags in 32 KB; 2^14 for long queues or heavy steps
            hb = heavy ? 14 : 13;
            while (ways_for(hb) < 2) ++hb;
        } else {
            hb = heavy ? 14 : (M * x.R >= 1024 ? 13 : 12);
        }
    }
    if (hb < 8 || hb > 15) return fail(ANN_ERR_ARG, "hash_bits=%d outside [8, 15]", hb);
    if (vmode == 4 && ways_for(hb) < 2)
        return fail(ANN_ERR_ARG, "visited_mode=4 with 2^%d sets: ids of %d bits leave no room for two tags", hb,
                    idbits);

    ann::SearchArgs &a = plan->a;
    memset(&a, 0, sizeof(a));
    a.base = x.base;
    a.scales = x.scales;
    a.base32 = x.base32;
    a.adj = x.adj;
    a.n = x.n;
    a.d = x.d;
    a.d_pad = x.d_pad;
    a.d_pad32 = x.d_pad32;
    a.R = x.R;
    a.entry = x.entry;
    a.metric = x.metric;
    a.queries = queries;
    a.nq = nq;
    a.k = k;
    a.L = L;
    a.M = M;
    a.k_arr = p->k_per_query;
    a.L_arr = p->L_per_query;
    a.M_arr = p->M_per_query;
    a.M0 = M0;
    a.t = t;
    a.R_ratio = p->R_ratio;
    a.merge_rule = p->merge_rule;
    a.patience = p->patience;
    a.rerank = p->rerank ? 1 : 0;
    a.hash_bits = hb;
    a.visited_mode = vmode >= 2 ? 1 : 0;
    if (p->l2_prefetch < 0 || p->l2_prefetch > 2)
        return fail(ANN_ERR_ARG, "l2_prefetch=%d not in {0, 1, 2}", p->l2_prefetch);
    a.l2_prefetch = p->l2_prefetch != 2;
    // neighbour groups serve the one-CTA sync kernel (the other kernels read every row by its id)
    a.hot_slot = (!async && csize == 1 && x.n_hot > 0) ? x.hot_slot : nullptr;
    a.group_prefetch = x.group_prefetch;
    if (p->gather < 0 || p->gather > 2) return fail(ANN_ERR_ARG, "gather=%d not in {0, 1, 2}", p->gather);
    // auto: one list per CTA (measured equal or faster than per-warp lists on every workload: much faster for
    // long rows, where a warp has few rows per step and its passes run part-empty; within 1 % for 128-d rows)
    a.block_gather = p->gather != 1;
    {
        const int tl = p->team_lanes;
        if (!(tl == -1 || tl == 0 || (tl > 0 && tl <= 32 && (tl & (tl - 1)) == 0)))
            return fail(ANN_ERR_ARG, "team_lanes=%d must be -1, 0 or a power of two up to 32", tl);
        auto log2_team = [tl](int cpr) {  // cpr = 16-byte chunks per row
            int ts = tl;
            if (tl == -1) {  // one chunk per lane
                ts = 1;
                while (ts < cpr && ts < 32) ts <<= 1;
            } else if (tl == 0) {  // auto: 4 lanes for rows of up to 64 chunks (1 KB), else 8 (measured best)
                ts = cpr <= 64 ? 4 : 8;
            }
            int lts = 0;
            while ((1 << lts) < ts) ++lts;
            return lts;
        };
        a.team_lanes = log2_team(x.d_pad * ann::storage_bytes(x.storage) / 16);
        a.team_lanes32 = log2_team(x.d_pad32 * 4 / 16);
    }
    a.out_ids = out_ids;
    a.out_dists = out_dists;
    a.stats = p->stats;
    a.work_counter = x.work_counter;
    a.persistent = p->persistent ? 1 : 0;
    a.order = p->order;
    a.phase_cycles = reinterpret_cast<long long *>(p->phase_cycles);
    a.Lcap = L;
    int need = M * x.R;
    if (a.rerank && L > need) need = L;
    if (!async) {  // the warps' fresh lists live in the candidate segment
        const int nw = threads / 32;
        const int fresh_entries = nw * ((M * x.R + nw - 1) / nw);  // one (id, row) pair per entry
        if (fresh_entries > need) need = fresh_entries;
    }
    a.Ccap = ann::next_pow2(need < 32 ? 32 : need);
    a.qfloats = x.d_pad > x.d_pad32 ? x.d_pad : x.d_pad32;
    auto smem_for = [&](int bits) {
        if (csize > 1) return ann::cluster_smem_size(a.qfloats, a.Lcap, a.Ccap, bits, M);
        return async ? ann::async_smem_size(a.qfloats, a.Lcap, threads / 32, bits)
                     : ann::sync_layout(a.qfloats, a.Lcap, a.Ccap, bits, M, slot_bytes_for(bits), threads / 32).total;
    };
    int smem = smem_for(a.hash_bits);
    // an automatic visited table shrinks until the layout fits (it may then forget more often)
    while (p->hash_bits == 0 && smem > max_dyn_smem() && a.hash_bits > 10) smem = smem_for(--a.hash_bits);
    a.slot_bytes = slot_bytes_for(a.hash_bits);
    a.tag_bits = (a.slot_bytes < 4 || vmode == 4) && idbits > a.hash_bits ? idbits - a.hash_bits : 0;
    a.ways = vmode == 4 ? ways_for(a.hash_bits) : 0;
    if (vmode == 4 && a.ways < 2)
        return fail(ANN_ERR_ARG, "visited_mode=4: the set words do not fit two tags at 2^%d sets", a.hash_bits);
    a.sync_lay = ann::sync_layout(a.qfloats, a.Lcap, a.Ccap, a.hash_bits, M, a.slot_bytes, threads / 32);
    if (smem > max_dyn_smem())
        return fail(ANN_ERR_ARG, "shared memory %d B exceeds the device limit %d B (lower L, M or hash_bits)",
                    smem, max_dyn_smem());
    plan->threads = threads;
    plan->smem = smem;
    plan->mode = p->mode;
    plan->storage = x.storage;
    plan->cluster = csize;
    if (csize > 1) a.persistent = 0;
    plan->grid = (int)(nq > 0x7fffffff ? 0x7fffffff : nq);
    if (a.persistent && csize == 1 && nq > 0) {
        int bps = 0;
        cudaError_t e = async ? ann::async_search_occupancy(x.storage, threads, smem, &bps)
                              : ann::sync_search_occupancy(x.storage, x.metric, threads, smem, &bps);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
        if (bps < 1) return fail(ANN_ERR_ARG, "kernel does not fit on an SM");
        int64_t g = (int64_t)bps * sm_count();
        plan->grid = (int)(g < nq ? g : nq);
    }
    return ANN_OK;
}

cudaError_t launch(const Plan &plan, cudaStream_t s) {
    if (plan.cluster > 1)
        return ann::launch_cluster_search(plan.a, plan.storage, plan.threads, plan.smem, plan.cluster, s);
    return plan.mode == ANN_MODE_ASYNC
               ? ann::launch_async_search(plan.a, plan.storage, plan.threads, plan.smem, plan.grid, s)
               : ann::launch_sync_search(plan.a, plan.storage, plan.threads, plan.smem, plan.grid, s);
}

int index_device(const ann_index *index) { return index->d.device; }

}  // namespace ann

namespace {

using ann::Plan;
using ann::plan_search;

// The work-counter slot of a stream. Work on one stream runs in order, so a
// stream can reuse its slot call after call; different streams get different
// slots. The per-thread default stream is one stream per host thread, so it
// is keyed by the thread as well.
int counter_slot(const ann_index *index, cudaStream_t s, int **out) {
    ann_index *ix = const_cast<ann_index *>(index);
    std::string key = std::to_string(reinterpret_cast<uintptr_t>(s));
    if (s == cudaStreamPerThread) {
        key += "/";
        key += std::to_string(std::hash<std::thread::id>()(std::this_thread::get_id()));
    } else if (s == cudaStreamLegacy) {
        key = "0";  // the legacy default stream, however it is named
    }
    std::lock_guard<std::mutex> lock(ix->slot_mu);
    auto it = ix->slot_of.find(key);
    int slot;
    if (it != ix->slot_of.end()) {
        slot = it->second;
    } else {
        if ((int)ix->slot_of.size() >= ann::kCounterSlots)
            return fail(ANN_ERR_STATE, "more than %d streams ran persistent searches on this index",
                        ann::kCounterSlots);
        slot = (int)ix->slot_of.size();
        ix->slot_of.emplace(key, slot);
    }
    *out = index->d.work_counter + (size_t)slot * ann::kCounterStride;
    return ANN_OK;
}

int launch_plan(const ann_index *index, const Plan &plan_in, cudaStream_t s) {
    if (plan_in.a.nq == 0) return ANN_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != index->d.device) return fail(ANN_ERR_STATE, "current device %d is not the index's device %d", dev, index->d.device);
    Plan plan = plan_in;
    if (plan.a.persistent) {
        int rc = counter_slot(index, s, &plan.a.work_counter);
        if (rc != ANN_OK) return rc;
        ANN_CUDA(cudaMemsetAsync(plan.a.work_counter, 0, sizeof(int), s));
    }
    cudaError_t e = ann::launch(plan, s);
    if (e != cudaSuccess) return cuda_fail(e, "search launch");
    return ANN_OK;
}

}  // namespace

namespace ann {
void set_error(const char *msg) { g_err = msg; }

cudaError_t ensure_dyn_smem(const void *kernel, int smem) {
    static std::mutex mu;
    static std::unordered_map<std::string, int> limit;  // (kernel, device) -> the limit set so far
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::string key = std::to_string(reinterpret_cast<uintptr_t>(kernel)) + "/" + std::to_string(dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = limit.find(key);
    if (it != limit.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) limit[key] = smem;
    return e;
}
}  // namespace ann

extern "C" {

int ann_index_create(const float *base, int64_t n, int32_t d, int32_t storage, const int32_t *adj, int32_t R,
                     int64_t entry, int32_t metric, int32_t flags, ann_index **out) {
    return create_impl(base, n, d, storage, adj, R, entry, metric, flags, out);
}

void ann_index_destroy(ann_index *index) {
    if (!index) return;
    free_index_data(index->d);
    delete index;
}

int ann_index_get_info(const ann_index *index, ann_index_info *info) {
    if (!index || !info) return fail(ANN_ERR_ARG, "index and info must not be NULL");
    const ann::IndexData &x = index->d;
    info->n = x.n;
    info->d = x.d;
    info->d_pad = x.d_pad;
    info->R = x.R;
    info->storage = x.storage;
    info->metric = x.metric;
    info->has_f32 = x.base32 != nullptr;
    info->entry = x.entry;
    info->device_bytes = x.device_bytes;
    info->n_hot = x.n_hot;
    return ANN_OK;
}

int ann_knn_bf16(const void *base, int64_t n, int32_t d, const void *queries, int64_t nq, int64_t self_offset,
                 int32_t metric, int32_t k, int32_t *out_ids, float *out_dists, void *stream) {
    if (!base || !queries || !out_ids || !out_dists) return fail(ANN_ERR_ARG, "null pointer");
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(ANN_ERR_ARG, "n=%lld outside [1, 2^31)", (long long)n);
    if (nq < 0 || nq >= (int64_t(1) << 31)) return fail(ANN_ERR_ARG, "nq=%lld outside [0, 2^31)", (long long)nq);
    if (d != 32 && d != 64 && d != 96 && d != 128) return fail(ANN_ERR_ARG, "d=%d not in {32, 64, 96, 128}", d);
    if (k < 1 || k > 64) return fail(ANN_ERR_ARG, "k=%d outside [1, 64]", k);
    if (metric != ANN_METRIC_L2 && metric != ANN_METRIC_IP) return fail(ANN_ERR_ARG, "metric=%d", metric);
    if (((uintptr_t)base & 15) || ((uintptr_t)queries & 15))
        return fail(ANN_ERR_ARG, "base and queries must be 16-byte aligned");
    if (self_offset < -1 || (self_offset >= 0 && self_offset + nq > n))
        return fail(ANN_ERR_ARG, "self_offset=%lld does not place the queries inside the base", (long long)self_offset);
    if (nq == 0) return ANN_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float *norms = nullptr;
    int *err = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&norms, (size_t)ann::knn_norms_rows(n) * 4 + 16)) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc(knn norms)");
    err = reinterpret_cast<int *>(reinterpret_cast<unsigned char *>(norms) + (size_t)ann::knn_norms_rows(n) * 4);
    int herr = 0;
    if ((e = cudaMemsetAsync(err, 0, 4, s)) == cudaSuccess &&
        (e = ann::launch_knn_bf16(base, n, d, queries, nq, self_offset, metric, k, out_ids, out_dists, norms, err,
                                  s)) == cudaSuccess &&
        (e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s)) == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFree(norms);
    if (e != cudaSuccess) return cuda_fail(e, "knn");
    if (herr) return fail(ANN_ERR_CUDA, "knn: a candidate merge did not converge");
    return ANN_OK;
}

int ann_index_group_neighbors(ann_index *index, float hot_fraction, int32_t prefetch) {
    if (!index) return fail(ANN_ERR_ARG, "index is NULL");
    if (!(hot_fraction >= 0.f && hot_fraction <= 0.05f))
        return fail(ANN_ERR_ARG, "hot_fraction=%g outside [0, 0.05]", (double)hot_fraction);
    if (prefetch != 0 && prefetch != 1) return fail(ANN_ERR_ARG, "prefetch=%d not in {0, 1}", prefetch);
    ann::IndexData &x = index->d;
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    if (dev != x.device) return fail(ANN_ERR_STATE, "current device %d is not the index's device %d", dev, x.device);
    const int64_t H = (int64_t)std::llround((double)hot_fraction * (double)x.n);
    if ((uint64_t)x.n + (uint64_t)H * (uint64_t)x.R >= (1ull << 32))
        return fail(ANN_ERR_ARG, "n + hot vertices * R must stay below 2^32 rows");
    ANN_CUDA(cudaDeviceSynchronize());
    const int64_t es = ann::storage_bytes(x.storage), row_bytes = (int64_t)x.d_pad * es;
    if (H == 0) {  // no groups: the search reads every row by its id (the spare rows stay allocated)
        cudaFree(x.hot_slot);
        x.hot_slot = nullptr;
        x.n_hot = 0;
        return ANN_OK;
    }
    // in-degrees, then the H vertices with the most in-edges (ties: the smaller id)
    std::vector<int32_t> deg(x.n);
    {
        int32_t *ddeg = nullptr;
        ANN_CUDA(cudaMalloc(&ddeg, (size_t)x.n * 4));
        cudaError_t e = cudaMemset(ddeg, 0, (size_t)x.n * 4);
        if (e == cudaSuccess) e = ann::launch_count_in_degree(x.adj, x.n * (int64_t)x.R, ddeg, 0);
        if (e == cudaSuccess) e = cudaMemcpy(deg.data(), ddeg, (size_t)x.n * 4, cudaMemcpyDeviceToHost);
        cudaFree(ddeg);
        if (e != cudaSuccess) return cuda_fail(e, "in-degree");
    }
    std::vector<int32_t> order(x.n);
    for (int64_t i = 0; i < x.n; ++i) order[i] = (int32_t)i;
    auto hotter = [&](int32_t a, int32_t b) { return deg[a] > deg[b] || (deg[a] == deg[b] && a < b); };
    std::nth_element(order.begin(), order.begin() + (H - 1), order.end(), hotter);
    std::sort(order.begin(), order.begin() + H);  // groups in id order
    std::vector<int32_t> slot(x.n, -1);
    for (int64_t s = 0; s < H; ++s) slot[order[s]] = (int32_t)s;
    // a base (and scale) buffer with room for the groups, the first n rows copied over
    const int64_t rows = x.n + H * x.R;
    unsigned char *nb = nullptr;
    float *nsc = nullptr;
    int32_t *dhot = nullptr, *dslot = nullptr;
    auto undo = [&](int code) {
        cudaFree(nb);
        cudaFree(nsc);
        cudaFree(dhot);
        cudaFree(dslot);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&nb, (size_t)rows * row_bytes)) != cudaSuccess) return undo(cuda_fail(e, "cudaMalloc(groups)"));
    if (x.scales && (e = cudaMalloc(&nsc, (size_t)rows * 4)) != cudaSuccess) return undo(cuda_fail(e, "cudaMalloc(scales)"));
    if ((e = cudaMalloc(&dhot, (size_t)H * 4)) != cudaSuccess) return undo(cuda_fail(e, "cudaMalloc(hot)"));
    if ((e = cudaMalloc(&dslot, (size_t)x.n * 4)) != cudaSuccess) return undo(cuda_fail(e, "cudaMalloc(hot_slot)"));
    e = cudaMemcpy(nb, x.base, (size_t)x.n * row_bytes, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && nsc) e = cudaMemcpy(nsc, x.scales, (size_t)x.n * 4, cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dhot, order.data(), (size_t)H * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dslot, slot.data(), (size_t)x.n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ann::launch_fill_groups(nb, nsc, x.adj, dhot, H, x.R, x.n, (int32_t)row_bytes, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dhot);
    dhot = nullptr;
    if (e != cudaSuccess) return undo(cuda_fail(e, "neighbour groups"));
    const bool alias32 = !x.owns_base32 && x.base32 == reinterpret_cast<float *>(x.base);
    const int64_t old_rows = x.n + x.n_hot * x.R;
    cudaFree(x.base);
    cudaFree(x.scales);
    cudaFree(x.hot_slot);
    x.base = nb;
    x.scales = nsc;
    x.hot_slot = dslot;
    if (alias32) x.base32 = reinterpret_cast<float *>(nb);
    x.device_bytes += (rows - old_rows) * row_bytes + (nsc ? (rows - old_rows) * 4 : 0) +
                      (old_rows == x.n ? x.n * 4 : 0);
    x.n_hot = H;
    x.group_prefetch = prefetch;
    return ANN_OK;
}

int ann_search_ex(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L, int32_t M,
                  int64_t *out_ids, float *out_dists, const ann_search_params *params, void *stream) {
    Plan plan;
    int rc = plan_search(index, queries, nq, k, L, M, out_ids, out_dists, params, &plan);
    if (rc != ANN_OK) return rc;
    return launch_plan(index, plan, reinterpret_cast<cudaStream_t>(stream));
}

int ann_search(const ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L, int32_t M,
               int64_t *out_ids, float *out_dists, void *stream) {
    return ann_search_ex(index, queries, nq, k, L, M, out_ids, out_dists, nullptr, stream);
}

int ann_search_host(ann_index *index, const float *queries, int64_t nq, int32_t k, int32_t L, int32_t M,
                    int64_t *out_ids, float *out_dists, const ann_search_params *params, void *stream) {
    if (!index) return fail(ANN_ERR_ARG, "index is NULL");
    if (nq == 0) return ANN_OK;
    ann::IndexData &x = index->d;
    const size_t qb = (size_t)nq * x.d * 4, ib = (size_t)nq * k * 8, db = (size_t)nq * k * 4;
    const size_t need = ((qb + 255) & ~size_t(255)) + ((ib + 255) & ~size_t(255)) + db;
    // validate before touching the staging buffers (device pointers are placeholders here)
    Plan plan;
    int rc = plan_search(index, reinterpret_cast<const float *>(16), nq, k, L, M,
                         reinterpret_cast<int64_t *>(16), reinterpret_cast<float *>(16), params, &plan);
    if (rc != ANN_OK) return rc;
    if (!queries || !out_ids || !out_dists) return fail(ANN_ERR_ARG, "host pointers must not be NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (x.stage_bytes < need) {
        ANN_CUDA(cudaStreamSynchronize(s));
        cudaFree(x.stage);
        x.stage = nullptr;
        x.stage_bytes = 0;
        ANN_CUDA(cudaMalloc(&x.stage, need));
        x.stage_bytes = need;
    }
    char *st = reinterpret_cast<char *>(x.stage);
    float *dq = reinterpret_cast<float *>(st);
    int64_t *dids = reinterpret_cast<int64_t *>(st + ((qb + 255) & ~size_t(255)));
    float *ddist = reinterpret_cast<float *>(st + ((qb + 255) & ~size_t(255)) + ((ib + 255) & ~size_t(255)));
    plan.a.queries = dq;
    plan.a.out_ids = dids;
    plan.a.out_dists = ddist;
    ANN_CUDA(cudaMemcpyAsync(dq, queries, qb, cudaMemcpyHostToDevice, s));
    rc = launch_plan(index, plan, s);
    if (rc != ANN_OK) return rc;
    ANN_CUDA(cudaMemcpyAsync(out_ids, dids, ib, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaMemcpyAsync(out_dists, ddist, db, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaStreamSynchronize(s));
    return ANN_OK;
}

int ann_search_describe(const ann_index *index, int64_t nq, int32_t k, int32_t L, int32_t M,
                        const ann_search_params *params, ann_launch_info *out) {
    if (!out) return fail(ANN_ERR_ARG, "out is NULL");
    Plan plan;
    int rc = plan_search(index, reinterpret_cast<const float *>(16), nq, k, L, M, reinterpret_cast<int64_t *>(16),
                         reinterpret_cast<float *>(16), params, &plan);
    if (rc != ANN_OK) return rc;
    out->threads = plan.threads;
    out->smem_bytes = plan.smem;
    out->grid = plan.cluster > 1 ? (int32_t)(nq * plan.cluster) : plan.grid;
    out->hash_bits = plan.a.hash_bits;
    out->cluster = plan.cluster;
    out->mode = plan.mode;
    out->visited_slot_bytes = plan.a.slot_bytes;
    out->visited_ways = plan.a.ways;
    return ANN_OK;
}

const char *ann_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free host-buffer search.
//
// For callers that must not allocate device memory at search time: processes
// whose device memory is reserved up front by another framework's caching
// allocator, or latency-critical threads that must not enter the CUDA
// allocator (it can block on the device). This entry point keeps all of its
// device scratch (the persistent grid's work counter and the staging copies
// of the queries and results) in one file-scope static device array, and
// calls no cudaMalloc, cudaFree or other allocating routine.
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)ANN_NOALLOC_SCRATCH_BYTES;

// Every GPU that loads this library holds this array until the process
// exits. In host code its name is only a stand-in for the symbol, never a
// device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ANN_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256];  // device address of g_noalloc_scratch per device ordinal

// Resolves the array's device address once per device, with that device
// current. The first call on a device does this; it may load the module, so
// that first call should happen before any stream capture.
int noalloc_scratch_address(void **out) {
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(ANN_ERR_STATE, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return ANN_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int ann_search_host_noalloc(const ann_index *index, const float *queries, int64_t nq, int32_t k,
                                       int32_t L, int32_t M, int64_t *out_ids, float *out_dists,
                                       const ann_search_params *params, void *stream) {
    if (!index) return fail(ANN_ERR_ARG, "index is NULL");
    if (nq == 0) return ANN_OK;
    ann_search_params p;
    memset(&p, 0, sizeof(p));
    if (params) p = *params;
    p.persistent = 1;
    if (p.cluster > 1)
        return fail(ANN_ERR_ARG, "cluster=%d: the allocation-free search runs one CTA per query (0 or 1)",
                    p.cluster);
    Plan plan;
    int rc = plan_search(index, reinterpret_cast<const float *>(16), nq, k, L, M,
                         reinterpret_cast<int64_t *>(16), reinterpret_cast<float *>(16), &p, &plan);
    if (rc != ANN_OK) return rc;
    if (!queries || !out_ids || !out_dists) return fail(ANN_ERR_ARG, "host pointers must not be NULL");
    const ann::IndexData &x = index->d;
    const size_t qb = (size_t)nq * x.d * 4, ib = (size_t)nq * k * 8, db = (size_t)nq * k * 4;
    const size_t need = 256 + align256(qb) + align256(ib) + db;
    if (need > kNoallocScratchBytes)
        return fail(ANN_ERR_ARG,
                    "batch needs %zu bytes of static device scratch (nq=%lld, d=%d, k=%d); the maximum is %zu bytes",
                    need, (long long)nq, x.d, k, kNoallocScratchBytes);
    int dev = 0;
    ANN_CUDA(cudaGetDevice(&dev));
    if (dev != x.device) return fail(ANN_ERR_STATE, "current device %d is not the index's device %d", dev, x.device);
    void *base = nullptr;
    rc = noalloc_scratch_address(&base);
    if (rc != ANN_OK) return rc;
    char *sb = reinterpret_cast<char *>(base);
    int *counter = reinterpret_cast<int *>(sb);
    float *dq = reinterpret_cast<float *>(sb + 256);
    int64_t *dids = reinterpret_cast<int64_t *>(sb + 256 + align256(qb));
    float *ddist = reinterpret_cast<float *>(sb + 256 + align256(qb) + align256(ib));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    plan.a.queries = dq;
    plan.a.out_ids = dids;
    plan.a.out_dists = ddist;
    plan.a.work_counter = counter;
    plan.a.persistent = 1;
    // the array keeps the previous call's contents: the counter must start at zero
    ANN_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    ANN_CUDA(cudaMemcpyAsync(dq, queries, qb, cudaMemcpyHostToDevice, s));
    cudaError_t e = ann::launch(plan, s);
    if (e != cudaSuccess) return cuda_fail(e, "search launch");
    ANN_CUDA(cudaMemcpyAsync(out_ids, dids, ib, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaMemcpyAsync(out_dists, ddist, db, cudaMemcpyDeviceToHost, s));
    ANN_CUDA(cudaStreamSynchronize(s));
    return ANN_OK;
}
