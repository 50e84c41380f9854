// batch.cu -- planned batches of queries with uneven k, L, M (ann_batch_*).
//
// The planner groups queries into buckets by L, orders each bucket by
// descending L (longest first, so a persistent grid does not end on one
// long query) and prepares one persistent launch per bucket, whose shared
// memory, block size and visited table are sized for that bucket only. A
// search forks the caller's stream into one stream per bucket (event
// record / wait), resets each bucket's work counter, launches, and joins
// back: all stream-ordered, no allocation, no host synchronisation, so the
// whole call can be captured into a CUDA graph and replayed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ann_internal.cuh"

namespace {

struct Bucket {
    ann::Plan plan;
    int count = 0;
    int offset = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t joined = nullptr;
};

int bfail(int code, const char *msg) {
    ann::set_error(msg);
    return code;
}

}  // namespace

struct ann_batch {
    const ann_index *index = nullptr;
    int64_t nq = 0;
    int32_t kmax = 0;
    int32_t *d_kLM = nullptr;   // k[nq], L[nq], M[nq]
    int32_t *d_order = nullptr; // bucket work lists back to back
    int *d_counters = nullptr;  // one per bucket
    cudaEvent_t fork = nullptr;
    std::vector<Bucket> buckets;
};

namespace {

void free_batch(ann_batch *b) {
    for (Bucket &k : b->buckets) {
        if (k.joined) cudaEventDestroy(k.joined);
        if (k.stream) cudaStreamDestroy(k.stream);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    cudaFree(b->d_kLM);
    cudaFree(b->d_order);
    cudaFree(b->d_counters);
    delete b;
}

}  // namespace

extern "C" {

int ann_batch_create(const ann_index *index, int64_t nq, const int32_t *k, const int32_t *L, const int32_t *M,
                     const ann_bucket_config *buckets, int32_t n_buckets, const ann_search_params *params,
                     ann_batch **out) {
    if (!out) return bfail(ANN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!index || nq < 1 || nq > 0x7fffffffll || !k || !L || !M)
        return bfail(ANN_ERR_ARG, "index, nq >= 1 and the host k / L / M arrays are required");
    if (params && (params->k_per_query || params->L_per_query || params->M_per_query || params->order))
        return bfail(ANN_ERR_ARG, "params of a batch must not carry per-query arrays or a work list");
    static const int32_t ladder[] = {32, 64, 128, 256, 512, 1024, 2048};
    std::vector<ann_bucket_config> cfg;
    if (buckets && n_buckets > 0) {
        cfg.assign(buckets, buckets + n_buckets);
    } else {
        for (int32_t v : ladder) cfg.push_back(ann_bucket_config{v, 0, 0});
    }
    for (size_t i = 0; i < cfg.size(); ++i)
        if (cfg[i].L_max < 1 || cfg[i].L_max > 2048 || (i > 0 && cfg[i].L_max <= cfg[i - 1].L_max))
            return bfail(ANN_ERR_ARG, "bucket L_max values must ascend within [1, 2048]");
    int32_t kmax = 0;
    std::vector<int> which(nq);
    for (int64_t i = 0; i < nq; ++i) {
        if (k[i] < 1 || L[i] < k[i] || L[i] > 2048 || M[i] < 1 || M[i] > 64)
            return bfail(ANN_ERR_ARG, "a query's k, L, M is outside 1 <= k <= L <= 2048, 1 <= M <= 64");
        int b = 0;
        while (b < (int)cfg.size() && L[i] > cfg[b].L_max) b++;
        if (b == (int)cfg.size()) return bfail(ANN_ERR_ARG, "a query's L exceeds the largest bucket");
        which[i] = b;
        kmax = std::max(kmax, k[i]);
    }
    ann_batch *bt = new (std::nothrow) ann_batch;
    if (!bt) return bfail(ANN_ERR_OOM, "host allocation");
    bt->index = index;
    bt->nq = nq;
    bt->kmax = kmax;
    // work lists: bucket by bucket, longest L first (ties by query number)
    std::vector<int32_t> order(nq);
    for (int64_t i = 0; i < nq; ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (which[a] != which[b]) return which[a] < which[b];
        return L[a] > L[b];
    });
    std::vector<int32_t> kLM(3 * nq);
    memcpy(kLM.data(), k, nq * 4);
    memcpy(kLM.data() + nq, L, nq * 4);
    memcpy(kLM.data() + 2 * nq, M, nq * 4);
    cudaError_t e = cudaMalloc(&bt->d_kLM, 3 * nq * 4);
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_order, nq * 4);
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_counters, cfg.size() * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(bt->d_kLM, kLM.data(), 3 * nq * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(bt->d_order, order.data(), nq * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_batch(bt);
        cudaGetLastError();
        return bfail(e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA, cudaGetErrorString(e));
    }
    ann_search_params base;
    memset(&base, 0, sizeof(base));
    if (params) base = *params;
    int64_t pos = 0;
    for (int b = 0; b < (int)cfg.size(); ++b) {
        int64_t n = 0;
        int32_t Lm = 0, Mm = 0;
        while (pos + n < nq && which[order[pos + n]] == b) {
            Lm = std::max(Lm, L[order[pos + n]]);
            Mm = std::max(Mm, M[order[pos + n]]);
            n++;
        }
        if (n == 0) continue;
        Bucket bk;
        bk.count = (int)n;
        bk.offset = (int)pos;
        ann_search_params p = base;
        p.k_per_query = bt->d_kLM;
        p.L_per_query = bt->d_kLM + nq;
        p.M_per_query = bt->d_kLM + 2 * nq;
        p.order = bt->d_order + pos;
        p.persistent = 1;
        if (cfg[b].threads) p.threads = cfg[b].threads;
        if (cfg[b].hash_bits) p.hash_bits = cfg[b].hash_bits;
        // device pointers for queries / outputs are bound at search time
        int rc = ann::plan_search(index, reinterpret_cast<const float *>(16), n, std::min(kmax, Lm), Lm, Mm,
                                  reinterpret_cast<int64_t *>(16), reinterpret_cast<float *>(16), &p, &bk.plan);
        if (rc != ANN_OK) {
            free_batch(bt);
            return rc;
        }
        bk.plan.a.k = kmax;  // output row stride (and per-query k bound) of the whole batch
        bk.plan.a.work_counter = bt->d_counters + bt->buckets.size();
        e = cudaStreamCreateWithFlags(&bk.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bk.joined, cudaEventDisableTiming);
        bt->buckets.push_back(bk);
        if (e != cudaSuccess) {
            free_batch(bt);
            return bfail(ANN_ERR_CUDA, cudaGetErrorString(e));
        }
        pos += n;
    }
    *out = bt;
    return ANN_OK;
}

int ann_batch_search(ann_batch *bt, const float *queries, int64_t *out_ids, float *out_dists, void *stream) {
    if (!bt || !queries || !out_ids || !out_dists) return bfail(ANN_ERR_ARG, "batch, queries and outputs must not be NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != ann::index_device(bt->index)) return bfail(ANN_ERR_STATE, "current device is not the index's device");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(bt->fork, s);
    for (size_t b = 0; e == cudaSuccess && b < bt->buckets.size(); ++b) {
        Bucket &bk = bt->buckets[b];
        bk.plan.a.queries = queries;
        bk.plan.a.out_ids = out_ids;
        bk.plan.a.out_dists = out_dists;
        e = cudaStreamWaitEvent(bk.stream, bt->fork, 0);
        if (e == cudaSuccess) e = cudaMemsetAsync(bk.plan.a.work_counter, 0, sizeof(int), bk.stream);
        if (e == cudaSuccess) e = ann::launch(bk.plan, bk.stream);
        if (e == cudaSuccess) e = cudaEventRecord(bk.joined, bk.stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, bk.joined, 0);
    }
    if (e != cudaSuccess) return bfail(ANN_ERR_CUDA, cudaGetErrorString(e));
    return ANN_OK;
}

int ann_batch_info(const ann_batch *bt, int32_t *n_buckets, int32_t *k_max) {
    if (!bt) return bfail(ANN_ERR_ARG, "batch is NULL");
    if (n_buckets) *n_buckets = (int32_t)bt->buckets.size();
    if (k_max) *k_max = bt->kmax;
    return ANN_OK;
}

void ann_batch_destroy(ann_batch *bt) {
    if (bt) free_batch(bt);
}

}  // extern "C"
