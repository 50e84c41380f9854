// serve.cu -- continuous-batching request server over an index (ann_serve_*).
//
// Requests arrive one at a time on the host. Device-resident request state is
// organised in `streams` groups of max_batch requests; each group owns a
// stream, device buffers (queries, per-request k / L / M, results, counters),
// pinned host mirrors and a completion event. A scheduler thread
//   - harvests groups whose event has fired (results copied out, latency
//     taken, completions queued for ann_serve_poll),
//   - fills every free group with waiting requests (the oldest and those of
//     its cost class: L in the same power-of-two range) and launches it:
//     H2D copy of the batch, one search launch with per-query k / L / M, D2H
//     copy of results and counters, event record -- all on the group's stream.
// Groups run concurrently on the device, so requests that arrive while
// others are running are admitted as soon as a group frees up and overlap
// with the work already on the GPU. No kernel or copy waits on another
// group; the host thread only polls events.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "ann_internal.cuh"

namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    uint64_t tag;
    int32_t k, L, M;
    double t_submit;
    std::vector<float> q;
};

struct Done {
    ann_result r;
    std::vector<int64_t> ids;
    std::vector<float> dists;
};

struct Group {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float *d_q = nullptr;
    int32_t *d_kLM = nullptr;  // k[b], L[b], M[b] back to back
    int64_t *d_ids = nullptr;
    float *d_dists = nullptr;
    ann_query_stats *d_stats = nullptr;
    float *h_q = nullptr;
    int32_t *h_kLM = nullptr;
    int64_t *h_ids = nullptr;
    float *h_dists = nullptr;
    ann_query_stats *h_stats = nullptr;
    std::vector<Request> reqs;
    bool busy = false;
    int status = ANN_OK;
};

}  // namespace

struct ann_server {
    const ann_index *index = nullptr;
    ann_serve_config cfg;
    ann_index_info info;
    int device = 0;
    std::vector<Group> groups;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    // waiting requests, one queue per cost class (L in the same power-of-two range: L <= 2048)
    static constexpr int kClasses = 12;
    std::deque<Request> pending[kClasses];
    int64_t npending = 0;
    std::deque<Done> done;
    int64_t accepted = 0;  // submitted and not yet collected
    bool stop = false;
    std::thread th;
};

namespace {

void free_group(Group &g) {
    cudaFree(g.d_q);
    cudaFree(g.d_kLM);
    cudaFree(g.d_ids);
    cudaFree(g.d_dists);
    cudaFree(g.d_stats);
    cudaFreeHost(g.h_q);
    cudaFreeHost(g.h_kLM);
    cudaFreeHost(g.h_ids);
    cudaFreeHost(g.h_dists);
    cudaFreeHost(g.h_stats);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
    g = Group();
}

cudaError_t alloc_group(Group &g, int B, int d, int kmax) {
    cudaError_t e;
#define TRY(x)                                \
    if ((e = (x)) != cudaSuccess) return e;
    TRY(cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking));
    TRY(cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming));
    TRY(cudaMalloc(&g.d_q, (size_t)B * d * 4));
    TRY(cudaMalloc(&g.d_kLM, (size_t)B * 3 * 4));
    TRY(cudaMalloc(&g.d_ids, (size_t)B * kmax * 8));
    TRY(cudaMalloc(&g.d_dists, (size_t)B * kmax * 4));
    TRY(cudaMalloc(&g.d_stats, (size_t)B * sizeof(ann_query_stats)));
    TRY(cudaHostAlloc(&g.h_q, (size_t)B * d * 4, cudaHostAllocDefault));
    TRY(cudaHostAlloc(&g.h_kLM, (size_t)B * 3 * 4, cudaHostAllocDefault));
    TRY(cudaHostAlloc(&g.h_ids, (size_t)B * kmax * 8, cudaHostAllocDefault));
    TRY(cudaHostAlloc(&g.h_dists, (size_t)B * kmax * 4, cudaHostAllocDefault));
    TRY(cudaHostAlloc(&g.h_stats, (size_t)B * sizeof(ann_query_stats), cudaHostAllocDefault));
#undef TRY
    return cudaSuccess;
}

size_t group_device_bytes(int B, int d, int kmax) {
    return (size_t)B * ((size_t)d * 4 + 12 + (size_t)kmax * 12 + sizeof(ann_query_stats));
}

// Copy the batch in, search, copy results out, record the event.
// Requests whose queue lengths share a power-of-two range share launches.
int cost_class(int L) {
    int c = 0;
    while ((1 << c) < L) ++c;
    return c;
}

void launch_group(ann_server *s, Group &g) {
    const int B = (int)g.reqs.size(), d = s->info.d, kmax = s->cfg.max_k;
    for (int i = 0; i < B; ++i) {
        memcpy(g.h_q + (size_t)i * d, g.reqs[i].q.data(), (size_t)d * 4);
        g.h_kLM[i] = g.reqs[i].k;
        g.h_kLM[B + i] = g.reqs[i].L;
        g.h_kLM[2 * B + i] = g.reqs[i].M;
    }
    g.status = ANN_OK;
    cudaError_t e = cudaMemcpyAsync(g.d_q, g.h_q, (size_t)B * d * 4, cudaMemcpyHostToDevice, g.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.d_kLM, g.h_kLM, (size_t)B * 12, cudaMemcpyHostToDevice, g.stream);
    if (e != cudaSuccess) g.status = ANN_ERR_CUDA;
    if (g.status == ANN_OK) {
        ann_search_params p;
        memset(&p, 0, sizeof(p));
        p.mode = s->cfg.mode;
        p.rerank = s->cfg.rerank;
        p.R_ratio = 0.8f;
        p.cluster = 1;  // one CTA per request: groups run side by side and share the SMs
        p.k_per_query = g.d_kLM;
        p.L_per_query = g.d_kLM + B;
        p.M_per_query = g.d_kLM + 2 * B;
        p.stats = g.d_stats;
        if (ann_search_ex(s->index, g.d_q, B, kmax, s->cfg.max_L, s->cfg.max_M, g.d_ids, g.d_dists, &p, g.stream) !=
            ANN_OK)
            g.status = ANN_ERR_CUDA;
    }
    if (g.status == ANN_OK) {
        e = cudaMemcpyAsync(g.h_ids, g.d_ids, (size_t)B * kmax * 8, cudaMemcpyDeviceToHost, g.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_dists, g.d_dists, (size_t)B * kmax * 4, cudaMemcpyDeviceToHost, g.stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_stats, g.d_stats, (size_t)B * sizeof(ann_query_stats),
                                                  cudaMemcpyDeviceToHost, g.stream);
        if (e != cudaSuccess) g.status = ANN_ERR_CUDA;
    }
    cudaEventRecord(g.done, g.stream);
    g.busy = true;
}

void harvest_group(ann_server *s, Group &g, std::deque<Done> &out) {
    const int B = (int)g.reqs.size(), kmax = s->cfg.max_k;
    const double t = now_us();
    for (int i = 0; i < B; ++i) {
        Done dn;
        const Request &rq = g.reqs[i];
        dn.r.tag = rq.tag;
        dn.r.k = rq.k;
        dn.r.status = g.status;
        dn.r.latency_us = t - rq.t_submit;
        dn.r.device_us = 0;
        dn.r.device_start_ns = dn.r.device_end_ns = 0;
        dn.ids.assign(kmax, -1);
        dn.dists.assign(kmax, std::numeric_limits<float>::infinity());
        if (g.status == ANN_OK) {
            const ann_query_stats &st = g.h_stats[i];
            dn.r.device_us = (double)(st.t_end_ns - st.t_start_ns) / 1e3;
            dn.r.device_start_ns = st.t_start_ns;
            dn.r.device_end_ns = st.t_end_ns;
            if (st.steps < 0) dn.r.status = ANN_ERR_ARG;
            memcpy(dn.ids.data(), g.h_ids + (size_t)i * kmax, (size_t)kmax * 8);
            memcpy(dn.dists.data(), g.h_dists + (size_t)i * kmax, (size_t)kmax * 4);
        }
        out.push_back(std::move(dn));
    }
    g.reqs.clear();
    g.busy = false;
}

void scheduler(ann_server *s) {
    cudaSetDevice(s->device);
    std::deque<Done> fresh;
    for (;;) {
        bool any_busy = false;
        for (Group &g : s->groups) {
            if (!g.busy) continue;
            const cudaError_t q = cudaEventQuery(g.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (q != cudaSuccess) g.status = ANN_ERR_CUDA;
            harvest_group(s, g, fresh);
        }
        std::unique_lock<std::mutex> lk(s->mu);
        if (!fresh.empty()) {
            for (auto &d : fresh) s->done.push_back(std::move(d));
            fresh.clear();
            s->cv_done.notify_all();
        }
        // admit waiting requests into every free group: the oldest request and the waiting ones of its cost
        // class (queue length L in the same power-of-two range), oldest first, so that short searches do not
        // wait for a long one in the same launch
        for (Group &g : s->groups) {
            if (g.busy || s->npending == 0) continue;
            int cls = -1;
            for (int c = 0; c < ann_server::kClasses; ++c)
                if (!s->pending[c].empty() && (cls < 0 || s->pending[c].front().t_submit < s->pending[cls].front().t_submit))
                    cls = c;
            std::deque<Request> &pq = s->pending[cls];
            while (!pq.empty() && (int)g.reqs.size() < s->cfg.max_batch) {
                g.reqs.push_back(std::move(pq.front()));
                pq.pop_front();
                s->npending--;
            }
            lk.unlock();
            launch_group(s, g);
            any_busy = true;
            lk.lock();
        }
        if (s->stop && s->npending == 0 && !any_busy) break;
        if (any_busy) {
            // poll the groups' events again at once: a timed sleep rounds up to the kernel's timer slack
            // (tens of microseconds), which every request would wait on top of its search
            lk.unlock();
            std::this_thread::yield();
        } else {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->stop || s->npending > 0; });
        }
    }
}

int serve_fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ann::set_error(buf);
    return code;
}

}  // namespace

extern "C" {

int ann_serve_create(const ann_index *index, const ann_serve_config *cfg_in, ann_server **out) {
    if (!out) return serve_fail(ANN_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!index) return serve_fail(ANN_ERR_ARG, "index is NULL");
    ann_serve_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_batch == 0) cfg.max_batch = 1024;
    if (cfg.streams == 0) cfg.streams = 4;
    if (cfg.max_k == 0) cfg.max_k = 100;
    if (cfg.max_L == 0) cfg.max_L = 1024;
    if (cfg.max_M == 0) cfg.max_M = 32;
    if (cfg.max_batch < 1 || cfg.streams < 1 || cfg.streams > 64)
        return serve_fail(ANN_ERR_ARG, "max_batch >= 1 and streams in [1, 64] required");
    if (cfg.max_L < 1 || cfg.max_L > 2048 || cfg.max_k < 1 || cfg.max_k > cfg.max_L || cfg.max_M < 1 || cfg.max_M > 64)
        return serve_fail(ANN_ERR_ARG, "limits max_k=%d max_L=%d max_M=%d outside those of ann_search_ex", cfg.max_k,
                          cfg.max_L, cfg.max_M);
    ann_server *s = new (std::nothrow) ann_server;
    if (!s) return serve_fail(ANN_ERR_OOM, "host allocation");
    s->index = index;
    if (ann_index_get_info(index, &s->info) != ANN_OK) {
        delete s;
        return ANN_ERR_ARG;
    }
    cudaGetDevice(&s->device);
    // admission budget: lower the number of groups until their device state fits
    const size_t per_group = group_device_bytes(cfg.max_batch, s->info.d, cfg.max_k);
    if (cfg.scratch_bytes > 0)
        while (cfg.streams > 1 && (size_t)cfg.streams * per_group > (size_t)cfg.scratch_bytes) cfg.streams--;
    if (cfg.scratch_bytes > 0 && per_group > (size_t)cfg.scratch_bytes) {
        delete s;
        return serve_fail(ANN_ERR_ARG, "one group of %d requests needs %zu device bytes > scratch_bytes %lld",
                          cfg.max_batch, per_group, (long long)cfg.scratch_bytes);
    }
    if (cfg.slots == 0) cfg.slots = 4 * cfg.streams * cfg.max_batch;
    s->cfg = cfg;
    s->groups.resize(cfg.streams);
    for (Group &g : s->groups) {
        cudaError_t e = alloc_group(g, cfg.max_batch, s->info.d, cfg.max_k);
        if (e != cudaSuccess) {
            for (Group &h : s->groups) free_group(h);
            delete s;
            cudaGetLastError();
            return serve_fail(e == cudaErrorMemoryAllocation ? ANN_ERR_OOM : ANN_ERR_CUDA, "group allocation: %s",
                              cudaGetErrorString(e));
        }
    }
    // dry-run the plan for the maxima so unsupported limits fail here, not per request
    {
        ann_search_params p;
        memset(&p, 0, sizeof(p));
        p.mode = cfg.mode;
        p.rerank = cfg.rerank;
        p.R_ratio = 0.8f;
        Group &g = s->groups[0];
        if (ann_search_ex(index, g.d_q, 0, cfg.max_k, cfg.max_L, cfg.max_M, g.d_ids, g.d_dists, &p, g.stream) != ANN_OK) {
            for (Group &h : s->groups) free_group(h);
            delete s;
            return ANN_ERR_ARG;
        }
    }
    try {
        s->th = std::thread(scheduler, s);
    } catch (...) {
        for (Group &h : s->groups) free_group(h);
        delete s;
        return serve_fail(ANN_ERR_STATE, "could not start the scheduler thread");
    }
    *out = s;
    return ANN_OK;
}

void ann_serve_destroy(ann_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Group &g : s->groups) {
        if (g.stream) cudaStreamSynchronize(g.stream);
        free_group(g);
    }
    delete s;
}

int ann_serve_submit(ann_server *s, const float *query, int32_t k, int32_t L, int32_t M, uint64_t tag) {
    if (!s || !query) return serve_fail(ANN_ERR_ARG, "server and query must not be NULL");
    if (k < 1 || L < k || L > s->cfg.max_L || k > s->cfg.max_k || M < 1 || M > s->cfg.max_M)
        return serve_fail(ANN_ERR_ARG, "k=%d L=%d M=%d outside the server limits (k<=%d, k<=L<=%d, M<=%d)", k, L, M,
                          s->cfg.max_k, s->cfg.max_L, s->cfg.max_M);
    Request r;
    r.tag = tag;
    r.k = k;
    r.L = L;
    r.M = M;
    r.q.assign(query, query + s->info.d);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return serve_fail(ANN_ERR_STATE, "server is shutting down");
        if (s->accepted >= s->cfg.slots) return serve_fail(ANN_ERR_BUSY, "all %d request slots are taken", s->cfg.slots);
        r.t_submit = now_us();
        s->pending[cost_class(r.L)].push_back(std::move(r));
        s->npending++;
        s->accepted++;
    }
    s->cv_work.notify_one();
    return ANN_OK;
}

int ann_serve_poll(ann_server *s, ann_result *results, int64_t *out_ids, float *out_dists, int32_t max,
                   int32_t timeout_us) {
    if (!s || !results || !out_ids || !out_dists || max < 1)
        return serve_fail(ANN_ERR_ARG, "server, results and output buffers must be valid and max >= 1");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty()) {
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us),
                            [&] { return !s->done.empty(); });
        if (s->done.empty()) return serve_fail(ANN_ERR_TIMEOUT, "no request completed within %d us", timeout_us);
    }
    const int kmax = s->cfg.max_k;
    int n = 0;
    while (n < max && !s->done.empty()) {
        Done &d = s->done.front();
        results[n] = d.r;
        memcpy(out_ids + (size_t)n * kmax, d.ids.data(), (size_t)kmax * 8);
        memcpy(out_dists + (size_t)n * kmax, d.dists.data(), (size_t)kmax * 4);
        s->done.pop_front();
        s->accepted--;
        n++;
    }
    return n;
}


int ann_serve_replay(ann_server *s, const float *queries, int64_t n_queries, const int64_t *qi, const int32_t *k,
                     const int32_t *L, const int32_t *M, const double *arrival_us, int64_t nreq, double *latency_us,
                     double *device_us, int32_t *status, double *wall_us, int64_t *busy_retries) {
    if (!s || !queries || !qi || !k || !L || !M || !latency_us || !device_us || !status || !wall_us || nreq < 0 ||
        n_queries < 1)
        return serve_fail(ANN_ERR_ARG, "server, queries, trace and output arrays must be valid");
    for (int64_t i = 0; i < nreq; ++i) {
        if (qi[i] < 0 || qi[i] >= n_queries) return serve_fail(ANN_ERR_ARG, "qi[%lld] outside the queries", (long long)i);
        if (arrival_us && (!(arrival_us[i] >= 0.0) || (i > 0 && arrival_us[i] < arrival_us[i - 1])))
            return serve_fail(ANN_ERR_ARG, "arrival_us must be non-negative and non-decreasing");
        latency_us[i] = device_us[i] = std::numeric_limits<double>::quiet_NaN();
        status[i] = ANN_ERR_STATE;  // not completed
    }
    const double t0 = now_us();
    const double deadline = t0 + (nreq && arrival_us ? arrival_us[nreq - 1] : 0.0) + 60e6;
    const int d = s->info.d;
    std::atomic<int64_t> retries{0};
    std::atomic<bool> give_up{false};
    std::atomic<int> submit_rc{ANN_OK};
    std::thread submitter([&] {
        for (int64_t i = 0; i < nreq && !give_up.load(); ++i) {
            if (arrival_us)
                while (now_us() - t0 < arrival_us[i]) {
                }
            for (;;) {
                const int rc = ann_serve_submit(s, queries + (size_t)qi[i] * d, k[i], L[i], M[i], (uint64_t)i);
                if (rc == ANN_OK) break;
                if (rc != ANN_ERR_BUSY || now_us() > deadline || give_up.load()) {
                    submit_rc.store(rc == ANN_ERR_BUSY ? ANN_ERR_TIMEOUT : rc);
                    give_up.store(true);
                    return;
                }
                retries.fetch_add(1);
            }
        }
    });
    const int B = 256;
    std::vector<ann_result> res(B);
    std::vector<int64_t> ids((size_t)B * s->cfg.max_k);
    std::vector<float> dd((size_t)B * s->cfg.max_k);
    int64_t got = 0;
    double t_last = t0;
    while (got < nreq && !give_up.load() && now_us() < deadline) {
        const int n = ann_serve_poll(s, res.data(), ids.data(), dd.data(), B, 1000);
        for (int j = 0; j < n; ++j) {
            const uint64_t t = res[j].tag;
            if (t >= (uint64_t)nreq) continue;
            latency_us[t] = res[j].latency_us;
            device_us[t] = res[j].device_us;
            status[t] = res[j].status;
            ++got;
        }
        if (n > 0) t_last = now_us();
    }
    give_up.store(true);
    submitter.join();
    *wall_us = t_last - t0;
    if (busy_retries) *busy_retries = retries.load();
    if (submit_rc.load() != ANN_OK && got < nreq) {
        const int rc = submit_rc.load();
        return rc == ANN_ERR_TIMEOUT ? serve_fail(ANN_ERR_TIMEOUT, "replay: the server took no request for 60 s")
                                     : rc;
    }
    if (got < nreq) return serve_fail(ANN_ERR_TIMEOUT, "replay: %lld of %lld requests completed in time",
                                      (long long)got, (long long)nreq);
    return ANN_OK;
}

}  // extern "C"
