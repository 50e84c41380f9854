// search_cluster.cu -- the synchronous top-M search of search_sync.cuh with one
// query spread over a thread-block cluster of C CTAs (C = 2, 4 or 8): the
// latency form, for few queries at a time.
//
// Every CTA of the cluster keeps an identical copy of the sorted queue and
// makes the same selection each step (top-M unchecked, Sec. 4.1-4.2). The
// step's adjacency slots are split over each CTA's warps as in the one-CTA
// kernel, but vertex u belongs to CTA (u mod C): only its owner inserts it
// into its visited set and gathers its row, so a step's row gathers are
// spread over C SMs. Each CTA filters its new candidates by the current L-th
// entry and publishes them in shared memory (double-buffered by step parity);
// after one cluster barrier every CTA reads all published lists through
// distributed shared memory, sorts their union, drops ids already queued
// (when some owner's visited set forgot a vertex) and merges: the same inputs
// in every CTA, so the queues stay identical and every CTA takes the same
// number of steps and barriers. Because ownership partitions the vertices,
// the union of the CTAs' new candidates is exactly the one-CTA kernel's, and
// the results are identical to it.
#include <cooperative_groups.h>

#include "search_common.cuh"

namespace cg = cooperative_groups;

namespace ann {

struct ClusterCtrl {
    int pub_n[2];      // survivors published in the step of this parity
    int pub_fresh[2];  // fresh vertices of this CTA in the step of this parity
    int pub_unsafe[2]; // this CTA's visited set may have forgotten a vertex (as of this step)
    int unsafe, anydup, first_un, sel_last, wevals;
    int wcnt[32];      // per-warp counts of the selection scan
    int rr_n;          // re-rank keys appended (rank 0, after the search; never read by another CTA)
    long long steps, expansions, dropped, t0;
    long long ph[4], tmark;  // rank 0's phase cycles (select, expand + distance, exchange, sort + merge)
};

// Segments: query, two queue buffers, per-warp fresh lists (then sort
// scratch), published survivors (two parities), the gathered union, dedupe
// flags, the visited set (this CTA's vertices) and the selection.
__host__ __device__ inline int cluster_smem_bytes(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap,
                                                  int *off) {
    int o = 0;
    off[0] = o; o += align16(qfloats * 4);          // query
    off[1] = o; o += align16(Lcap * 8);             // queue
    off[2] = o; o += align16(Lcap * 8);             // next queue
    off[3] = o; o += align16(Ccap * 8);             // fresh (id, row) pairs; sort scratch; re-rank ids
    off[4] = o; o += align16(Ccap * 8);             // published survivors, parity 0
    off[5] = o; o += align16(Ccap * 8);             // published survivors, parity 1
    off[6] = o; o += align16(Ccap * 8);             // gathered union; re-rank keys
    off[7] = o; o += align16(Ccap);                 // dup flags
    off[8] = o; o += align16((1 << hash_bits) * 4); // visited set (own vertices)
    off[9] = o; o += align16(2 * Mcap * 4);         // selected vertices and their queue positions
    return o;
}

template <int NT, int STORE, bool L2>
__global__ void __launch_bounds__(NT, 1) cluster_search_kernel(const SearchArgs a) {
    constexpr int NW = NT / 32;
    constexpr uint32_t ES = STORE == ANN_STORE_F32 ? 4u : STORE == ANN_STORE_E4M3 ? 1u : 2u;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClusterCtrl ctl;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t row_bytes = (uint32_t)a.d_pad * ES;
    const uint32_t cpr = row_bytes / 16u;
    int off[10];
    cluster_smem_bytes(a.qfloats, a.Lcap, a.Ccap, a.hash_bits, a.M, off);
    float *qv = reinterpret_cast<float *>(smem + off[0]);
    entry_t *Q = reinterpret_cast<entry_t *>(smem + off[1]);
    entry_t *Qn = reinterpret_cast<entry_t *>(smem + off[2]);
    entry_t *cand = reinterpret_cast<entry_t *>(smem + off[3]);
    entry_t *pub[2] = {reinterpret_cast<entry_t *>(smem + off[4]), reinterpret_cast<entry_t *>(smem + off[5])};
    entry_t *uni = reinterpret_cast<entry_t *>(smem + off[6]);
    unsigned char *dup = smem + off[7];
    uint32_t *table = reinterpret_cast<uint32_t *>(smem + off[8]);
    int *sel_id = reinterpret_cast<int *>(smem + off[9]);
    int *sel_pos = sel_id + a.M;
    const int H = 1 << a.hash_bits;
    const int R = a.R;
    const int slots_w = (a.M * R + NW - 1) / NW;
    uint2 *fresh = reinterpret_cast<uint2 *>(cand) + (size_t)warp * slots_w;
    const uint32_t r_recip = 0xFFFFFFFFu / (uint32_t)R + 1u;

    // one query per cluster; identical in every CTA of the cluster
    const int item = (int)(blockIdx.x / C);
    const bool live = item < a.nq;
    const int qi = live ? (a.order ? a.order[item] : item) : 0;
    const int k = live ? (a.k_arr ? a.k_arr[qi] : a.k) : 1;
    const int L = live ? (a.L_arr ? a.L_arr[qi] : a.L) : 1;
    const int Mmax = live ? (a.M_arr ? a.M_arr[qi] : a.M) : 1;
    const bool bad = !live || k < 1 || k > a.k || L < k || L > a.L || Mmax < 1 || Mmax > a.M;
    if (bad) {
        if (live && rank == 0) {
            for (int i = tid; i < a.k; i += NT) {
                a.out_ids[(size_t)qi * a.k + i] = -1;
                a.out_dists[(size_t)qi * a.k + i] = __int_as_float(0x7f800000);
            }
            if (tid == 0 && a.stats) {
                ann_query_stats st = {};
                st.steps = -1;
                a.stats[qi] = st;
            }
        }
        cluster.sync();
        return;
    }

    if (tid == 0) {
        ctl.t0 = global_ns();
        ctl.steps = ctl.expansions = ctl.dropped = 0;
        ctl.pub_n[0] = ctl.pub_n[1] = 0;
        ctl.pub_fresh[0] = ctl.pub_fresh[1] = 0;
        ctl.unsafe = 0;
        ctl.first_un = 0;
        ctl.wevals = 0;
        ctl.ph[0] = ctl.ph[1] = ctl.ph[2] = ctl.ph[3] = 0;
    }
    const float *qg = a.queries + (size_t)qi * a.d;
    for (int i = tid; i < a.qfloats; i += NT) qv[i] = i < a.d ? qg[i] : 0.f;
    {
        const uint32_t empty = a.ways ? 0u : kEmptySlot;
        for (int i = tid; i < H; i += NT) table[i] = empty;
    }
    if (tid == 0) fresh[0] = make_uint2((uint32_t)a.entry, (uint32_t)a.entry);
    __syncthreads();
    // the entry point: every CTA computes the same key; its owner marks it visited
    if (warp == 0)
        warp_keys_append_m<STORE, 4, L2>(a.base, a.scales, cpr, qv, fresh, 1, a.team_lanes, kEmptyEntry, uni,
                                         &ctl.pub_n[1]);
    __syncthreads();
    if (tid == 0) {
        Q[0] = uni[0];
        ctl.pub_n[1] = 0;
        if ((int)(a.entry % C) == rank) visit_set(table, a, (uint32_t)a.entry);
    }
    __syncthreads();

    int Mcur = a.M0 < Mmax ? a.M0 : Mmax;
    int step = 0;
    int qlen = 1;
    const bool prof = a.phase_cycles != nullptr && rank == 0;
    if (prof && tid == 0) ctl.tmark = clock64();
#define ANN_CPHASE(i)                                  \
    if (prof && tid == 0) {                            \
        const long long now_ = clock64();              \
        ctl.ph[i] += now_ - ctl.tmark;                 \
        ctl.tmark = now_;                              \
    }
    for (;;) {
        const int par = step & 1;
        // --- select (every CTA, identical): the first Mcur unchecked entries, all warps scanning
        const int found = select_step<NW>(Q, qlen, ctl.first_un, Mcur, sel_id, sel_pos, ctl.wcnt,
                                               &ctl.sel_last);
        ANN_CPHASE(0)
        const int nact = found < Mcur ? found : Mcur;
        if (nact == 0) break;  // identical in every CTA: all leave the loop at the same step
        step++;

        // --- this CTA's own neighbours: adjacency -> visited set -> fresh lists -> distances -> published
        const int nf = expand_step<NW>(a, table, sel_id, nact, r_recip, row_bytes, fresh, nullptr, nullptr, C, rank,
                                       &ctl.unsafe);
        if (lane == 0 && nf) atomicAdd(&ctl.wevals, nf);
        const entry_t limit = qlen >= L ? (Q[L - 1] & kMask) : kEmptyEntry;
        if (!gather_fixed<STORE, L2>(a.base, a.scales, cpr, a.team_lanes, qv, nullptr, fresh, nf, 0, 1, limit,
                                     pub[par], &ctl.pub_n[par]))
            warp_keys_append_m<STORE, 4, L2>(a.base, a.scales, cpr, qv, fresh, nf, a.team_lanes, limit, pub[par],
                                             &ctl.pub_n[par]);
        __syncthreads();
        if (tid == 0) ctl.pub_unsafe[par] = ctl.unsafe;
        ANN_CPHASE(1)
        cluster.sync();  // every CTA's survivors of this step are published
        // gather the union in rank order (the same order in every CTA): every thread reads all
        // counts at once, then copies its share of all lists in one pass (two remote round trips)
        int cn[8];
        int tot = 0, any_unsafe = 0;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            cn[r] = 0;
            if (r < C) {
                cn[r] = *cluster.map_shared_rank(&ctl.pub_n[par], r);
                any_unsafe |= *cluster.map_shared_rank(&ctl.pub_unsafe[par], r);
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) tot += cn[r];
        for (int i = tid; i < tot; i += NT) {
            int r = 0, base_r = 0;
#pragma unroll
            for (int rr = 0; rr < 7; ++rr)
                if (r == rr && i - base_r >= cn[rr]) {
                    base_r += cn[rr];
                    r = rr + 1;
                }
            uni[i] = cluster.map_shared_rank(pub[par], r)[i - base_r];
        }
        if (tid < nact) Q[sel_pos[tid]] |= kChecked;  // the selection is taken: mark it
        if (tid == 0) {
            ctl.pub_n[par ^ 1] = 0;  // the next step's list (every CTA read it before this step's barrier)
            ctl.steps++;
            ctl.expansions += nact;
            ctl.first_un = ctl.sel_last + 1;
        }
        __syncthreads();
        ANN_CPHASE(2)
        if (tot > 0) {
            const int ncl = sort_dedupe_merge<NT>(Q, qlen, uni, tot, cand, Qn, L, any_unsafe != 0, dup, &ctl.anydup,
                                                  &ctl.dropped, &ctl.first_un);
            qlen = min(L, qlen + ncl);
            entry_t *t = Q;
            Q = Qn;
            Qn = t;
        } else {
            __syncthreads();
        }
        ANN_CPHASE(3)
        if (step % a.t == 0) Mcur = min(2 * Mcur, Mmax);
    }
#undef ANN_CPHASE

    // distance evaluations of the whole cluster: every CTA's own fresh vertices (read before the last barrier)
    long long evals = 1;
    if (rank == 0 && tid == 0)
        for (int r = 0; r < C; ++r) evals += *cluster.map_shared_rank(&ctl.wevals, r);
    // output from rank 0 (optionally re-ranked with FP32 rows)
    if (rank == 0) {
        const entry_t *res = Q;
        if (a.rerank) {
            for (int i = tid; i < qlen; i += NT) {
                const uint32_t id = entry_id(Q[i]);
                cand[i] = (entry_t)id;
                if (a.l2_prefetch) prefetch_row_l2(a.base32, (uint32_t)a.d_pad32 * 4u, id);
            }
            if (tid == 0) ctl.rr_n = 0;
            __syncthreads();
            if (!gather_fixed<ANN_STORE_F32, L2>(a.base32, nullptr, (uint32_t)a.d_pad32 / 4u, a.team_lanes32, qv,
                                                 cand, nullptr, qlen, warp, NW, kEmptyEntry, uni, &ctl.rr_n))
                compute_keys_teams_m<ANN_STORE_F32, NT, L2, 2>(a.base32, nullptr, a.d_pad32, qv, cand, qlen,
                                                               a.team_lanes32, kEmptyEntry, uni, &ctl.rr_n);
            __syncthreads();
            if (k <= 32) {
                res = block_topk<NT>(uni, qlen, k, cand, uni);
            } else {
                int P = 32;
                while (P < qlen) P <<= 1;
                for (int i = qlen + tid; i < P; i += NT) uni[i] = kEmptyEntry;
                __syncthreads();
                block_bitonic_sort<NT>(uni, P);
                res = uni;
            }
        }
        int64_t *oid = a.out_ids + (size_t)qi * a.k;
        float *odist = a.out_dists + (size_t)qi * a.k;
        for (int i = tid; i < a.k; i += NT) {
            if (i < k && i < qlen) {
                oid[i] = (int64_t)entry_id(res[i]);
                odist[i] = entry_key(res[i]);
            } else {
                oid[i] = -1;
                odist[i] = __int_as_float(0x7f800000);
            }
        }
        if (tid == 0 && a.stats) {
            ann_query_stats st;
            st.steps = ctl.steps;
            st.expansions = ctl.expansions;
            st.evals = evals;
            st.hash_resets = 0;
            st.dup_dropped = ctl.dropped;
            st.merges = 0;
            st.t_start_ns = ctl.t0;
            st.t_end_ns = global_ns();
            a.stats[qi] = st;
        }
        if (tid == 0 && prof)
            for (int i = 0; i < 4; ++i) a.phase_cycles[(size_t)qi * 4 + i] = ctl.ph[i];
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

int cluster_smem_size(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap) {
    int off[10];
    return cluster_smem_bytes(qfloats, Lcap, Ccap, hash_bits, Mcap, off);
}

template <int NT, int STORE>
static cudaError_t claunch_t(const SearchArgs &a, int smem, int csize, cudaStream_t s) {
    auto fn = a.metric == ANN_METRIC_L2 ? cluster_search_kernel<NT, STORE, true> : cluster_search_kernel<NT, STORE, false>;
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.nq * csize));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

#define ANN_CLUSTER_STORE(NT, ...)                                             \
    switch (storage) {                                                         \
        case ANN_STORE_F32: return claunch_t<NT, ANN_STORE_F32>(__VA_ARGS__);   \
        case ANN_STORE_BF16: return claunch_t<NT, ANN_STORE_BF16>(__VA_ARGS__); \
        case ANN_STORE_F16: return claunch_t<NT, ANN_STORE_F16>(__VA_ARGS__);   \
        case ANN_STORE_E4M3: return claunch_t<NT, ANN_STORE_E4M3>(__VA_ARGS__); \
    }                                                                          \
    return cudaErrorInvalidValue;

cudaError_t launch_cluster_search(const SearchArgs &a, int storage, int threads, int smem, int csize,
                                  cudaStream_t s) {
    switch (threads) {
        case 128: ANN_CLUSTER_STORE(128, a, smem, csize, s)
        case 256: ANN_CLUSTER_STORE(256, a, smem, csize, s)
        case 512: ANN_CLUSTER_STORE(512, a, smem, csize, s)
    }
    return cudaErrorInvalidValue;
}

}  // namespace ann
