// search_cluster.cu -- the synchronous top-M search of search_sync.cu with one
// query spread over a thread-block cluster of C CTAs (C = 2, 4 or 8).
//
// Every CTA of the cluster keeps an identical copy of the sorted queue and
// makes the same selection each step (top-M unchecked, Sec. 4.1-4.2). The
// neighbours of the selected vertices are partitioned by owner: vertex u
// belongs to CTA (u mod C), which alone keeps it in its visited table and
// gathers its row, so a step's row gathers are spread over C SMs. Each CTA
// filters its new candidates by the current L-th entry and publishes them in
// shared memory (double-buffered by step parity); after one cluster barrier
// every CTA reads all published lists through distributed shared memory,
// sorts their union, drops ids already queued and merges - the same inputs
// in every CTA, so the queues stay identical and every CTA takes the same
// number of steps and barriers. Because ownership partitions the vertices,
// the union of the CTAs' new candidates is exactly the single-CTA kernel's,
// and the results are identical to it.
#include <cooperative_groups.h>

#include "search_common.cuh"

namespace cg = cooperative_groups;

namespace ann {

struct ClusterCtrl {
    int nact, ncand, qlen, hash_count, anydup, ns, nloc;
    int pub_n[2];       // published survivors per step parity
    int pub_fresh[2];   // new candidates per step parity (for the counters)
    long long steps, expansions, evals, resets, dropped, t0;
};

__host__ __device__ inline int cluster_smem_bytes(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap,
                                                  int *off) {
    int o = 0;
    off[0] = o; o += align16(qfloats * 4);          // query
    off[1] = o; o += align16(Lcap * 8);             // queue
    off[2] = o; o += align16(Lcap * 8);             // next queue
    off[3] = o; o += align16(Ccap * 8);             // local candidates
    off[4] = o; o += align16(Ccap * 8);             // published survivors, parity 0
    off[5] = o; o += align16(Ccap * 8);             // published survivors, parity 1
    off[6] = o; o += align16(Ccap * 8);             // gathered union
    off[7] = o; o += align16(Ccap);                 // dup flags
    off[8] = o; o += align16((1 << hash_bits) * 4); // visited table (own vertices)
    off[9] = o; o += align16(Mcap * 4);             // selected vertices
    return o;
}

template <int NT, int STORE>
__global__ void __launch_bounds__(NT, 1) cluster_search_kernel(const SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ClusterCtrl ctl;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t row_bytes = (uint32_t)a.d_pad * (STORE == ANN_STORE_F32 ? 4u : STORE == ANN_STORE_E4M3 ? 1u : 2u);
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
    int *act = reinterpret_cast<int *>(smem + off[9]);
    const int H = 1 << a.hash_bits;
    const int R = a.R;

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
        ctl.steps = ctl.expansions = ctl.resets = ctl.dropped = 0;
        ctl.evals = 1;
        ctl.pub_n[0] = ctl.pub_n[1] = 0;
    }
    const float *qg = a.queries + (size_t)qi * a.d;
    for (int i = tid; i < a.qfloats; i += NT) qv[i] = i < a.d ? qg[i] : 0.f;
    for (int i = tid; i < H; i += NT) table[i] = kEmptySlot;
    if (tid == 0) cand[0] = (entry_t)(uint32_t)a.entry;
    __syncthreads();
    // the entry point: every CTA computes the same key; its owner marks it visited
    compute_keys<STORE, NT>(a.base, a.scales, a.d_pad, a.metric, qv, cand, 1);
    __syncthreads();
    if (tid == 0) {
        Q[0] = cand[0];
        ctl.qlen = 1;
        ctl.hash_count = 0;
        if ((int)(a.entry % C) == rank) {
            visited_insert(table, a.hash_bits, (uint32_t)a.entry);
            ctl.hash_count = 1;
        }
    }
    __syncthreads();

    int Mcur = a.M0 < Mmax ? a.M0 : Mmax;
    int step = 0;
    for (;;) {
        const int qlen = ctl.qlen;
        if (ctl.hash_count * 2 > H) {  // forget own vertices when half full (keep own queued ids)
            for (int i = tid; i < H; i += NT) table[i] = kEmptySlot;
            __syncthreads();
            for (int i = tid; i < qlen; i += NT) {
                const uint32_t u = entry_id(Q[i]);
                if ((int)(u % C) == rank) visited_insert(table, a.hash_bits, u);
            }
            __syncthreads();
            if (tid == 0) {
                int own = 0;
                for (int i = 0; i < qlen; ++i) own += (int)(entry_id(Q[i]) % C) == rank;
                ctl.hash_count = own;
                ctl.resets++;
            }
        }
        if (warp == 0) {
            int found = 0;
            for (int b = 0; b < qlen && found < Mcur; b += 32) {
                const int i = b + lane;
                const entry_t e = i < qlen ? Q[i] : kChecked;
                const bool un = !(e & kChecked);
                const unsigned bal = __ballot_sync(kFull, un);
                const int r = found + __popc(bal & ((1u << lane) - 1u));
                if (un && r < Mcur) {
                    act[r] = (int)entry_id(e);
                    Q[i] = e | kChecked;
                }
                found += __popc(bal);
            }
            if (lane == 0) {
                ctl.nact = found < Mcur ? found : Mcur;
                ctl.ncand = 0;
                ctl.nloc = 0;
            }
        }
        __syncthreads();
        const int nact = ctl.nact;
        if (nact == 0) break;  // identical in every CTA: all leave the loop at the same step
        step++;
        const int par = step & 1;
        if (tid == 0) {
            ctl.steps++;
            ctl.expansions += nact;
        }
        // own neighbours of the selected vertices -> visited filter -> local candidates
        const int total = nact * R;
        for (int b = warp * 32; b < total; b += NT) {
            const int i = b + lane;
            int u = -1;
            if (i < total) {
                const int aidx = i / R, r = i - aidx * R;
                u = __ldg(a.adj + (size_t)act[aidx] * R + r);
                if (u >= 0 && (u % C) != rank) u = -1;
            }
            const bool fresh = u >= 0 && visited_insert(table, a.hash_bits, (uint32_t)u) != 0;
            const unsigned bal = __ballot_sync(kFull, fresh);
            int basepos = 0;
            if (lane == 0 && bal) basepos = atomicAdd(&ctl.ncand, __popc(bal));
            basepos = __shfl_sync(kFull, basepos, 0);
            if (fresh) {
                cand[basepos + __popc(bal & ((1u << lane) - 1u))] = (entry_t)(uint32_t)u;
                if (a.l2_prefetch) prefetch_row_l2(a.base, row_bytes, (uint32_t)u);
            }
        }
        __syncthreads();
        const int nc = ctl.ncand;
        if (tid == 0) ctl.hash_count += nc;
        const entry_t limit = qlen >= L ? (Q[L - 1] & kMask) : kEmptyEntry;
        if (nc > 0)
            compute_keys_teams<STORE, NT>(a.base, a.scales, a.d_pad, a.metric, qv, cand, nc, a.team_lanes, limit,
                                          pub[par], &ctl.nloc);
        __syncthreads();
        if (tid == 0) {
            ctl.pub_n[par] = ctl.nloc;
            ctl.pub_fresh[par] = nc;
        }
        cluster.sync();  // every CTA's survivors of this step are published
        // gather the union in rank order (the same order in every CTA)
        int tot = 0;
        for (int r = 0; r < C; ++r) {
            const int *rn = cluster.map_shared_rank(&ctl.pub_n[par], r);
            const entry_t *rp = cluster.map_shared_rank(pub[par], r);
            const int n = *rn;
            for (int i = tid; i < n; i += NT) uni[tot + i] = rp[i];
            tot += n;
            if (tid == 0 && rank == 0) ctl.evals += *cluster.map_shared_rank(&ctl.pub_fresh[par], r);
        }
        __syncthreads();
        if (tot > 0) {
            if (tot <= 32) {
                if (warp == 0) {
                    entry_t e = lane < tot ? uni[lane] : kEmptyEntry;
                    e = warp_sort32(e);
                    uni[lane] = e;
                }
                __syncthreads();
            } else {
                int P = 64;
                while (P < tot) P <<= 1;
                for (int i = tot + tid; i < P; i += NT) uni[i] = kEmptyEntry;
                __syncthreads();
                block_bitonic_sort<NT>(uni, P);
            }
            long long dropped = 0;
            const int nl = block_merge_dedupe<NT>(Q, qlen, uni, tot, L, Qn, dup, &ctl.anydup, &dropped);
            if (tid == 0) {
                ctl.dropped += dropped;
                ctl.qlen = nl;
            }
            entry_t *t = Q;
            Q = Qn;
            Qn = t;
        }
        __syncthreads();
        if (step % a.t == 0) Mcur = min(2 * Mcur, Mmax);
    }

    // output from rank 0 (optionally re-ranked with FP32 rows)
    if (rank == 0) {
        const int qlen = ctl.qlen;
        const entry_t *res = Q;
        if (a.rerank) {
            for (int i = tid; i < qlen; i += NT) {
                const uint32_t id = entry_id(Q[i]);
                cand[i] = (entry_t)id;
                if (a.l2_prefetch) prefetch_row_l2(a.base32, (uint32_t)a.d_pad32 * 4u, id);
            }
            __syncthreads();
            compute_keys<ANN_STORE_F32, NT>(a.base32, nullptr, a.d_pad32, a.metric, qv, cand, qlen);
            int P = 32;
            while (P < qlen) P <<= 1;
            for (int i = qlen + tid; i < P; i += NT) cand[i] = kEmptyEntry;
            __syncthreads();
            block_bitonic_sort<NT>(cand, P);
            res = cand;
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
            st.evals = ctl.evals;
            st.hash_resets = ctl.resets;
            st.dup_dropped = ctl.dropped;
            st.merges = 0;
            st.t_start_ns = ctl.t0;
            st.t_end_ns = global_ns();
            a.stats[qi] = st;
        }
    }
    cluster.sync();  // no CTA leaves while another may still read its shared memory
}

int cluster_smem_size(int qfloats, int Lcap, int Ccap, int hash_bits, int Mcap) {
    int off[10];
    return cluster_smem_bytes(qfloats, Lcap, Ccap, hash_bits, Mcap, off);
}

template <int NT, int STORE>
static cudaError_t claunch_t(const SearchArgs &a, int smem, int csize, cudaStream_t s) {
    auto fn = cluster_search_kernel<NT, STORE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
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
