// search_sync.cu -- bulk-synchronous top-M best-first search, one CTA per query.
//
// Follows Algorithm 1 (BFiS) generalised by Sec. 4.1 to expand the top-M
// unchecked candidates per step, with the Sec. 4.2 staged schedule (M starts
// at M0 and doubles every t steps up to M_max). Every step is a CTA barrier,
// so the result is deterministic: it is the same top-L queue the sequential
// definition produces, whatever order the warps touch it in.
//
// Per step, inside one CTA:
//   select   warp 0 takes the first min(M_s, #unchecked) unchecked entries of
//            the sorted queue by ballot + popc and marks them checked;
//   expand   all threads read the M adjacency rows (coalesced int32 rows) and
//            insert each neighbour into the shared-memory visited table;
//            survivors get a slot in the candidate buffer (warp-aggregated
//            atomics);
//   distance teams of lanes gather the candidates' rows with 16-byte
//            non-caching loads and reduce partial sums with shuffles;
//   sort     bitonic sort of the packed (key, id) candidates;
//   merge    drop candidates whose id is already queued (only possible after
//            the visited table forgot a vertex), then a rank-based parallel
//            merge of the queue and the candidates, truncated to L.
// The visited table is reset to the queue's ids when it is half full; the
// queue is then still the top-L of everything seen (a forgotten vertex that
// is met again either duplicates a queued id, which the merge drops, or ranks
// below the L-th entry again), so ids are unchanged and only the distance
// count grows.
#include "search_common.cuh"

namespace ann {

struct Ctrl {
    int nact;
    int ncand;
    int qlen;
    int hash_count;
    int anydup;
    int ns;      // candidates that beat the L-th queued entry this step
    int unsafe;  // 1 once the visited table may have forgotten a vertex this query
    int qi;
    // per-query counters, updated by thread 0 only
    long long steps, expansions, evals, resets, dropped, t0;
    long long ph[4], tmark;  // phase cycles (select, expand, distance, sort+merge) when requested
};

// One insert into the query's visited set, whichever form it has: 0 = was
// present, 1 = inserted, 2 or 3 = inserted while another vertex may have been
// forgotten (probe limit, eviction).
__device__ __forceinline__ int visit_set(uint32_t *table, const SearchArgs &a, uint32_t id) {
    if (a.visited_mode == 0) return visited_insert(table, a.hash_bits, id);
    if (a.slot_bytes == 1) return visited_tag<1>(table, a.hash_bits, a.tag_bits, id);
    if (a.slot_bytes == 2) return visited_tag<2>(table, a.hash_bits, a.tag_bits, id);
    return visited_exchange(table, a.hash_bits, id);
}

template <int NT, int STORE>
__global__ void __launch_bounds__(NT, 65536 / (NT * 64)) sync_search_kernel(const SearchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Ctrl ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int row_bytes = a.d_pad * (STORE == ANN_STORE_F32 ? 4 : STORE == ANN_STORE_E4M3 ? 1 : 2);
    const SmemLayout lay = sync_layout(a.qfloats, a.Lcap, a.Ccap, a.hash_bits, a.M,
                                       a.tma_rows * row_bytes + a.pipe_bytes, a.slot_bytes);
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(smem + lay.bar_off);
    unsigned char *stage = smem + lay.stage_off;
    unsigned parity = 0;
    if (a.tma_rows > 0) {
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
    }
    float *qv = reinterpret_cast<float *>(smem + lay.q_off);
    entry_t *Qa = reinterpret_cast<entry_t *>(smem + lay.q0_off);
    entry_t *Qb = reinterpret_cast<entry_t *>(smem + lay.q1_off);
    entry_t *cand = reinterpret_cast<entry_t *>(smem + lay.cand_off);
    entry_t *surv = reinterpret_cast<entry_t *>(smem + lay.cand2_off);
    unsigned char *dup = smem + lay.dup_off;
    uint32_t *table = reinterpret_cast<uint32_t *>(smem + lay.hash_off);
    int *act = reinterpret_cast<int *>(smem + lay.act_off);
    const int H = 1 << a.hash_bits;
    const int R = a.R;

    for (;;) {
        if (tid == 0) {
            const int item = a.persistent ? atomicAdd(a.work_counter, 1) : (int)blockIdx.x;
            ctl.qi = item >= a.nq ? -1 : (a.order ? a.order[item] : item);
            ctl.t0 = global_ns();
            ctl.steps = ctl.expansions = ctl.resets = ctl.dropped = 0;
            ctl.evals = 1;
            ctl.unsafe = 0;
            ctl.ph[0] = ctl.ph[1] = ctl.ph[2] = ctl.ph[3] = 0;
        }
        __syncthreads();
        const int qi = ctl.qi;
        if (qi < 0) break;  // work list exhausted

        const int k = a.k_arr ? a.k_arr[qi] : a.k;
        const int L = a.L_arr ? a.L_arr[qi] : a.L;
        const int Mmax = a.M_arr ? a.M_arr[qi] : a.M;
        const bool bad = k < 1 || k > a.k || L < k || L > a.L || Mmax < 1 || Mmax > a.M;
        if (bad) {
            for (int i = tid; i < a.k; i += NT) {
                a.out_ids[(size_t)qi * a.k + i] = -1;
                a.out_dists[(size_t)qi * a.k + i] = __int_as_float(0x7f800000);
            }
            if (tid == 0 && a.stats) {
                ann_query_stats st = {};
                st.steps = -1;
                a.stats[qi] = st;
            }
            if (!a.persistent) break;
            __syncthreads();
            continue;
        }

        // query into shared memory, zero padded; clear the visited table
        const float *qg = a.queries + (size_t)qi * a.d;
        for (int i = tid; i < a.qfloats; i += NT) qv[i] = i < a.d ? qg[i] : 0.f;
        {
            const int words = (H * a.slot_bytes) >> 2;
            const uint32_t empty = a.slot_bytes < 4 ? 0u : kEmptySlot;
            for (int i = tid; i < words; i += NT) table[i] = empty;
        }
        if (tid == 0) {
            cand[0] = (entry_t)(uint32_t)a.entry;
            ctl.ns = 0;
        }
        __syncthreads();
        // the entry point P: distance, queue = [P], visited = {P}
        compute_keys_teams<STORE, NT>(a.base, a.scales, a.d_pad, a.metric, qv, cand, 1, a.team_lanes, kEmptyEntry,
                                      surv, &ctl.ns);
        __syncthreads();
        if (tid == 0) {
            Qa[0] = surv[0];
            visit_set(table, a, (uint32_t)a.entry);
            ctl.hash_count = 1;
        }
        __syncthreads();

        int Mcur = a.M0 < Mmax ? a.M0 : Mmax;
        int step = 0;
        int qlen = 1;  // the same in every thread
        entry_t *Q = Qa, *Qn = Qb;
        const bool prof = a.phase_cycles != nullptr;
        if (prof && tid == 0) ctl.tmark = clock64();
#define ANN_PHASE(i)                                   \
    if (prof && tid == 0) {                            \
        const long long now_ = clock64();              \
        ctl.ph[i] += now_ - ctl.tmark;                 \
        ctl.tmark = now_;                              \
    }
        for (;;) {
            // --- forget the visited table when half full (keep the queued ids);
            // the direct-mapped cache never resets, it forgets by eviction
            if (a.visited_mode == 0 && ctl.hash_count * 2 > H) {
                for (int i = tid; i < H; i += NT) table[i] = kEmptySlot;
                __syncthreads();
                for (int i = tid; i < qlen; i += NT) visited_insert(table, a.hash_bits, entry_id(Q[i]));
                if (tid == 0) {
                    ctl.hash_count = qlen;
                    ctl.resets++;
                    ctl.unsafe = 1;
                }
            }
            // --- select the first Mcur unchecked entries (rank order) and mark them
            if (warp == 0) {
                int found = 0;
                for (int b = 0; b < qlen && found < Mcur; b += 32) {
                    const int i = b + lane;
                    entry_t e = i < qlen ? Q[i] : kChecked;
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
                    ctl.anydup = 0;
                    ctl.ns = 0;
                }
            }
            __syncthreads();
            ANN_PHASE(0)
            const int nact = ctl.nact;
            if (nact == 0) break;  // no unchecked vertex left
            step++;
            if (tid == 0) {
                ctl.steps++;
                ctl.expansions += nact;
            }

            // --- expand: adjacency rows -> visited filter -> candidate ids
            {
                // Each thread issues all of its adjacency loads (up to four ids), then all of its visited
                // updates, then the warp appends its fresh vertices with one scan and one atomic. The thread
                // that finds a fresh vertex also asks L2 for its row.
                constexpr int KA = 4;
                const int total = nact * R;
                for (int b0 = warp * 32; b0 < total; b0 += NT * KA) {
                    int u[KA];
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        const int i = b0 + k * NT + lane;
                        u[k] = -1;
                        if (i < total) {
                            const int aidx = i / R, r = i - aidx * R;
                            u[k] = __ldg(a.adj + (size_t)act[aidx] * R + r);
                        }
                    }
                    unsigned fresh = 0;  // bit k: u[k] was not in the visited set
                    bool forgot = false;
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        if (u[k] >= 0) {
                            const int ins = visit_set(table, a, (uint32_t)u[k]);
                            if (ins != 0) fresh |= 1u << k;
                            if (ins >= 2) forgot = true;
                        }
                    }
                    if (forgot) ctl.unsafe = 1;  // a vertex may have been forgotten: repeats possible
                    const int cnt = __popc(fresh);
                    int incl = cnt;  // inclusive scan of the per-lane counts
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const int v = __shfl_up_sync(kFull, incl, off);
                        if (lane >= off) incl += v;
                    }
                    int base = 0;
                    if (lane == 31 && incl > 0) base = atomicAdd(&ctl.ncand, incl);
                    int pos = __shfl_sync(kFull, base, 31) + incl - cnt;
#pragma unroll
                    for (int k = 0; k < KA; ++k) {
                        if (fresh >> k & 1u) {
                            cand[pos++] = (entry_t)(uint32_t)u[k];
                            if (a.l2_prefetch) prefetch_row_l2(a.base, row_bytes, (uint32_t)u[k]);
                        }
                    }
                }
            }
            __syncthreads();
            ANN_PHASE(1)
            const int nc = ctl.ncand;
            if (tid == 0) {
                ctl.hash_count += nc;
                ctl.evals += nc;
            }
            if (nc > 0) {
                // --- distances; only candidates below the L-th queued entry survive
                const entry_t limit = qlen >= L ? (Q[L - 1] & kMask) : kEmptyEntry;
                if (STORE != ANN_STORE_E4M3 && a.tma_rows > 0) {
                    if (!compute_keys_tma<STORE, NT>(a.base, a.d_pad, a.metric, qv, cand, nc, stage, a.tma_rows, bar,
                                                     &parity, limit, surv, &ctl.ns)) {
                        // a staging batch never arrived: fail this query, let the copies land, stop
                        mbar_wait(bar, parity ^ 1u, 1 << 22);
                        for (int i = tid; i < a.k; i += NT) {
                            a.out_ids[(size_t)qi * a.k + i] = -1;
                            a.out_dists[(size_t)qi * a.k + i] = __int_as_float(0x7f800000);
                        }
                        if (tid == 0 && a.stats) {
                            ann_query_stats st = {};
                            st.steps = -2;
                            a.stats[qi] = st;
                        }
                        return;
                    }
                } else if (STORE != ANN_STORE_E4M3 && a.pipe_bytes > 0) {
                    compute_keys_pipe<STORE, NT>(a.base, a.scales, a.d_pad, a.metric, qv, cand, nc, stage, limit, surv,
                                                 &ctl.ns);
                    __syncthreads();
                } else {
                    // four chunks in flight per lane: a few spilled registers outside the gather loop cost less
                    // than a second round trip per row (measured 3-4 % faster than two)
                    compute_keys_teams<STORE, NT, 4>(a.base, a.scales, a.d_pad, a.metric, qv, cand, nc, a.team_lanes,
                                                  limit, surv, &ctl.ns);
                    __syncthreads();
                }
                ANN_PHASE(2)
                const int ns = ctl.ns;
                if (ns > 0) {
                    // --- sort the survivors by (key, id) into srt
                    entry_t *srt = surv;
                    if (ns <= 32) {
                        if (warp == 0) {
                            entry_t e = lane < ns ? surv[lane] : kEmptyEntry;
                            e = warp_sort32(e);
                            surv[lane] = e;
                        }
                        __syncthreads();
                    } else if (ns > 64 && ns <= NT) {
                        // two barriers instead of a bitonic sort's dozen (at 64 or fewer the bitonic one is as cheap)
                        block_rank_sort<NT>(surv, ns, cand);  // the candidate ids are not needed any more
                        srt = cand;
                    } else {
                        int P = 64;
                        while (P < ns) P <<= 1;
                        for (int i = ns + tid; i < P; i += NT) surv[i] = kEmptyEntry;
                        __syncthreads();
                        block_bitonic_sort<NT>(surv, P);
                    }
                    int ncl = ns;
                    if (ctl.unsafe) {
                        // --- drop ids already queued or repeated (only after the table forgot)
                        int any = 0;
                        for (int j = tid; j < ns; j += NT) {
                            const entry_t c = srt[j];
                            bool d = (j > 0 && srt[j - 1] == c);
                            if (!d) {
                                const int pos = count_below(Q, qlen, c);
                                d = pos < qlen && (Q[pos] & kMask) == c;
                            }
                            dup[j] = d;
                            any |= d;
                        }
                        if (__syncthreads_or(any)) {
                            if (warp == 0) {
                                int outp = 0;
                                for (int b = 0; b < ns; b += 32) {
                                    const int j = b + lane;
                                    const bool keep = j < ns && !dup[j];
                                    const entry_t c = j < ns ? srt[j] : 0ull;
                                    const unsigned bal = __ballot_sync(kFull, keep);
                                    if (keep) srt[outp + __popc(bal & ((1u << lane) - 1u))] = c;
                                    outp += __popc(bal);
                                }
                                if (lane == 0) ctl.anydup = outp;
                            }
                            __syncthreads();
                            ncl = ctl.anydup;
                            if (tid == 0) ctl.dropped += ns - ncl;
                        }
                    }
                    // --- merge queue and survivors, truncated to L (merge path: one search per thread)
                    block_merge_path<NT>(Q, qlen, srt, ncl, Qn, L);
                    __syncthreads();  // the new queue is complete; nothing of the old one is read again
                    qlen = min(L, qlen + ncl);
                    entry_t *tmp = Q;
                    Q = Qn;
                    Qn = tmp;
                }
            }
            ANN_PHASE(3)
            if (step % a.t == 0) Mcur = min(2 * Mcur, Mmax);
        }
#undef ANN_PHASE

        // --- output: first k of the queue, optionally re-ranked with FP32 rows
        const entry_t *res = Q;
        if (a.rerank) {
            for (int i = tid; i < qlen; i += NT) {
                const uint32_t id = entry_id(Q[i]);
                cand[i] = (entry_t)id;
                if (a.l2_prefetch) prefetch_row_l2(a.base32, (uint32_t)a.d_pad32 * 4u, id);
            }
            if (tid == 0) ctl.ns = 0;
            __syncthreads();
            // every key is kept (limit = the empty entry), in whatever order the teams finish
            compute_keys_teams<ANN_STORE_F32, NT>(a.base32, nullptr, a.d_pad32, a.metric, qv, cand, qlen,
                                                     a.team_lanes32, kEmptyEntry, surv, &ctl.ns);
            __syncthreads();
            if (k <= 32) {
                // only the k best are output: select them instead of sorting the whole queue
                res = block_topk<NT>(surv, qlen, k, cand, surv);
            } else {
                int P = 32;
                while (P < qlen) P <<= 1;
                for (int i = qlen + tid; i < P; i += NT) surv[i] = kEmptyEntry;
                __syncthreads();
                block_bitonic_sort<NT>(surv, P);
                res = surv;
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
            st.evals = ctl.evals;
            st.hash_resets = ctl.resets;
            st.dup_dropped = ctl.dropped;
            st.merges = 0;
            st.t_start_ns = ctl.t0;
            st.t_end_ns = global_ns();
            a.stats[qi] = st;
        }
        if (tid == 0 && prof)
            for (int i = 0; i < 4; ++i) a.phase_cycles[(size_t)qi * 4 + i] = ctl.ph[i];
        if (!a.persistent) break;
        __syncthreads();
    }
}

template <int NT, int STORE>
static cudaError_t launch_t(const SearchArgs &a, int smem, int grid, cudaStream_t s) {
    auto fn = sync_search_kernel<NT, STORE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT, int STORE>
static cudaError_t occ_t(int smem, int *bps) {
    auto fn = sync_search_kernel<NT, STORE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, NT, smem);
}

#define ANN_DISPATCH_STORE(NT, FN, ...)                                          \
    switch (storage) {                                                           \
        case ANN_STORE_F32: return FN<NT, ANN_STORE_F32>(__VA_ARGS__);           \
        case ANN_STORE_BF16: return FN<NT, ANN_STORE_BF16>(__VA_ARGS__);         \
        case ANN_STORE_F16: return FN<NT, ANN_STORE_F16>(__VA_ARGS__);           \
        case ANN_STORE_E4M3: return FN<NT, ANN_STORE_E4M3>(__VA_ARGS__);         \
    }                                                                            \
    return cudaErrorInvalidValue;

template <int NT>
static cudaError_t launch_nt(const SearchArgs &a, int storage, int smem, int grid, cudaStream_t s) {
    ANN_DISPATCH_STORE(NT, launch_t, a, smem, grid, s)
}
template <int NT>
static cudaError_t occ_nt(int storage, int smem, int *bps) {
    ANN_DISPATCH_STORE(NT, occ_t, smem, bps)
}

cudaError_t launch_sync_search(const SearchArgs &a, int storage, int threads, int smem, int grid,
                               cudaStream_t s) {
    switch (threads) {
        case 64: return launch_nt<64>(a, storage, smem, grid, s);
        case 128: return launch_nt<128>(a, storage, smem, grid, s);
        case 256: return launch_nt<256>(a, storage, smem, grid, s);
        case 512: return launch_nt<512>(a, storage, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t sync_search_occupancy(int storage, int threads, int smem, int *bps) {
    switch (threads) {
        case 64: return occ_nt<64>(storage, smem, bps);
        case 128: return occ_nt<128>(storage, smem, bps);
        case 256: return occ_nt<256>(storage, smem, bps);
        case 512: return occ_nt<512>(storage, smem, bps);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ann
