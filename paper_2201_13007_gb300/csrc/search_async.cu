// search_async.cu -- Algorithm 3 (Speed-ANN intra-query parallel search) with
// the Algorithm 2 merge test, one CTA per query, one warp per walker.
//
// Global step (CTA-wide, between barriers):
//   deal   the unchecked entries of the global queue S go round-robin, by
//          rank, to the M active walkers' private queues; checked entries
//          stay in S;
//   walk   in sub-steps: in each, every active walker (warp) with an
//          unchecked entry expands the first one of its private queue
//          (insert the unvisited neighbours, resize to L), sharing one
//          visited set with the other walkers (shared-memory CAS, no
//          ordering between walkers within a sub-step: the loosely
//          synchronised visiting map of Sec. 4.4), and records its update
//          position (best rank at which a new candidate landed, L if none).
//          A CTA barrier ends the sub-step; then every thread evaluates the
//          same merge test for the checker walker (round robin): if the
//          checker expanded in this sub-step and mean(U) >= L * R (Algorithm
//          2), or, with the stall rule, the walkers' mean count of expansions
//          since the deal that inserted nothing into their top L reaches the
//          patience; or if no walker expanded, the walk ends. Sub-steps are cheap on a GPU (one
//          CTA barrier), so the walkers advance in lock-step as in the
//          oracle's reading of Algorithm 3, and every update position the
//          checker averages is from the same sub-step;
//   merge  the private queues merge into S (dedupe by id, checked wins),
//          S is resized to L, and M doubles while M < M_max.
// The search ends when a deal finds no unchecked entry. No warp ever waits on
// another except at CTA barriers that every warp reaches.
#include "search_common.cuh"

namespace ann {

struct AsyncCtrl {
    long long qi;
    int nun;
    int ncheck;
    int chunk_tot[64];
    int merged_len;
    int hash_count;
    // per sub-step parity and walker: (stall count << 16) | (update position << 1) | expanded-in-this-sub-step
    int walk[2][32];
};

__host__ __device__ inline int async_smem_bytes(int qfloats, int Lcap, int walkers, int hash_bits, int *offs) {
    int o = 0;
    offs[0] = o; o += align16(qfloats * 4);                 // query
    offs[1] = o; o += align16(Lcap * 8);                    // S
    offs[2] = o; o += align16(Lcap * 8);                    // S'
    offs[3] = o; o += align16(walkers * Lcap * 8);          // private queues
    offs[4] = o; o += align16(walkers * 32 * 8);            // per-walker candidates
    offs[5] = o; o += align16(Lcap > 32 ? Lcap : 32);       // dup flags
    offs[6] = o; o += align16((1 << hash_bits) * 4);        // visited table
    offs[7] = o; o += align16(walkers * 4);                 // private queue lengths
    return o;
}

// One insert into the walkers' shared visited set: the set-associative cache
// of tags (a.ways > 0; it forgets a vertex only when a fourth one enters its
// set) or an open-addressing table reset when half full. 0 = seen before.
__device__ __forceinline__ int async_visit(uint32_t *table, const SearchArgs &a, uint32_t id) {
    if (a.ways == 3) return visited_assoc<3>(table, a.hash_bits, a.tag_bits, id);
    if (a.ways == 2) return visited_assoc<2>(table, a.hash_bits, a.tag_bits, id);
    return visited_insert(table, a.hash_bits, id);
}

template <int NT, int STORE>
__global__ void __launch_bounds__(NT, (NT >= 512 ? 1 : 65536 / (NT * 128))) async_search_kernel(const SearchArgs a) {
    constexpr int T = NT / 32;  // walkers
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ AsyncCtrl ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int off[8];
    async_smem_bytes(a.qfloats, a.Lcap, T, a.hash_bits, off);
    float *qv = reinterpret_cast<float *>(smem + off[0]);
    entry_t *Sa = reinterpret_cast<entry_t *>(smem + off[1]);
    entry_t *Sb = reinterpret_cast<entry_t *>(smem + off[2]);
    entry_t *LSall = reinterpret_cast<entry_t *>(smem + off[3]);
    entry_t *CWall = reinterpret_cast<entry_t *>(smem + off[4]);
    unsigned char *dup = smem + off[5];
    uint32_t *table = reinterpret_cast<uint32_t *>(smem + off[6]);
    int *lsn = reinterpret_cast<int *>(smem + off[7]);
    const int H = 1 << a.hash_bits;
    const int R = a.R;
    const int Lcap = a.Lcap;

    for (;;) {
        if (tid == 0) {
            const int item = a.persistent ? atomicAdd(a.work_counter, 1) : (int)blockIdx.x;
            ctl.qi = item >= a.nq ? -1 : (a.order ? a.order[item] : item);
        }
        __syncthreads();
        const long long qi = ctl.qi;
        if (qi < 0) break;  // work list exhausted
        const int64_t t0 = global_ns();
        const int k = a.k_arr ? a.k_arr[qi] : a.k;
        const int L = a.L_arr ? a.L_arr[qi] : a.L;
        const int Mmax = a.M_arr ? a.M_arr[qi] : a.M;
        int64_t *oid = a.out_ids + (size_t)qi * a.k;
        float *odist = a.out_dists + (size_t)qi * a.k;
        if (k < 1 || k > a.k || L < k || L > a.L || Mmax < 1 || Mmax > a.M || Mmax > T) {
            for (int i = tid; i < a.k; i += NT) {
                oid[i] = -1;
                odist[i] = __int_as_float(0x7f800000);
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
        const float threshold = (float)L * a.R_ratio;

        const float *qg = a.queries + (size_t)qi * a.d;
        for (int i = tid; i < a.qfloats; i += NT) qv[i] = i < a.d ? qg[i] : 0.f;
        for (int i = tid; i < H; i += NT) table[i] = a.ways ? 0u : kEmptySlot;
        entry_t *CW0 = CWall;
        if (tid == 0) CW0[0] = (entry_t)(uint32_t)a.entry;
        __syncthreads();
        if (warp == 0) warp_compute_keys<STORE>(a.base, a.scales, a.d_pad, a.metric, qv, CW0, 1);
        __syncthreads();
        if (tid == 0) {
            Sa[0] = CW0[0];
            async_visit(table, a, (uint32_t)a.entry);
            ctl.hash_count = 1;
        }
        __syncthreads();

        entry_t *S = Sa, *Sn = Sb;
        int slen = 1;
        int M = a.M0 < Mmax ? a.M0 : Mmax;
        long long checker = 0;
        long long gsteps = 0, merges = 0, resets = 0, dropped = 0;
        long long w_exp = 0, w_evals = 0;  // per-warp counters (lane 0)
        for (;;) {
            // ---------------- deal: block scan of the unchecked flags over S
            const int nchunks = (slen + 31) / 32;
            for (int c = warp; c < nchunks; c += T) {
                const int i = c * 32 + lane;
                const bool un = i < slen && !(S[i] & kChecked);
                const unsigned bal = __ballot_sync(kFull, un);
                if (lane == 0) ctl.chunk_tot[c] = __popc(bal);
            }
            __syncthreads();
            if (warp == 0) {
                // exclusive prefix over at most 64 chunks
                int v0 = lane < nchunks ? ctl.chunk_tot[lane] : 0;
                int v1 = lane + 32 < nchunks ? ctl.chunk_tot[lane + 32] : 0;
                int s0 = v0, s1 = v1;
                for (int o = 1; o < 32; o <<= 1) {
                    int t0s = __shfl_up_sync(kFull, s0, o), t1s = __shfl_up_sync(kFull, s1, o);
                    if (lane >= o) { s0 += t0s; s1 += t1s; }
                }
                const int tot0 = __shfl_sync(kFull, s0, 31);
                __syncwarp();
                if (lane < nchunks) ctl.chunk_tot[lane] = s0 - v0;
                if (lane + 32 < nchunks) ctl.chunk_tot[lane + 32] = tot0 + s1 - v1;
                const int tot1 = __shfl_sync(kFull, s1, 31);
                if (lane == 0) ctl.nun = tot0 + tot1;
            }
            __syncthreads();
            const int nun = ctl.nun;
            if (nun == 0) break;  // all private queues would be empty
            for (int c = warp; c < nchunks; c += T) {
                const int i = c * 32 + lane;
                const entry_t e = i < slen ? S[i] : kChecked;
                const bool un = i < slen && !(e & kChecked);
                const unsigned bal = __ballot_sync(kFull, un);
                const int ru = ctl.chunk_tot[c] + __popc(bal & ((1u << lane) - 1u));
                if (un) {
                    const int w = ru % M;
                    LSall[(size_t)w * Lcap + ru / M] = e;
                } else if (i < slen) {
                    const int rc = c * 32 + lane - (ctl.chunk_tot[c] + __popc(bal & ((1u << lane) - 1u)));
                    Sn[rc] = e;
                }
            }
            const int nactive = nun < M ? nun : M;
            if (tid < T) lsn[tid] = tid < nactive ? (nun - tid + M - 1) / M : 0;
            __syncthreads();
            {
                entry_t *t = S;
                S = Sn;
                Sn = t;
            }
            slen = slen - nun;
            const int chk = (int)(checker % nactive);

            // ---------------- walkers, in lock-step sub-steps (one CTA barrier each)
            bool raised = false;
            {
                entry_t *Q = LSall + (size_t)warp * Lcap;
                entry_t *cw = CWall + warp * 32;
                int ql = warp < nactive ? lsn[warp] : 0;
                int upos_w = 0;   // this walker's update position (U is reset to 0 at each deal)
                int stall_w = 0;  // its expansions since the deal that inserted nothing into its top L
                for (int sub = 0;; ++sub) {
                    const int par = sub & 1;
                    bool expanded = false;
                    if (warp < nactive) {
                        int idx = -1;
                        for (int b = 0; b < ql; b += 32) {
                            const int i = b + lane;
                            const bool un = i < ql && !(Q[i] & kChecked);
                            const unsigned bal = __ballot_sync(kFull, un);
                            if (bal) {
                                idx = b + __ffs(bal) - 1;
                                break;
                            }
                        }
                        if (idx >= 0) {
                            expanded = true;
                            const entry_t ev = Q[idx];
                            __syncwarp();
                            if (lane == 0) Q[idx] = ev | kChecked;
                            __syncwarp();
                            const uint32_t v = entry_id(ev);
                            w_exp++;
                            int upos = L;
                            for (int r0 = 0; r0 < R; r0 += 32) {
                                const int r = r0 + lane;
                                const int u = r < R ? __ldg(a.adj + (size_t)v * R + r) : -1;
                                const bool fresh = u >= 0 && async_visit(table, a, (uint32_t)u) != 0;
                                const unsigned bal = __ballot_sync(kFull, fresh);
                                const int nf = __popc(bal);
                                if (fresh) cw[__popc(bal & ((1u << lane) - 1u))] = (entry_t)(uint32_t)u;
                                __syncwarp();
                                if (nf == 0) continue;
                                if (lane == 0) atomicAdd(&ctl.hash_count, nf);
                                w_evals += nf;
                                warp_compute_keys<STORE>(a.base, a.scales, a.d_pad, a.metric, qv, cw, nf);
                                entry_t e = lane < nf ? cw[lane] : kEmptyEntry;
                                e = warp_sort32(e);
                                // drop ids already in this private queue (or repeated in this row)
                                const entry_t prev = __shfl_up_sync(kFull, e, 1);
                                int pq = lane < nf ? count_below(Q, ql, e) : ql;
                                const bool dupl =
                                    lane < nf && ((pq < ql && (Q[pq] & kMask) == e) || (lane > 0 && prev == e));
                                const bool keep = lane < nf && !dupl;
                                const unsigned kb = __ballot_sync(kFull, keep);
                                const int nk = __popc(kb);
                                __syncwarp();
                                if (keep) cw[__popc(kb & ((1u << lane) - 1u))] = e;
                                __syncwarp();
                                // target ranks of the kept candidates (against the old queue)
                                entry_t cnew = lane < nk ? cw[lane] : kEmptyEntry;
                                const int pnew = lane < nk ? lane + count_below(Q, ql, cnew) : L;
                                // move the existing entries at or after the first insertion point, back to front
                                const int p0 = __shfl_sync(kFull, pnew, 0);
                                for (int b = ((ql + 31) / 32 - 1) * 32; b >= 0 && b + 32 > p0 - 0; b -= 32) {
                                    const int i = b + lane;
                                    const entry_t ei = i < ql ? Q[i] : 0ull;
                                    const int pi = i < ql ? i + count_below(cw, nk, ei & kMask) : L;
                                    __syncwarp();
                                    if (i < ql && pi < L && pi != i) Q[pi] = ei;
                                    __syncwarp();
                                }
                                if (lane < nk && pnew < L) Q[pnew] = cnew;
                                __syncwarp();
                                ql = min(L, ql + nk);
                                if (nk > 0 && p0 < upos) upos = p0;
                            }
                            upos_w = upos;
                            if (upos == L) stall_w++;
                        }
                    }
                    if (lane == 0 && warp < T)
                        ctl.walk[par][warp] = (min(stall_w, 32767) << 16) | (upos_w << 1) | (expanded ? 1 : 0);
                    __syncthreads();  // the sub-step is over: every walker's word for it is written
                    // every thread evaluates the same test (Algorithm 2 for the checker; none expanded = all idle)
                    bool any = false;
                    int sum = 0, stalls = 0;
                    for (int w2 = 0; w2 < nactive; ++w2) {
                        const int wd = ctl.walk[par][w2];
                        any |= (wd & 1) != 0;
                        sum += (wd >> 1) & 0x7FFF;
                        stalls += wd >> 16;
                    }
                    if (!any) break;
                    const bool test = a.merge_rule == 1 ? (float)stalls / (float)nactive >= a.patience
                                                        : (float)sum / (float)nactive >= threshold;
                    if ((ctl.walk[par][chk] & 1) && test) {
                        raised = true;
                        break;
                    }
                }
                if (warp < nactive && lane == 0) lsn[warp] = ql;
            }
            __syncthreads();
            if (raised) checker++;
            // ---------------- merge the private queues into S
            for (int w = 0; w < nactive; ++w) {
                slen = block_merge_dedupe<NT>(S, slen, LSall + (size_t)w * Lcap, lsn[w], L, Sn, dup,
                                              &ctl.merged_len, &dropped);
                entry_t *t = S;
                S = Sn;
                Sn = t;
            }
            merges++;
            gsteps++;
            if (M < Mmax) M = min(2 * M, Mmax);
            // forget the visited table when half full (keep the queued ids)
            if (!a.ways && ctl.hash_count * 2 > H) {
                for (int i = tid; i < H; i += NT) table[i] = kEmptySlot;
                __syncthreads();
                for (int i = tid; i < slen; i += NT) visited_insert(table, a.hash_bits, entry_id(S[i]));
                __syncthreads();
                if (tid == 0) ctl.hash_count = slen;
                resets++;
            }
            __syncthreads();
        }

        // ---------------- output (optionally re-ranked with FP32 rows)
        const entry_t *res = S;
        if (a.rerank) {
            entry_t *buf = LSall;  // free now; holds T * Lcap >= next_pow2(L) entries (host checks)
            for (int i = tid; i < slen; i += NT) buf[i] = (entry_t)entry_id(S[i]);
            __syncthreads();
            compute_keys<ANN_STORE_F32, NT>(a.base32, nullptr, a.d_pad32, a.metric, qv, buf, slen);
            int P = 32;
            while (P < slen) P <<= 1;
            for (int i = slen + tid; i < P; i += NT) buf[i] = kEmptyEntry;
            __syncthreads();
            block_bitonic_sort<NT>(buf, P);
            res = buf;
        }
        for (int i = tid; i < a.k; i += NT) {
            if (i < k && i < slen) {
                oid[i] = (int64_t)entry_id(res[i]);
                odist[i] = entry_key(res[i]);
            } else {
                oid[i] = -1;
                odist[i] = __int_as_float(0x7f800000);
            }
        }
        // per-warp counters
        __shared__ long long red[2][T];
        if (lane == 0) {
            red[0][warp] = w_exp;
            red[1][warp] = w_evals;
        }
        __syncthreads();
        if (tid == 0 && a.stats) {
            long long ex = 0, ev = 1;
            for (int w = 0; w < T; ++w) {
                ex += red[0][w];
                ev += red[1][w];
            }
            ann_query_stats st;
            st.steps = gsteps;
            st.expansions = ex;
            st.evals = ev;
            st.hash_resets = resets;
            st.dup_dropped = dropped;
            st.merges = merges;
            st.t_start_ns = t0;
            st.t_end_ns = global_ns();
            a.stats[qi] = st;
        }
        if (!a.persistent) break;
        __syncthreads();
    }
}

int async_smem_size(int qfloats, int Lcap, int walkers, int hash_bits) {
    int off[8];
    return async_smem_bytes(qfloats, Lcap, walkers, hash_bits, off);
}

template <int NT, int STORE>
static cudaError_t alaunch_t(const SearchArgs &a, int smem, int grid, cudaStream_t s) {
    auto fn = async_search_kernel<NT, STORE>;
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, NT, smem, s>>>(a);
    return cudaGetLastError();
}

template <int NT, int STORE>
static cudaError_t aocc_t(int smem, int *bps) {
    auto fn = async_search_kernel<NT, STORE>;
    cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, NT, smem);
}

#define ANN_ASYNC_STORE(NT, FN, ...)                                     \
    switch (storage) {                                                   \
        case ANN_STORE_F32: return FN<NT, ANN_STORE_F32>(__VA_ARGS__);   \
        case ANN_STORE_BF16: return FN<NT, ANN_STORE_BF16>(__VA_ARGS__); \
        case ANN_STORE_F16: return FN<NT, ANN_STORE_F16>(__VA_ARGS__);   \
        case ANN_STORE_E4M3: return FN<NT, ANN_STORE_E4M3>(__VA_ARGS__); \
    }                                                                    \
    return cudaErrorInvalidValue;

template <int NT>
static cudaError_t alaunch_nt(const SearchArgs &a, int storage, int smem, int grid, cudaStream_t s) {
    ANN_ASYNC_STORE(NT, alaunch_t, a, smem, grid, s)
}
template <int NT>
static cudaError_t aocc_nt(int storage, int smem, int *bps) {
    ANN_ASYNC_STORE(NT, aocc_t, smem, bps)
}

cudaError_t launch_async_search(const SearchArgs &a, int storage, int threads, int smem, int grid,
                                cudaStream_t s) {
    switch (threads) {
        case 64: return alaunch_nt<64>(a, storage, smem, grid, s);
        case 128: return alaunch_nt<128>(a, storage, smem, grid, s);
        case 256: return alaunch_nt<256>(a, storage, smem, grid, s);
        case 512: return alaunch_nt<512>(a, storage, smem, grid, s);
        case 1024: return alaunch_nt<1024>(a, storage, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t async_search_occupancy(int storage, int threads, int smem, int *bps) {
    switch (threads) {
        case 64: return aocc_nt<64>(storage, smem, bps);
        case 128: return aocc_nt<128>(storage, smem, bps);
        case 256: return aocc_nt<256>(storage, smem, bps);
        case 512: return aocc_nt<512>(storage, smem, bps);
        case 1024: return aocc_nt<1024>(storage, smem, bps);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ann
