// search_sync.cuh -- bulk-synchronous top-M best-first search, one CTA per query.
//
// Follows Algorithm 1 (BFiS) generalised by Sec. 4.1 to expand the top-M
// unchecked candidates per step, with the Sec. 4.2 staged schedule (M starts
// at M0 and doubles every t steps up to M_max). Every step ends in CTA
// barriers, so the result is deterministic: it is the same top-L queue the
// sequential definition produces, whatever order the warps touch it in.
//
// One step, inside one CTA of NW warps:
//   select   warp 0 takes the first min(M_s, #unchecked) unchecked entries of
//            the sorted queue by ballot + popc, starting past a prefix known to
//            be checked;
//   expand   the step's M_s * R adjacency slots are split evenly over the
//            warps (one lane per slot, coalesced int32 rows); each warp
//            inserts its neighbours into the shared visited set and appends
//            the fresh ones to its own list (one warp scan per batch of
//            slots), asking L2 for each fresh row as it goes;
//   distance each warp gathers its own fresh rows with teams of lanes (16-byte
//            non-caching loads, shuffle reduction) and appends every
//            candidate below the queue's L-th entry to the CTA's survivor
//            list. One barrier; then each warp marks its selected entries
//            checked;
//   sort     the survivors by (key, id): warp sort, run-rank sort or bitonic;
//   merge    drop survivors whose id is already queued (only possible once
//            the visited set forgot a vertex), then a merge-path merge of the
//            queue and the survivors, truncated to L.
// The visited set may forget vertices (a direct-mapped cache evicts, an
// open-addressing table is reset to the queued ids when half full); the queue
// is then still the top-L of everything seen (a forgotten vertex that is met
// again either duplicates a queued id, which the merge drops, or ranks below
// the L-th entry again), so ids are unchanged and only the distance count
// grows.
#pragma once

#include "search_common.cuh"

namespace ann {

struct Ctrl {
    int ns[2];     // survivors appended in the step of this parity
    int nfresh[2]; // block gather: fresh vertices appended in the step of this parity
    int hash_count;
    int do_reset;  // open addressing: the table is half full, reset it before the next select
    int anydup;
    int unsafe;    // 1 once the visited set may have forgotten a vertex this query
    int first_un;  // every queue entry before this position is checked
    int qi, k, L, Mmax;  // the query and its settings (kept here, not in registers, across the step loop)
    int wevals;    // fresh vertices of this query, summed per warp and step
    int sel_last;             // the step's selection: queue position of the last entry taken
    int wcnt[32];             // per-warp counts of the selection scan
    // per-query counters, updated by thread 0 only
    long long steps, expansions, evals, resets, dropped, t0;
    long long ph[4], tmark;  // phase cycles (select, expand, distance, sort+merge) when requested
};

template <int NT, int STORE, bool L2>
__global__ void __launch_bounds__(NT, 65536 / (NT * 64)) sync_search_kernel(const SearchArgs a) {
    constexpr int NW = NT / 32;
    constexpr uint32_t ES = STORE == ANN_STORE_F32 ? 4u : STORE == ANN_STORE_E4M3 ? 1u : 2u;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Ctrl ctl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t row_bytes = (uint32_t)a.d_pad * ES;
    const uint32_t cpr = row_bytes / 16u;
    const SmemLayout &lay = a.sync_lay;
    float *qv = reinterpret_cast<float *>(smem + lay.q_off);
    entry_t *Qa = reinterpret_cast<entry_t *>(smem + lay.q0_off);
    entry_t *Qb = reinterpret_cast<entry_t *>(smem + lay.q1_off);
    entry_t *cand = reinterpret_cast<entry_t *>(smem + lay.cand_off);
    entry_t *surv = reinterpret_cast<entry_t *>(smem + lay.cand2_off);
    unsigned char *dup = smem + lay.dup_off;
    uint32_t *table = reinterpret_cast<uint32_t *>(smem + lay.hash_off);
    const int H = 1 << a.hash_bits;
    const int R = a.R;
    // the step's selected vertices (ids, queue positions), and this warp's fresh vertices: a step's M * R
    // adjacency slots are split evenly over the warps, slot i of the step being slot i mod R of the
    // (i / R)-th selected vertex; i / R = umulhi(i, ceil(2^32 / R)), exact while i < 2^32 / R^2
    int *sel_id = reinterpret_cast<int *>(smem + lay.act_off);
    int *sel_pos = sel_id + a.M;
    const int slots_w = (a.M * R + NW - 1) / NW;  // most slots one warp expands in a step
    uint2 *fresh = reinterpret_cast<uint2 *>(cand) + (size_t)warp * slots_w;  // (id, row) pairs
    const uint32_t r_recip = 0xFFFFFFFFu / (uint32_t)R + 1u;

    for (;;) {
        if (tid == 0) {
            const int item = a.persistent ? atomicAdd(a.work_counter, 1) : (int)blockIdx.x;
            const int q = item >= a.nq ? -1 : (a.order ? a.order[item] : item);
            ctl.qi = q;
            if (q >= 0) {
                ctl.k = a.k_arr ? a.k_arr[q] : a.k;
                ctl.L = a.L_arr ? a.L_arr[q] : a.L;
                ctl.Mmax = a.M_arr ? a.M_arr[q] : a.M;
            }
            ctl.wevals = 0;
            ctl.t0 = global_ns();
            ctl.steps = ctl.expansions = ctl.resets = ctl.dropped = 0;
            ctl.evals = 1;
            ctl.unsafe = 0;
            ctl.first_un = 0;
            ctl.do_reset = 0;
            ctl.ph[0] = ctl.ph[1] = ctl.ph[2] = ctl.ph[3] = 0;
        }
        __syncthreads();
        const int qi = ctl.qi;
        if (qi < 0) break;  // work list exhausted

        const bool bad = ctl.k < 1 || ctl.k > a.k || ctl.L < ctl.k || ctl.L > a.L || ctl.Mmax < 1 || ctl.Mmax > a.M;
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
            const uint32_t empty = (a.slot_bytes < 4 || a.ways) ? 0u : kEmptySlot;
            for (int i = tid; i < words; i += NT) table[i] = empty;
        }
        if (tid == 0) {
            ctl.ns[0] = ctl.ns[1] = 0;
            ctl.nfresh[0] = ctl.nfresh[1] = 0;
            fresh[0] = make_uint2((uint32_t)a.entry, (uint32_t)a.entry);
        }
        __syncthreads();
        // the entry point P: distance, queue = [P], visited = {P}
        if (warp == 0)
            warp_keys_append_m<STORE, 4, L2>(a.base, a.scales, cpr, qv, fresh, 1, a.team_lanes, kEmptyEntry, surv,
                                             &ctl.ns[1]);
        __syncthreads();
        if (tid == 0) {
            Qa[0] = surv[0];
            visit_set(table, a, (uint32_t)a.entry);
            ctl.hash_count = 1;
            ctl.ns[1] = 0;
        }
        __syncthreads();

        int Mcur = a.M0 < ctl.Mmax ? a.M0 : ctl.Mmax;
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
            // --- forget the open-addressing table when half full (keep the queued ids);
            // the direct-mapped cache never resets, it forgets by eviction
            // (decided by thread 0 after the last step's distance barrier, so every thread sees one value)
            if (ctl.do_reset) {
                for (int i = tid; i < H; i += NT) table[i] = kEmptySlot;
                __syncthreads();
                for (int i = tid; i < qlen; i += NT) visited_insert(table, a.hash_bits, entry_id(Q[i]));
                if (tid == 0) {
                    ctl.hash_count = qlen;
                    ctl.do_reset = 0;
                    ctl.resets++;
                    ctl.unsafe = 1;
                }
                __syncthreads();
            }
            const int par = step & 1;
            // --- select: the first Mcur unchecked entries (rank order) of the stable queue, all warps
            // scanning from first_un (entries before it are all checked)
            const int found = select_step<NW>(Q, qlen, ctl.first_un, Mcur, sel_id, sel_pos, ctl.wcnt,
                                                   &ctl.sel_last);
            const int nact = found < Mcur ? found : Mcur;
            if (nact == 0) break;  // no unchecked vertex left (identical in every warp)
            ANN_PHASE(0)
            step++;

            // --- expand this warp's share of the step's adjacency slots: adjacency -> visited set -> fresh
            // list (+ L2 prefetch)
            const int nf = expand_step<NW>(a, table, sel_id, nact, r_recip, row_bytes, fresh,
                                           a.block_gather ? reinterpret_cast<uint2 *>(cand) : nullptr,
                                           &ctl.nfresh[par], 1, 0, &ctl.unsafe);
            __syncwarp();
            if (lane == 0) {
                if (nf) {
                    atomicAdd(&ctl.wevals, nf);
                    if (a.visited_mode == 0) atomicAdd(&ctl.hash_count, nf);
                }
            }
            ANN_PHASE(1)

            // --- distances of this warp's fresh rows; only candidates below the L-th queued entry survive
            const int L = ctl.L;
            const entry_t limit = qlen >= L ? (Q[L - 1] & kMask) : kEmptyEntry;
            // four chunks in flight per lane (one 128-d BF16 row per 4-lane team in one round trip); each warp
            // gathers its own list, or, with a block gather (long rows: few per warp), every warp takes every
            // NW-th pass of one list for the CTA
            {
                const uint2 *gl = fresh;
                int gn = nf, gb = 0, gs = 1;
                if (a.block_gather) {
                    __syncthreads();  // the CTA's list is complete
                    gl = reinterpret_cast<const uint2 *>(cand);
                    gn = ctl.nfresh[par];
                    gb = warp;
                    gs = NW;
                }
                if (!gather_fixed<STORE, L2>(a.base, a.scales, cpr, a.team_lanes, qv, nullptr, gl, gn, gb, gs, limit,
                                             surv, &ctl.ns[par]))
                    warp_keys_append_m<STORE, 4, L2>(a.base, a.scales, cpr, qv, gl, gn, a.team_lanes, limit, surv,
                                                     &ctl.ns[par], gb, gs);
            }
            __syncthreads();
            ANN_PHASE(2)
            const int ns = ctl.ns[par];
            if (tid < nact) Q[sel_pos[tid]] |= kChecked;  // the selection is taken: mark it
            if (tid == 0) {
                ctl.ns[par ^ 1] = 0;  // next step's counters (last read before this step's barrier)
                ctl.nfresh[par ^ 1] = 0;
                ctl.steps++;
                ctl.expansions += nact;
                ctl.first_un = ctl.sel_last + 1;
                ctl.do_reset = a.visited_mode == 0 && ctl.hash_count * 2 > H;
            }
            if (ns > 0) {
                // --- sort the survivors, drop ids already queued (only after the visited set forgot a vertex),
                // merge into the other queue buffer truncated to L
                const int ncl = sort_dedupe_merge<NT>(Q, qlen, surv, ns, cand, Qn, ctl.L, ctl.unsafe != 0, dup,
                                                      &ctl.anydup, &ctl.dropped, &ctl.first_un);
                qlen = min(ctl.L, qlen + ncl);
                entry_t *tmp = Q;
                Q = Qn;
                Qn = tmp;
            } else {
                __syncthreads();  // the marks and first_un are visible before the next select
            }
            ANN_PHASE(3)
            if (step % a.t == 0) Mcur = min(2 * Mcur, ctl.Mmax);
        }
#undef ANN_PHASE

        // --- output: first k of the queue, optionally re-ranked with FP32 rows
        const int k = ctl.k;
        const entry_t *res = Q;
        if (a.rerank) {
            for (int i = tid; i < qlen; i += NT) {
                const uint32_t id = entry_id(Q[i]);
                cand[i] = (entry_t)id;
                if (a.l2_prefetch) prefetch_row_l2(a.base32, (uint32_t)a.d_pad32 * 4u, id);
            }
            if (tid == 0) ctl.ns[0] = 0;
            __syncthreads();
            // every key is kept (limit = the empty entry), in whatever order the teams finish
            if (!gather_fixed<ANN_STORE_F32, L2>(a.base32, nullptr, (uint32_t)a.d_pad32 / 4u, a.team_lanes32, qv,
                                                 cand, nullptr, qlen, warp, NW, kEmptyEntry, surv, &ctl.ns[0]))
                compute_keys_teams_m<ANN_STORE_F32, NT, L2, 2>(a.base32, nullptr, a.d_pad32, qv, cand, qlen,
                                                               a.team_lanes32, kEmptyEntry, surv, &ctl.ns[0]);
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
            st.evals = ctl.evals + ctl.wevals;
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

// One kernel per metric: the distance formula is a compile-time choice.
template <int NT, int STORE>
static auto sync_kernel_for(int metric) {
    return metric == ANN_METRIC_L2 ? sync_search_kernel<NT, STORE, true> : sync_search_kernel<NT, STORE, false>;
}

// Launch / occupancy of the kernels of one storage type (each storage type is
// instantiated in a translation unit of its own: search_sync_<storage>.cu).
template <int STORE>
cudaError_t launch_sync_store(const SearchArgs &a, int threads, int smem, int grid, cudaStream_t s) {
    auto go = [&](auto fn) -> cudaError_t {
        cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
        switch (threads) {
            case 64: fn<<<grid, 64, smem, s>>>(a); break;
            case 128: fn<<<grid, 128, smem, s>>>(a); break;
            case 256: fn<<<grid, 256, smem, s>>>(a); break;
            case 512: fn<<<grid, 512, smem, s>>>(a); break;
        }
        return cudaGetLastError();
    };
    switch (threads) {
        case 64: return go(sync_kernel_for<64, STORE>(a.metric));
        case 128: return go(sync_kernel_for<128, STORE>(a.metric));
        case 256: return go(sync_kernel_for<256, STORE>(a.metric));
        case 512: return go(sync_kernel_for<512, STORE>(a.metric));
    }
    return cudaErrorInvalidValue;
}

template <int STORE>
cudaError_t occupancy_sync_store(int metric, int threads, int smem, int *bps) {
    auto occ = [&](auto fn, int nt) -> cudaError_t {
        cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void *>(fn), smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, fn, nt, smem);
    };
    switch (threads) {
        case 64: return occ(sync_kernel_for<64, STORE>(metric), 64);
        case 128: return occ(sync_kernel_for<128, STORE>(metric), 128);
        case 256: return occ(sync_kernel_for<256, STORE>(metric), 256);
        case 512: return occ(sync_kernel_for<512, STORE>(metric), 512);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ann
