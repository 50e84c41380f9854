// search_common.cuh -- device building blocks of the graph-search kernels:
// key encoding, distance gather, visited hash, bitonic sort, merge.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ann_internal.cuh"

namespace ann {

static constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------- key bits
// Order-preserving map float -> uint32 (ascending floats give ascending
// integers); -0 is folded into +0 first so equal keys compare equal.
__device__ __forceinline__ uint32_t key_bits(float f) {
    uint32_t u = __float_as_uint(f + 0.0f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_value(uint32_t b) {
    uint32_t u = (b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b;
    return __uint_as_float(u);
}
__device__ __forceinline__ entry_t pack_entry(float key, uint32_t id) {
    return ((entry_t)key_bits(key) << 32) | (entry_t)id;
}
__device__ __forceinline__ uint32_t entry_id(entry_t e) { return (uint32_t)(e & 0x7FFFFFFFull); }
__device__ __forceinline__ float entry_key(entry_t e) { return key_value((uint32_t)(e >> 32)); }

// -------------------------------------------------------- distance gather
// One 16-byte chunk of a stored row against the matching FP32 query
// elements. L2: sum (q - x)^2; IP: sum q * x (negated by the caller).
template <int STORE> struct Chunk;

template <> struct Chunk<ANN_STORE_F32> {
    static constexpr int kElems = 4;
    __device__ static __forceinline__ float l2(const uint4 c, const float *q, float) {
        float acc = 0.f, t;
        t = q[0] - __uint_as_float(c.x); acc = fmaf(t, t, acc);
        t = q[1] - __uint_as_float(c.y); acc = fmaf(t, t, acc);
        t = q[2] - __uint_as_float(c.z); acc = fmaf(t, t, acc);
        t = q[3] - __uint_as_float(c.w); acc = fmaf(t, t, acc);
        return acc;
    }
    __device__ static __forceinline__ float ip(const uint4 c, const float *q, float) {
        float acc = q[0] * __uint_as_float(c.x);
        acc = fmaf(q[1], __uint_as_float(c.y), acc);
        acc = fmaf(q[2], __uint_as_float(c.z), acc);
        acc = fmaf(q[3], __uint_as_float(c.w), acc);
        return acc;
    }
};

template <typename H2> __device__ __forceinline__ float2 to_f2(uint32_t w);
template <> __device__ __forceinline__ float2 to_f2<__nv_bfloat162>(uint32_t w) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&w);
    return __bfloat1622float2(h);
}
template <> __device__ __forceinline__ float2 to_f2<__half2>(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}

template <typename H2> struct Chunk16 {
    static constexpr int kElems = 8;
    __device__ static __forceinline__ float l2(const uint4 c, const float *q, float) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 v = to_f2<H2>(w[i]);
            float t0 = q[2 * i] - v.x, t1 = q[2 * i + 1] - v.y;
            acc = fmaf(t0, t0, acc);
            acc = fmaf(t1, t1, acc);
        }
        return acc;
    }
    __device__ static __forceinline__ float ip(const uint4 c, const float *q, float) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 v = to_f2<H2>(w[i]);
            acc = fmaf(q[2 * i], v.x, acc);
            acc = fmaf(q[2 * i + 1], v.y, acc);
        }
        return acc;
    }
};
template <> struct Chunk<ANN_STORE_BF16> : Chunk16<__nv_bfloat162> {};
template <> struct Chunk<ANN_STORE_F16> : Chunk16<__half2> {};

template <> struct Chunk<ANN_STORE_E4M3> {
    static constexpr int kElems = 16;
    __device__ static __forceinline__ float2 dq(uint16_t pair, float s) {
        __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
        float2 f = __half22float2(*reinterpret_cast<__half2 *>(&hr));
        return make_float2(__fmul_rn(s, f.x), __fmul_rn(s, f.y));
    }
    __device__ static __forceinline__ float l2(const uint4 c, const float *q, float s) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 a = dq((uint16_t)(w[i] & 0xFFFF), s), b = dq((uint16_t)(w[i] >> 16), s);
            float t;
            t = q[4 * i] - a.x;     acc = fmaf(t, t, acc);
            t = q[4 * i + 1] - a.y; acc = fmaf(t, t, acc);
            t = q[4 * i + 2] - b.x; acc = fmaf(t, t, acc);
            t = q[4 * i + 3] - b.y; acc = fmaf(t, t, acc);
        }
        return acc;
    }
    __device__ static __forceinline__ float ip(const uint4 c, const float *q, float s) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 a = dq((uint16_t)(w[i] & 0xFFFF), s), b = dq((uint16_t)(w[i] >> 16), s);
            acc = fmaf(q[4 * i], a.x, acc);
            acc = fmaf(q[4 * i + 1], a.y, acc);
            acc = fmaf(q[4 * i + 2], b.x, acc);
            acc = fmaf(q[4 * i + 3], b.y, acc);
        }
        return acc;
    }
};

__device__ __forceinline__ uint4 ld_row_chunk(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Keys of the nc candidates whose ids sit in the low word of cand[0..nc),
// written back packed. A team of TS lanes (a power of two, TS >= chunks per
// row when the row has at most 32 chunks) gathers one row with 16-byte
// loads; each team keeps U rows in flight; partial sums are reduced with
// xor shuffles inside the team. All warps of the block take part.
template <int STORE, int NT, int U = 2>
__device__ __forceinline__ void compute_keys(const void *rows, const float *scales, int row_elems,
                                             int metric, const float *qv, entry_t *cand, int nc) {
    constexpr int NW = NT / 32;
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cpr = row_elems / EPC;  // chunks per row (rows are padded to 16 bytes)
    int ts = 1;
    while (ts < cpr && ts < 32) ts <<= 1;
    const int rpw = 32 / ts;
    const int team = lane / ts, tl = lane & (ts - 1);
    const int iters = (cpr + ts - 1) / ts;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = warp * rpw * U; c0 < nc; c0 += NW * rpw * U) {
        float acc[U];
        uint32_t id[U];
        bool valid[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int c = c0 + u * rpw + team;
            valid[u] = c < nc;
            id[u] = valid[u] ? (uint32_t)(cand[c] & 0xFFFFFFFFull) : 0u;
            acc[u] = 0.f;
            sc[u] = 1.f;
            if (STORE == ANN_STORE_E4M3 && valid[u]) sc[u] = __ldg(scales + id[u]);
        }
        for (int it = 0; it < iters; ++it) {
            const int ch = tl + it * ts;
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (valid[u] && ch < cpr) v[u] = ld_row_chunk(rbase + (size_t)id[u] * cpr + ch);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (valid[u] && ch < cpr) {
                    const float *qc = qv + ch * EPC;
                    acc[u] += metric == ANN_METRIC_L2 ? Chunk<STORE>::l2(v[u], qc, sc[u])
                                                     : Chunk<STORE>::ip(v[u], qc, sc[u]);
                }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            for (int off = ts >> 1; off > 0; off >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], off);
            if (tl == 0 && valid[u]) {
                float key = metric == ANN_METRIC_L2 ? acc[u] : -acc[u];
                cand[c0 + u * rpw + team] = pack_entry(key, id[u]);
            }
        }
    }
}

// ------------------------------------------------------------- visited set
// Open addressing over 2^bits uint32 slots (kEmptySlot = free), linear
// probing. Returns 1 if id was inserted now, 0 if it was already present,
// 2 if no free slot was found within the probe limit (the caller treats the
// vertex as new: a forgotten vertex only costs a repeated distance, and the
// merge drops ids already queued).
__device__ __forceinline__ int visited_insert(uint32_t *table, int bits, uint32_t id) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t h = (id * 0x9E3779B1u) >> (32 - bits);
#pragma unroll 1
    for (int p = 0; p < 64; ++p) {
        uint32_t old = atomicCAS(table + h, kEmptySlot, id);
        if (old == kEmptySlot) return 1;
        if (old == id) return 0;
        h = (h + 1u) & mask;
    }
    return 2;
}

// ------------------------------------------------------------ bitonic sort
__device__ __forceinline__ entry_t cmpx(entry_t v, int j, int k, int i) {
    entry_t p = __shfl_xor_sync(kFull, v, j);
    const bool up = (i & k) == 0;
    const bool lower = (i & j) == 0;
    return (lower == up) ? (v < p ? v : p) : (v < p ? p : v);
}

// Ascending sort of s[0..P), P a power of two >= 32 (pad with kEmptyEntry).
// Compare-exchange distances below 32 run in registers with shuffles, wider
// ones through shared memory. Ends with a __syncthreads().
template <int NT>
__device__ void block_bitonic_sort(entry_t *s, int P) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int seg = warp; seg < P / 32; seg += NW) {
        const int i = seg * 32 + lane;
        entry_t v = s[i];
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) v = cmpx(v, j, k, i);
        s[i] = v;
    }
    __syncthreads();
    for (int k = 64; k <= P; k <<= 1) {
        for (int j = k >> 1; j >= 32; j >>= 1) {
            for (int i = threadIdx.x; i < P / 2; i += NT) {
                const int lo = (i / j) * 2 * j + (i % j), hi = lo + j;
                const bool up = (lo & k) == 0;
                entry_t x = s[lo], y = s[hi];
                if ((x > y) == up) {
                    s[lo] = y;
                    s[hi] = x;
                }
            }
            __syncthreads();
        }
        for (int seg = warp; seg < P / 32; seg += NW) {
            const int i = seg * 32 + lane;
            entry_t v = s[i];
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) v = cmpx(v, j, k, i);
            s[i] = v;
        }
        __syncthreads();
    }
}

// Number of entries of sorted A[0..n) that are below x, comparing with the
// checked flag masked off.
__device__ __forceinline__ int count_below(const entry_t *A, int n, entry_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((A[mid] & kMask) < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (int64_t)t;
}

}  // namespace ann

namespace ann {

// Warp-level key computation for the nc <= 32 candidates whose ids sit in the
// low word of c[0..nc) (a per-warp shared buffer); results are written back
// packed. Same team layout as compute_keys, one warp only.
template <int STORE, int U = 4>
__device__ __forceinline__ void warp_compute_keys(const void *rows, const float *scales, int row_elems,
                                                  int metric, const float *qv, entry_t *c, int nc) {
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31;
    const int cpr = row_elems / EPC;
    int ts = 1;
    while (ts < cpr && ts < 32) ts <<= 1;
    const int rpw = 32 / ts;
    const int team = lane / ts, tl = lane & (ts - 1);
    const int iters = (cpr + ts - 1) / ts;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = 0; c0 < nc; c0 += rpw * U) {
        float acc[U];
        uint32_t id[U];
        bool valid[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + u * rpw + team;
            valid[u] = j < nc;
            id[u] = valid[u] ? (uint32_t)(c[j] & 0xFFFFFFFFull) : 0u;
            acc[u] = 0.f;
            sc[u] = 1.f;
            if (STORE == ANN_STORE_E4M3 && valid[u]) sc[u] = __ldg(scales + id[u]);
        }
        for (int it = 0; it < iters; ++it) {
            const int ch = tl + it * ts;
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (valid[u] && ch < cpr) v[u] = ld_row_chunk(rbase + (size_t)id[u] * cpr + ch);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (valid[u] && ch < cpr) {
                    const float *qc = qv + ch * EPC;
                    acc[u] += metric == ANN_METRIC_L2 ? Chunk<STORE>::l2(v[u], qc, sc[u])
                                                     : Chunk<STORE>::ip(v[u], qc, sc[u]);
                }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            for (int off = ts >> 1; off > 0; off >>= 1) acc[u] += __shfl_xor_sync(kFull, acc[u], off);
            if (tl == 0 && valid[u]) {
                const float key = metric == ANN_METRIC_L2 ? acc[u] : -acc[u];
                c[c0 + u * rpw + team] = pack_entry(key, id[u]);
            }
        }
    }
    __syncwarp();
}

// Ascending sort of the 32 entries held one per lane.
__device__ __forceinline__ entry_t warp_sort32(entry_t v) {
    const int i = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) v = cmpx(v, j, k, i);
    return v;
}

// Merge sorted, duplicate-free C[0..nc) into sorted Q[0..qlen) (all threads
// of the block), keeping the first L entries in Qn. A candidate whose id is
// already in Q is dropped; if it carries the checked flag the queued copy
// takes it ("checked wins"). Adjacent equal candidates are also dropped.
// dup is a byte buffer of >= nc entries, ctl_out an int in shared memory.
// Returns the new length. Ends with a __syncthreads().
template <int NT>
__device__ int block_merge_dedupe(entry_t *Q, int qlen, entry_t *C, int nc, int L, entry_t *Qn,
                                  unsigned char *dup, int *ctl_out, long long *dropped) {
    int any = 0;
    for (int j = threadIdx.x; j < nc; j += NT) {
        const entry_t c = C[j] & kMask;
        bool d = (j > 0 && (C[j - 1] & kMask) == c);
        if (!d) {
            const int pos = count_below(Q, qlen, c);
            if (pos < qlen && (Q[pos] & kMask) == c) {
                d = true;
                if (C[j] & kChecked) Q[pos] |= kChecked;
            }
        }
        dup[j] = d;
        any |= d;
    }
    int ncl = nc;
    if (__syncthreads_or(any)) {
        if ((threadIdx.x >> 5) == 0) {
            const int lane = threadIdx.x & 31;
            int out = 0;
            for (int b = 0; b < nc; b += 32) {
                const int j = b + lane;
                const bool keep = j < nc && !dup[j];
                const entry_t c = j < nc ? C[j] : 0ull;
                const unsigned bal = __ballot_sync(kFull, keep);
                if (keep) C[out + __popc(bal & ((1u << lane) - 1u))] = c;
                out += __popc(bal);
            }
            if (lane == 0) *ctl_out = out;
        }
        __syncthreads();
        ncl = *ctl_out;
        if (dropped) *dropped += nc - ncl;
    }
    for (int i = threadIdx.x; i < qlen; i += NT) {
        const entry_t e = Q[i];
        const int pos = i + count_below(C, ncl, e & kMask);
        if (pos < L) Qn[pos] = e;
    }
    for (int j = threadIdx.x; j < ncl; j += NT) {
        const entry_t c = C[j];
        const int pos = j + count_below(Q, qlen, c & kMask);
        if (pos < L) Qn[pos] = c;
    }
    __syncthreads();
    return min(L, qlen + ncl);
}

}  // namespace ann

namespace ann {

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// compute_keys with the rows staged through shared memory: the whole block
// issues 16-byte cp.async copies of up to stage_rows candidate rows (and
// their FP8 scales) at once, waits for them, then lane teams reduce each row
// from shared memory. Many rows are in flight per CTA without holding them
// in registers. stage holds stage_rows * row_bytes bytes (+ stage_rows
// floats after it for the scales). Ends with a __syncthreads().
template <int STORE, int NT>
__device__ void compute_keys_staged(const void *rows, const float *scales, int row_elems, int metric,
                                    const float *qv, entry_t *cand, int nc, unsigned char *stage,
                                    int stage_rows) {
    constexpr int NW = NT / 32;
    constexpr int EPC = Chunk<STORE>::kElems;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cpr = row_elems / EPC;
    const int row_bytes = cpr * 16;
    int ts = 1;
    while (ts < cpr && ts < 32) ts <<= 1;
    const int rpw = 32 / ts;
    const int team = lane / ts, tl = lane & (ts - 1);
    const int iters = (cpr + ts - 1) / ts;
    const unsigned char *g = reinterpret_cast<const unsigned char *>(rows);
    float *ssc = reinterpret_cast<float *>(stage + (size_t)stage_rows * row_bytes);
    for (int b0 = 0; b0 < nc; b0 += stage_rows) {
        const int nb = min(stage_rows, nc - b0);
        for (int i = tid; i < nb * cpr; i += NT) {
            const int r = i / cpr, ch = i - r * cpr;
            const uint32_t id = (uint32_t)(cand[b0 + r] & 0xFFFFFFFFull);
            cp_async16(stage + (size_t)r * row_bytes + ch * 16, g + (size_t)id * row_bytes + ch * 16);
        }
        if (STORE == ANN_STORE_E4M3)
            for (int r = tid; r < nb; r += NT) cp_async4(ssc + r, scales + (uint32_t)(cand[b0 + r] & 0xFFFFFFFFull));
        cp_async_wait_all();
        __syncthreads();
        for (int c0 = warp * rpw; c0 < nb; c0 += NW * rpw) {
            const int r = c0 + team;
            const bool valid = r < nb;
            float acc = 0.f;
            const float sc = (STORE == ANN_STORE_E4M3 && valid) ? ssc[r] : 1.f;
            for (int it = 0; it < iters; ++it) {
                const int ch = tl + it * ts;
                if (valid && ch < cpr) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(stage + (size_t)r * row_bytes + ch * 16);
                    const float *qc = qv + ch * EPC;
                    acc += metric == ANN_METRIC_L2 ? Chunk<STORE>::l2(v, qc, sc) : Chunk<STORE>::ip(v, qc, sc);
                }
            }
            for (int off = ts >> 1; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
            if (tl == 0 && valid) {
                const uint32_t id = (uint32_t)(cand[b0 + r] & 0xFFFFFFFFull);
                cand[b0 + r] = pack_entry(metric == ANN_METRIC_L2 ? acc : -acc, id);
            }
        }
        __syncthreads();
    }
}

}  // namespace ann
