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
// Packed two-lane FP32 arithmetic (sub.f32x2 / fma.f32x2 / mul.f32x2): each
// instruction does the work of two scalar ones, each lane rounded exactly as
// the scalar operation would be.
__device__ __forceinline__ unsigned long long f2u(float2 v) {
    return ((unsigned long long)__float_as_uint(v.y) << 32) | __float_as_uint(v.x);
}
__device__ __forceinline__ float2 u2f(unsigned long long u) {
    return make_float2(__uint_as_float((uint32_t)u), __uint_as_float((uint32_t)(u >> 32)));
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)), "l"(f2u(c)));
    return u2f(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
// acc += (q - x)^2 (L2) or acc += q * x (inner product), two lanes at a time
__device__ __forceinline__ void acc_pair(float2 &acc, float2 q, float2 x, bool l2) {
    if (l2) {
        const float2 d = sub2(q, x);
        acc = fma2(d, d, acc);
    } else {
        acc = fma2(q, x, acc);
    }
}

// One 16-byte chunk of a stored row against the matching FP32 query
// elements, accumulated into a packed pair of partial sums.
template <int STORE> struct Chunk;

template <> struct Chunk<ANN_STORE_F32> {
    static constexpr int kElems = 4;
    __device__ static __forceinline__ void add(float2 &acc, const uint4 c, const float *q, float, bool l2) {
        const float4 qq = *reinterpret_cast<const float4 *>(q);
        acc_pair(acc, make_float2(qq.x, qq.y), make_float2(__uint_as_float(c.x), __uint_as_float(c.y)), l2);
        acc_pair(acc, make_float2(qq.z, qq.w), make_float2(__uint_as_float(c.z), __uint_as_float(c.w)), l2);
    }
};

template <typename H2> __device__ __forceinline__ float2 to_f2(uint32_t w);
template <> __device__ __forceinline__ float2 to_f2<__nv_bfloat162>(uint32_t w) {
    // bfloat16 -> float is exact: the 16 bits become the high half of the float
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
template <> __device__ __forceinline__ float2 to_f2<__half2>(uint32_t w) {
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    return __half22float2(h);
}

template <typename H2> struct Chunk16 {
    static constexpr int kElems = 8;
    __device__ static __forceinline__ void add(float2 &acc, const uint4 c, const float *q, float, bool l2) {
        const float4 qa = *reinterpret_cast<const float4 *>(q);
        const float4 qb = *reinterpret_cast<const float4 *>(q + 4);
        acc_pair(acc, make_float2(qa.x, qa.y), to_f2<H2>(c.x), l2);
        acc_pair(acc, make_float2(qa.z, qa.w), to_f2<H2>(c.y), l2);
        acc_pair(acc, make_float2(qb.x, qb.y), to_f2<H2>(c.z), l2);
        acc_pair(acc, make_float2(qb.z, qb.w), to_f2<H2>(c.w), l2);
    }
};
template <> struct Chunk<ANN_STORE_BF16> : Chunk16<__nv_bfloat162> {};
template <> struct Chunk<ANN_STORE_F16> : Chunk16<__half2> {};

template <> struct Chunk<ANN_STORE_E4M3> {
    static constexpr int kElems = 16;
    __device__ static __forceinline__ float2 dq(uint16_t pair, float s) {
        __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)pair, __NV_E4M3);
        const float2 f = __half22float2(*reinterpret_cast<__half2 *>(&hr));
        return mul2(make_float2(s, s), f);  // the stored value: float32(scale * code)
    }
    __device__ static __forceinline__ void add(float2 &acc, const uint4 c, const float *q, float s, bool l2) {
        const uint32_t w[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 qq = *reinterpret_cast<const float4 *>(q + 4 * i);
            acc_pair(acc, make_float2(qq.x, qq.y), dq((uint16_t)(w[i] & 0xFFFF), s), l2);
            acc_pair(acc, make_float2(qq.z, qq.w), dq((uint16_t)(w[i] >> 16), s), l2);
        }
    }
};

// Ask L2 for one row. No completion is tracked and no register is held, so
// every row of a step can be in flight at once. Each lane names its own row.
// Rows of up to 1 KB take one prefetch.global.L2 per 128-byte line they touch
// (at most 9 instructions, issued by every lane at once); longer rows take
// one bulk prefetch (cp.async.bulk.prefetch.L2), whose address is
// warp-uniform, so lanes with different rows issue it one after another --
// still fewer instructions than a line at a time for a 2-4 KB row.
__device__ __forceinline__ void prefetch_row_l2(const void *rows, uint32_t row_bytes, uint32_t id) {
    const char *row = static_cast<const char *>(rows) + (size_t)id * row_bytes;
    const size_t p = __cvta_generic_to_global(row);  // the .global state space address of the row
    if (row_bytes > 1024) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(row_bytes) : "memory");
        return;
    }
    const size_t end = p + row_bytes;
    for (size_t a = p & ~size_t(127); a < end; a += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// Ask L2 for one contiguous range (16-byte aligned start, bytes a multiple
// of 16) with a single bulk prefetch. The address must be the same in every
// lane that executes it; callers issue it from one lane.
__device__ __forceinline__ void prefetch_range_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint4 ld_row_chunk(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

// Keys of the nc candidates whose ids sit in the low word of cand[0..nc).
// A team of TS lanes (a power of two, TS >= chunks per row when the row has
// at most 32 chunks) gathers one row with 16-byte loads; each team keeps U
// rows in flight; partial sums are reduced with xor shuffles inside the team.
// All warps of the block take part. With out == nullptr the packed entries
// are written back in place; otherwise only entries below `limit` (in
// (key, id) order) are appended to out[] through the shared counter *out_n.
template <int STORE, int NT, bool L2, int U = 2>
__device__ __forceinline__ void compute_keys_m(const void *rows, const float *scales, int row_elems,
                                               const float *qv, entry_t *cand, int nc, entry_t limit,
                                               entry_t *out, int *out_n) {
    constexpr int NW = NT / 32;
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int cpr = row_elems / EPC;  // chunks per row (rows are padded to 16 bytes)
    int ts = 1;
    while (ts < cpr && ts < 32) ts <<= 1;
    const int rpw = 32 / ts;
    const int team = lane / ts, tl = lane & (ts - 1);
    const int iters = (cpr + ts - 1) / ts;
    constexpr bool l2 = L2;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = warp * rpw * U; c0 < nc; c0 += NW * rpw * U) {
        float2 acc[U];
        uint32_t id[U];
        bool valid[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * rpw + team;
            valid[u] = c < nc;
            id[u] = valid[u] ? (uint32_t)(cand[c] & 0xFFFFFFFFull) : 0u;
            acc[u] = make_float2(0.f, 0.f);
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
                if (valid[u] && ch < cpr) Chunk<STORE>::add(acc[u], v[u], qv + ch * EPC, sc[u], l2);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float r = acc[u].x + acc[u].y;
            for (int off = ts >> 1; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
            const entry_t e = pack_entry(l2 ? r : -r, id[u]);
            const bool write = tl == 0 && valid[u];
            if (out == nullptr) {
                if (write) cand[c0 + u * rpw + team] = e;
            } else {
                const bool keep = write && e < limit;
                const unsigned bal = __ballot_sync(kFull, keep);
                int base = 0;
                if (lane == 0 && bal) base = atomicAdd(out_n, __popc(bal));
                base = __shfl_sync(kFull, base, 0);
                if (keep) out[base + __popc(bal & ((1u << lane) - 1u))] = e;
            }
        }
    }
}

// The metric is a template parameter of the loop bodies, so only one
// distance formula is compiled into each: a runtime test inside the chunk
// math would be if-converted into both formulas.
template <int STORE, int NT, int U = 2>
__device__ __forceinline__ void compute_keys(const void *rows, const float *scales, int row_elems,
                                             int metric, const float *qv, entry_t *cand, int nc,
                                             entry_t limit = kEmptyEntry, entry_t *out = nullptr,
                                             int *out_n = nullptr) {
    if (metric == ANN_METRIC_L2)
        compute_keys_m<STORE, NT, true, U>(rows, scales, row_elems, qv, cand, nc, limit, out, out_n);
    else
        compute_keys_m<STORE, NT, false, U>(rows, scales, row_elems, qv, cand, nc, limit, out, out_n);
}

// Same contract as the filtered compute_keys, with teams of ts lanes (a
// power of two, 1..32) per row and each lane walking its own chunks of the
// row (chunk tl, tl + ts, ...), G of them in flight per round. A warp covers
// 32 / ts rows at once, so the shuffle reduction (log2 ts levels) and the
// append are paid once per 32 / ts rows; with small teams that is far fewer
// instructions per row than one chunk per lane.
template <int STORE, int NT, bool L2, int G>
__device__ __forceinline__ void compute_keys_teams_m(const void *rows, const float *scales, int row_elems,
                                                     const float *qv, const entry_t *cand, int nc, int lts,
                                                     entry_t limit, entry_t *out, int *out_n) {
    constexpr int NW = NT / 32;
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ts = 1 << lts, rpw = 32 >> lts;
    const int cpr = row_elems / EPC;
    const int team = lane >> lts, tl = lane & (ts - 1);
    constexpr bool l2 = L2;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = warp * rpw; c0 < nc; c0 += NW * rpw) {
        const int c = c0 + team;
        const bool valid = c < nc;
        const uint32_t id = valid ? (uint32_t)(cand[c] & 0xFFFFFFFFull) : 0u;
        const float sc = (STORE == ANN_STORE_E4M3 && valid) ? __ldg(scales + id) : 1.f;
        const uint4 *rp = rbase + (size_t)id * cpr;
        float2 acc = make_float2(0.f, 0.f);
        if (valid) {
            for (int ch0 = tl; ch0 < cpr; ch0 += ts * G) {
                uint4 v[G];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (ch0 + g * ts < cpr) v[g] = ld_row_chunk(rp + ch0 + g * ts);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (ch0 + g * ts < cpr) Chunk<STORE>::add(acc, v[g], qv + (ch0 + g * ts) * EPC, sc, l2);
            }
        }
        float r = acc.x + acc.y;
        for (int off = ts >> 1; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
        const entry_t e = pack_entry(l2 ? r : -r, id);
        const bool keep = tl == 0 && valid && e < limit;
        const unsigned bal = __ballot_sync(kFull, keep);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(out_n, __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (keep) out[base + __popc(bal & ((1u << lane) - 1u))] = e;
    }
}

template <int STORE, int NT, int G = 2>
__device__ __forceinline__ void compute_keys_teams(const void *rows, const float *scales, int row_elems, int metric,
                                                   const float *qv, const entry_t *cand, int nc, int lts,
                                                   entry_t limit, entry_t *out, int *out_n) {
    if (metric == ANN_METRIC_L2)
        compute_keys_teams_m<STORE, NT, true, G>(rows, scales, row_elems, qv, cand, nc, lts, limit, out, out_n);
    else
        compute_keys_teams_m<STORE, NT, false, G>(rows, scales, row_elems, qv, cand, nc, lts, limit, out, out_n);
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

// Direct-mapped visited cache: slot = hash(id); an insert exchanges the slot
// with id. Returns 0 if the slot already held id (visited), 1 if the slot was
// empty, 3 if another id was evicted (that id is now forgotten: it may be
// evaluated again, and the merge must drop ids already queued).
__device__ __forceinline__ int visited_exchange(uint32_t *table, int bits, uint32_t id) {
    const uint32_t h = (id * 0x9E3779B1u) >> (32 - bits);
    const uint32_t old = atomicExch(table + h, id);
    if (old == id) return 0;
    return old == kEmptySlot ? 1 : 3;
}

// Direct-mapped cache of W-byte tags (W = 1 or 2) over 2^bits slots. With
// b = bits + tag_bits >= the bits of any id, h = (id * odd constant) mod 2^b
// is a bijection on [0, 2^b): the top `bits` of h choose the slot and the low
// tag_bits of h are stored there (plus one; 0 = empty). (slot, tag) therefore
// names exactly one id: a slot never claims a vertex it did not see, it can
// only forget one when another takes its slot. Slots are updated with a
// 32-bit CAS on the word that holds them. Returns 0 if the id was present,
// 1 if it went into an empty slot, 3 if it replaced another vertex (or the
// CAS kept losing, which is treated the same way: a forgotten vertex only
// costs a repeated distance, and the merge drops an id that is queued twice).
template <int W>
__device__ __forceinline__ int visited_tag(uint32_t *table, int bits, int tag_bits, uint32_t id) {
    constexpr int PER = 4 / W;
    constexpr uint32_t MASK = W == 1 ? 0xFFu : 0xFFFFu;
    const int b = bits + tag_bits;
    uint32_t h = id * 0x9E3779B1u;
    if (b < 32) h &= (1u << b) - 1u;
    const uint32_t slot = h >> tag_bits;
    const uint32_t tag = (h & ((1u << tag_bits) - 1u)) + 1u;
    uint32_t *wp = table + slot / PER;
    const int sh = (int)(slot % PER) * 8 * W;
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(wp);
    for (int it = 0; it < 32; ++it) {
        const uint32_t cur = (old >> sh) & MASK;
        if (cur == tag) return 0;
        const uint32_t prev = atomicCAS(wp, old, (old & ~(MASK << sh)) | (tag << sh));
        if (prev == old) return cur == 0u ? 1 : 3;
        old = prev;
    }
    return 3;
}

// Set-associative visited cache: 2^bits sets of one 32-bit word, each word
// holding W fields of tag_bits + 1 bits (a tag plus one; 0 = an empty way),
// the newest in the lowest field. As in visited_tag, h = (id * odd constant)
// mod 2^b with b = bits + tag_bits >= the bits of any id is a bijection: the
// top `bits` of h choose the set and the low tag_bits are the tag, so (set,
// tag) names exactly one id and the cache never claims a vertex it did not
// see. An insert that finds the tag in one of the W fields returns 0; else
// the word shifts up by one field (first in, first out: the oldest way falls
// out) and the tag enters the lowest field, returning 1 if no vertex fell out
// and 3 if one was forgotten. The word is replaced with a CAS (a lost race
// re-reads the word; after 32 losses the vertex is treated as fresh, which
// only costs a repeated distance).
template <int W>
__device__ __forceinline__ int visited_assoc(uint32_t *table, int bits, int tag_bits, uint32_t id) {
    const int b = bits + tag_bits;
    uint32_t h = id * 0x9E3779B1u;
    if (b < 32) h &= (1u << b) - 1u;
    const uint32_t set = h >> tag_bits;
    const uint32_t tag = (h & ((1u << tag_bits) - 1u)) + 1u;
    const int fw = tag_bits + 1;  // W * fw <= 32 (host checks)
    const uint32_t fmask = (1u << fw) - 1u;
    const uint32_t wmask = W * fw >= 32 ? 0xFFFFFFFFu : (1u << (W * fw)) - 1u;
    uint32_t *wp = table + set;
    uint32_t old = *reinterpret_cast<volatile uint32_t *>(wp);
    for (int it = 0; it < 32; ++it) {
        bool seen = false;
#pragma unroll
        for (int w = 0; w < W; ++w) seen |= ((old >> (w * fw)) & fmask) == tag;
        if (seen) return 0;
        const uint32_t prev = atomicCAS(wp, old, ((old << fw) | tag) & wmask);
        if (prev == old) return ((old >> ((W - 1) * fw)) & fmask) ? 3 : 1;
        old = prev;
    }
    return 3;
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
template <int STORE, bool L2, int U>
__device__ __forceinline__ void warp_compute_keys_m(const void *rows, const float *scales, int row_elems,
                                                    const float *qv, entry_t *c, int nc) {
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31;
    const int cpr = row_elems / EPC;
    int ts = 1;
    while (ts < cpr && ts < 32) ts <<= 1;
    const int rpw = 32 / ts;
    const int team = lane / ts, tl = lane & (ts - 1);
    const int iters = (cpr + ts - 1) / ts;
    constexpr bool l2 = L2;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = 0; c0 < nc; c0 += rpw * U) {
        float2 acc[U];
        uint32_t id[U];
        bool valid[U];
        float sc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = c0 + u * rpw + team;
            valid[u] = j < nc;
            id[u] = valid[u] ? (uint32_t)(c[j] & 0xFFFFFFFFull) : 0u;
            acc[u] = make_float2(0.f, 0.f);
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
                if (valid[u] && ch < cpr) Chunk<STORE>::add(acc[u], v[u], qv + ch * EPC, sc[u], l2);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float r = acc[u].x + acc[u].y;
            for (int off = ts >> 1; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
            if (tl == 0 && valid[u]) c[c0 + u * rpw + team] = pack_entry(l2 ? r : -r, id[u]);
        }
    }
    __syncwarp();
}

template <int STORE, int U = 4>
__device__ __forceinline__ void warp_compute_keys(const void *rows, const float *scales, int row_elems,
                                                  int metric, const float *qv, entry_t *c, int nc) {
    if (metric == ANN_METRIC_L2)
        warp_compute_keys_m<STORE, true, U>(rows, scales, row_elems, qv, c, nc);
    else
        warp_compute_keys_m<STORE, false, U>(rows, scales, row_elems, qv, c, nc);
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

// Ascending sort of in[0..n), 32 < n <= NT, into out[0..n) (disjoint from
// in). Warp w sorts the run in[32w, 32w + 32) in registers and writes it
// back; each element's rank is then its lane plus, for every other run, the
// entries of that run below it (runs after its own) or not above it (runs
// before its own), by a branch-free binary search. Equal entries thus keep
// run order and every rank is distinct. Two barriers instead of the
// log^2-many of a bitonic sort. Ends with a __syncthreads().
template <int NT>
__device__ void block_rank_sort(entry_t *in, int n, entry_t *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = (n + 31) >> 5;
    entry_t v = kEmptyEntry;
    if (warp < S) {
        const int i = warp * 32 + lane;
        v = warp_sort32(i < n ? in[i] : kEmptyEntry);
        in[i] = v;
    }
    __syncthreads();
    if (warp < S && v != kEmptyEntry) {
        int r = lane;
        for (int s = 0; s < S; ++s) {
            if (s == warp) continue;
            const entry_t *A = in + 32 * s;
            const bool before = s < warp;
            int p = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const entry_t x = A[p + step - 1];
                if (before ? x <= v : x < v) p += step;
            }
            if (p == 31 && (before ? A[31] <= v : A[31] < v)) p = 32;
            r += p;
        }
        out[r] = v;
    }
    __syncthreads();
}

// Sorts in[0, n) ascending for n above a block's worth of entries: warps
// sort runs of 32 in registers, then log2(n / 32) rounds merge adjacent runs
// pairwise, each output placed by a merge-path co-rank search (ties taken
// from the left run), ping-ponging between in and tmp (n entries each).
// Returns the array holding the result; ends with a __syncthreads().
template <int NT>
__device__ entry_t *block_merge_sort(entry_t *in, int n, entry_t *tmp) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int S = (n + 31) >> 5;
    for (int r = warp; r < S; r += NW) {
        const int i = r * 32 + lane;
        const entry_t v = warp_sort32(i < n ? in[i] : kEmptyEntry);
        if (i < n) in[i] = v;
    }
    __syncthreads();
    entry_t *src = in, *dst = tmp;
    for (int w = 32; w < n; w <<= 1) {
        for (int i = threadIdx.x; i < n; i += NT) {
            const int p0 = i / (2 * w) * (2 * w);
            const int o = i - p0;
            const entry_t *A = src + p0;
            const int a = min(w, n - p0);
            const entry_t *B = A + a;
            const int b = max(0, min(w, n - p0 - w));
            int lo = max(0, o - b), hi = min(o, a);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A[mid] <= B[o - 1 - mid]) lo = mid + 1;
                else hi = mid;
            }
            const int kk = o - lo;
            dst[i] = (lo < a && (kk >= b || A[lo] <= B[kk])) ? A[lo] : B[kk];
        }
        __syncthreads();
        entry_t *t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// The k smallest of in[0..n) (k <= 32), ascending, at the front of the
// returned array (fewer if n < k). Warp w sorts runs of 32 in registers and
// keeps the first k of each in tmp; the c = ceil(n / 32) * k kept entries
// contain the k smallest and are sorted by one warp (c <= 32), by
// block_rank_sort into out (c <= NT), else by a bitonic sort over tmp. in is
// read only before the first barrier, so out may be in. tmp holds at least
// next_pow2(c) entries and out at least c. Ends with a __syncthreads().
// Returns the array the result is in (out or tmp).
template <int NT>
__device__ entry_t *block_topk(const entry_t *in, int n, int k, entry_t *tmp, entry_t *out) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int runs = (n + 31) >> 5;
    for (int r = warp; r < runs; r += NW) {
        const int i = r * 32 + lane;
        const entry_t v = warp_sort32(i < n ? in[i] : kEmptyEntry);
        if (lane < k) tmp[r * k + lane] = v;
    }
    const int c = runs * k;
    __syncthreads();
    if (c <= 32) {
        if (warp == 0) {
            const entry_t v = warp_sort32(lane < c ? tmp[lane] : kEmptyEntry);
            if (lane < k) out[lane] = v;
        }
        __syncthreads();
        return out;
    }
    if (c <= NT) {
        block_rank_sort<NT>(tmp, c, out);
        return out;
    }
    int P = 64;
    while (P < c) P <<= 1;
    for (int i = c + threadIdx.x; i < P; i += NT) tmp[i] = kEmptyEntry;
    __syncthreads();
    block_bitonic_sort<NT>(tmp, P);
    return tmp;
}

// Merge path: the first min(L, qlen + ns) entries of the merge of sorted
// Q[0..qlen) (ordered with the checked flag masked off) and sorted S[0..ns)
// (no entry of S equal to one of Q) go to out. Thread t owns a contiguous
// range of output positions: one binary search on its starting diagonal
// finds how many of its predecessors come from Q, then it merges its range
// sequentially. No barrier inside.
template <int NT>
__device__ __forceinline__ void block_merge_path(const entry_t *Q, int qlen, const entry_t *S, int ns, entry_t *out,
                                                 int L) {
    const int total = min(L, qlen + ns);
    const int per = (total + NT - 1) / NT;
    const int d0 = threadIdx.x * per;
    if (d0 >= total) return;
    const int d1 = min(d0 + per, total);
    int lo = max(0, d0 - ns), hi = min(d0, qlen);
    while (lo < hi) {  // the smallest i with Q[i] after S[d0 - 1 - i]
        const int i = (lo + hi) >> 1;
        if ((Q[i] & kMask) < S[d0 - 1 - i]) lo = i + 1;
        else hi = i;
    }
    int i = lo, j = d0 - lo;
    for (int d = d0; d < d1; ++d) {
        const bool takeQ = j >= ns || (i < qlen && (Q[i] & kMask) < S[j]);
        out[d] = takeQ ? Q[i++] : S[j++];
    }
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

// ------------------------------------------------------- warp row gathers
// Keys of the nf candidates fr[0..nf) (one warp): fr[c].x is the vertex id
// and fr[c].y the row that holds its vector (the id itself, or a row of a
// neighbour group). Teams of 2^lts lanes per row; each lane walks its own
// 16-byte chunks of the row, G of them in flight. The warp takes passes
// pass_begin, pass_begin + pass_step, ... of 32 >> lts candidates.
// Candidates below `limit` are appended to out[] through the shared counter
// *out_n. No barrier.
template <int STORE, int G, bool L2>
__device__ __forceinline__ void warp_keys_append_m(const void *rows, const float *scales, uint32_t cpr,
                                                   const float *qv, const uint2 *fr, int nf, int lts,
                                                   entry_t limit, entry_t *out, int *out_n, int pass_begin = 0,
                                                   int pass_step = 1) {
    constexpr int EPC = Chunk<STORE>::kElems;
    const int lane = threadIdx.x & 31;
    const int ts = 1 << lts, rpw = 32 >> lts;
    const int team = lane >> lts, tl = lane & (ts - 1);
    constexpr bool l2 = L2;
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows);
    for (int c0 = pass_begin * rpw; c0 < nf; c0 += pass_step * rpw) {
        const int c = c0 + team;
        const bool valid = c < nf;
        const uint2 f = valid ? fr[c] : make_uint2(0u, 0u);
        const uint32_t id = f.x;
        const float sc = (STORE == ANN_STORE_E4M3 && valid) ? __ldg(scales + f.y) : 1.f;
        const uint4 *rp = rbase + (size_t)f.y * cpr;
        float2 acc = make_float2(0.f, 0.f);
        if (valid) {
            for (uint32_t ch0 = tl; ch0 < cpr; ch0 += ts * G) {
                uint4 v[G];
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (ch0 + g * ts < cpr) v[g] = ld_row_chunk(rp + ch0 + g * ts);
#pragma unroll
                for (int g = 0; g < G; ++g)
                    if (ch0 + g * ts < cpr) Chunk<STORE>::add(acc, v[g], qv + (ch0 + g * ts) * EPC, sc, l2);
            }
        }
        float r = acc.x + acc.y;
        for (int off = ts >> 1; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
        const entry_t e = pack_entry(l2 ? r : -r, id);
        const bool keep = tl == 0 && valid && e < limit;
        const unsigned bal = __ballot_sync(kFull, keep);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(out_n, __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (keep) out[base + __popc(bal & ((1u << lane) - 1u))] = e;
    }
}

// The same contract as warp_keys_append_m for rows of exactly CPL << LTS
// chunks: the team size, the chunks each lane reads and the rounds of G
// loads in flight are compile-time constants, so the gather has no bounds
// test per chunk and no runtime shift or loop count. The candidates are the
// (id, row) pairs fr[], or, when list is given, the ids in the low words of
// list[] (each the row of its own vector). Candidates c_begin,
// c_begin + c_step, ... in passes of 32 >> LTS; a lane past the end of the
// list re-reads a valid row and its key is dropped.
template <int STORE, bool L2, int LTS, int CPL, int G>
__device__ __forceinline__ void warp_keys_fixed(const void *rows, const float *scales, const float *qv,
                                                const entry_t *list, const uint2 *fr, int nf, int c_begin,
                                                int c_step, entry_t limit, entry_t *out, int *out_n) {
    static_assert(CPL % G == 0, "rounds of G chunks must cover the lane's chunks");
    constexpr int EPC = Chunk<STORE>::kElems;
    constexpr int TS = 1 << LTS, RPW = 32 >> LTS, CPR = CPL * TS;
    const int lane = threadIdx.x & 31;
    const int team = lane >> LTS, tl = lane & (TS - 1);
    const uint4 *rbase = reinterpret_cast<const uint4 *>(rows) + tl;
    const float *qt = qv + tl * EPC;
    for (int c0 = c_begin; c0 < nf; c0 += c_step) {
        const int c = c0 + team;
        const bool valid = c < nf;
        const int cc = valid ? c : c0;
        uint32_t id, row;
        if (list) {
            id = row = (uint32_t)(list[cc] & 0xFFFFFFFFull);
        } else {
            const uint2 f = fr[cc];
            id = f.x;
            row = f.y;
        }
        const float sc = STORE == ANN_STORE_E4M3 ? __ldg(scales + row) : 1.f;
        const uint4 *rp = rbase + (size_t)row * CPR;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int r0 = 0; r0 < CPL; r0 += G) {
            uint4 v[G];
#pragma unroll
            for (int g = 0; g < G; ++g) v[g] = ld_row_chunk(rp + (r0 + g) * TS);
#pragma unroll
            for (int g = 0; g < G; ++g) Chunk<STORE>::add(acc, v[g], qt + (r0 + g) * TS * EPC, sc, L2);
        }
        float r = acc.x + acc.y;
#pragma unroll
        for (int off = TS >> 1; off > 0; off >>= 1) r += __shfl_xor_sync(kFull, r, off);
        const entry_t e = pack_entry(L2 ? r : -r, id);
        const bool keep = tl == 0 && valid && e < limit;
        const unsigned bal = __ballot_sync(kFull, keep);
        int base = 0;
        if (lane == 0 && bal) base = atomicAdd(out_n, __popc(bal));
        base = __shfl_sync(kFull, base, 0);
        if (keep) out[base + __popc(bal & ((1u << lane) - 1u))] = e;
        (void)RPW;
    }
}

// Row shapes with a fixed-geometry gather (the workloads' 32-, 96-, 128- and
// 960-dimensional rows at the automatic team size); other shapes take the
// generic loop. Returns false if the shape has no fixed form.
template <int STORE, bool L2>
__device__ __forceinline__ bool gather_fixed(const void *rows, const float *scales, uint32_t cpr, int lts,
                                             const float *qv, const entry_t *list, const uint2 *fr, int nf,
                                             int c_begin, int c_step_rows, entry_t limit, entry_t *out,
                                             int *out_n) {
#define ANN_FIXED(LTS_, CPL_, G_)                                                                            \
    if (lts == LTS_ && cpr == (uint32_t)((CPL_) << (LTS_))) {                                                \
        warp_keys_fixed<STORE, L2, LTS_, CPL_, G_>(rows, scales, qv, list, fr, nf, c_begin << (5 - (LTS_)),  \
                                                   c_step_rows << (5 - (LTS_)), limit, out, out_n);          \
        return true;                                                                                         \
    }
    if constexpr (STORE == ANN_STORE_BF16 || STORE == ANN_STORE_F16) {
        ANN_FIXED(2, 4, 4)   // 128-d
        ANN_FIXED(2, 3, 3)   // 96-d
        ANN_FIXED(3, 15, 5)  // 960-d
    } else if constexpr (STORE == ANN_STORE_F32) {
        ANN_FIXED(2, 8, 4)   // 128-d
        ANN_FIXED(2, 6, 3)   // 96-d
        ANN_FIXED(2, 2, 2)   // 32-d
        ANN_FIXED(3, 30, 5)  // 960-d
    } else {
        ANN_FIXED(2, 15, 5)  // 960-d
        ANN_FIXED(2, 2, 2)   // 128-d
    }
#undef ANN_FIXED
    return false;
}

// ------------------------------------------------------- one search step

// One insert into the query's visited set, whichever form it has: 0 = was
// present, 1 = inserted, 2 or 3 = inserted while another vertex may have been
// forgotten (probe limit, eviction).
__device__ __forceinline__ int visit_set(uint32_t *table, const SearchArgs &a, uint32_t id) {
    if (a.ways == 3) return visited_assoc<3>(table, a.hash_bits, a.tag_bits, id);
    if (a.ways == 2) return visited_assoc<2>(table, a.hash_bits, a.tag_bits, id);
    if (a.visited_mode == 0) return visited_insert(table, a.hash_bits, id);
    if (a.slot_bytes == 1) return visited_tag<1>(table, a.hash_bits, a.tag_bits, id);
    if (a.slot_bytes == 2) return visited_tag<2>(table, a.hash_bits, a.tag_bits, id);
    return visited_exchange(table, a.hash_bits, id);
}

// One warp's share of a step's expansion: the step's nact * R adjacency
// slots (slot i is slot i mod R of selected vertex sel_id[i / R]; r_recip =
// ceil(2^32 / R) makes i / R one umulhi) are split evenly over the NW warps.
// Each neighbour that the visited set did not hold is appended, as an (id,
// row) pair, to this warp's list `fresh` (or, if `block` is given, to one list
// for the CTA through the counter *block_n), and its row is asked of L2. With
// owners > 1 (a power of two) only vertices u with u mod owners == owner are
// inserted and listed: the vertices this CTA of a cluster owns. A hot vertex
// of a neighbour grouping gives its neighbours' rows in its group block
// (one bulk prefetch for the block). Sets *unsafe if an insert may have
// forgotten another vertex. Returns the fresh vertices this warp found.
// The step's selection (Sec. 4.1, top-M): the first Mcur unchecked entries
// of the stable queue Q[0, qlen) in queue order, taken into sel_id / sel_pos
// by rank. The scan starts at first_un (every entry before it is checked)
// and covers NW * 32 entries per round, one 32-entry chunk per warp; a block
// scan of the warps' counts gives each chunk its first rank. Returns, in
// every thread, the number of unchecked entries seen (at least the number
// taken); *sel_last gets the queue position of the last entry taken (-1 if
// none). wcnt is NW ints of shared memory. Every thread of the block must
// call it; when the scan ran, it ends with a barrier.
template <int NW>
__device__ __forceinline__ int select_unchecked(const entry_t *Q, int qlen, int first_un, int Mcur, int *sel_id,
                                                int *sel_pos, int *wcnt, int *sel_last) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (threadIdx.x == 0) *sel_last = -1;
    int found = 0;
    for (int base = first_un & ~31; found < Mcur && base < qlen; base += NW * 32) {
        const int i = base + warp * 32 + lane;
        const entry_t e = i < qlen ? Q[i] : kChecked;
        const bool un = !(e & kChecked);
        const unsigned bal = __ballot_sync(kFull, un);
        if (lane == 0) wcnt[warp] = __popc(bal);
        __syncthreads();
        int total = 0, pre = 0;
#pragma unroll
        for (int w2 = 0; w2 < NW; ++w2) {
            const int c = wcnt[w2];
            total += c;
            pre += w2 < warp ? c : 0;
        }
        const int r = found + pre + __popc(bal & lt_mask);
        const bool take = un && r < Mcur;
        if (take) {
            sel_id[r] = (int)entry_id(e);
            sel_pos[r] = i;
        }
        const unsigned tb = __ballot_sync(kFull, take);
        if (tb && lane == 0) atomicMax(sel_last, base + warp * 32 + 31 - __clz(tb));
        found += total;
        __syncthreads();
    }
    return found;
}

// The same selection scanned by warp 0 alone, 32 entries per round, then
// one barrier. With eight warps or fewer (the small CTAs that run many
// queries per SM) this keeps the step's live state in registers; the
// block-wide scan above serves the larger CTAs that run one query alone.
template <int NW>
__device__ __forceinline__ int select_step(const entry_t *Q, int qlen, int first_un, int Mcur, int *sel_id,
                                           int *sel_pos, int *wcnt, int *sel_last) {
    if constexpr (NW >= 16) {
        return select_unchecked<NW>(Q, qlen, first_un, Mcur, sel_id, sel_pos, wcnt, sel_last);
    } else {
        const int lane = threadIdx.x & 31;
        if ((threadIdx.x >> 5) == 0) {
            int found = 0, last_pos = -1;
            for (int b = first_un & ~31; b < qlen && found < Mcur; b += 32) {
                const int i = b + lane;
                const entry_t e = i < qlen ? Q[i] : kChecked;
                const bool un = !(e & kChecked);
                const unsigned bal = __ballot_sync(kFull, un);
                const int r = found + __popc(bal & ((1u << lane) - 1u));
                const bool take = un && r < Mcur;
                if (take) {
                    sel_id[r] = (int)entry_id(e);
                    sel_pos[r] = i;
                }
                const unsigned tb = __ballot_sync(kFull, take);
                if (tb) last_pos = b + 31 - __clz(tb);
                found += __popc(bal);
            }
            if (lane == 0) {
                wcnt[0] = found;
                *sel_last = last_pos;
            }
        }
        __syncthreads();
        return wcnt[0];
    }
}

template <int NW>
__device__ __forceinline__ int expand_step(const SearchArgs &a, uint32_t *table, const int *sel_id, int nact,
                                           uint32_t r_recip, uint32_t row_bytes, uint2 *fresh, uint2 *block,
                                           int *block_n, int owners, int owner, int *unsafe) {
    constexpr int KA = 4;  // slots per lane whose loads are in flight together
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = a.R;
    const int total = nact * R;
    const int per = (total + NW - 1) / NW;
    const int beg = warp * per, end = min(beg + per, total);
    int nf = 0;
    for (int b0 = beg; b0 < end; b0 += 32 * KA) {
        int u[KA];
        uint32_t urow[KA];  // the row holding u's vector: u, or its copy in a neighbour group
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            const int i = b0 + kk * 32 + lane;
            u[kk] = -1;
            urow[kk] = 0;
            if (i < end) {
                const uint32_t j = __umulhi((uint32_t)i, r_recip);
                const uint32_t slot = (uint32_t)i - j * (uint32_t)R;
                const uint32_t v = (uint32_t)sel_id[j];
                u[kk] = __ldg(a.adj + (size_t)v * (uint32_t)R + slot);
                if (owners > 1 && u[kk] >= 0 && ((uint32_t)u[kk] & (uint32_t)(owners - 1)) != (uint32_t)owner)
                    u[kk] = -1;
                urow[kk] = (uint32_t)u[kk];
                if (a.hot_slot) {
                    // a hot vertex: its neighbours' rows lie in one block after the base rows, in adjacency
                    // order; one bulk prefetch (from the lane with its first slot) asks L2 for the block
                    const int hs = __ldg(a.hot_slot + v);
                    if (hs >= 0) {
                        const uint32_t r0 = (uint32_t)a.n + (uint32_t)hs * (uint32_t)R;
                        urow[kk] = r0 + slot;
                        if (slot == 0 && a.l2_prefetch && a.group_prefetch == 0)
                            prefetch_range_l2(static_cast<const char *>(a.base) + (size_t)r0 * row_bytes,
                                              (uint32_t)R * row_bytes);
                    }
                }
            }
        }
        unsigned fr = 0;  // bit kk: u[kk] was not in the visited set
        bool forgot = false;
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            if (u[kk] >= 0) {
                const int ins = visit_set(table, a, (uint32_t)u[kk]);
                if (ins != 0) fr |= 1u << kk;
                if (ins >= 2) forgot = true;
            }
        }
        if (forgot) *unsafe = 1;  // a vertex may have been forgotten: repeats possible
        const int cnt = __popc(fr);
        int incl = cnt;  // inclusive scan of the per-lane counts
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += v;
        }
        const int wtot = __shfl_sync(kFull, incl, 31);
        int pos;
        if (block) {  // one list for the whole CTA
            int base = 0;
            if (lane == 31 && wtot) base = atomicAdd(block_n, wtot);
            pos = __shfl_sync(kFull, base, 31) + incl - cnt;
        } else {
            pos = nf + incl - cnt;
        }
        uint2 *dst = block ? block : fresh;
#pragma unroll
        for (int kk = 0; kk < KA; ++kk) {
            if (fr >> kk & 1u) {
                dst[pos++] = make_uint2((uint32_t)u[kk], urow[kk]);
                if (a.l2_prefetch && (urow[kk] < (uint32_t)a.n || a.group_prefetch))
                    prefetch_row_l2(a.base, row_bytes, urow[kk]);
            }
        }
        nf += wtot;
    }
    return nf;
}

// The ns (> 0) survivors in surv, sorted by (key, id) (one warp for 32 or
// fewer, a bitonic sort in place up to 64, warp runs plus binary-search ranks
// into `scratch` up to NT, else warp runs merged pairwise between surv and
// `scratch`), are merged into the sorted queue Q[0..qlen): when
// `unsafe` (the visited set may have forgotten a vertex) survivors whose id
// is already queued, or repeated, are dropped first (counted in *dropped).
// The first min(L, qlen + kept) entries go to Qn by merge path. *first_un
// (every entry before it is checked) is lowered to the first survivor's new
// rank. Every thread calls it with the same arguments; it ends with a
// barrier. Returns the number of survivors kept.
template <int NT>
__device__ __forceinline__ int sort_dedupe_merge(const entry_t *Q, int qlen, entry_t *surv, int ns, entry_t *scratch,
                                                 entry_t *Qn, int L, bool unsafe, unsigned char *dup, int *anydup,
                                                 long long *dropped, int *first_un) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
        block_rank_sort<NT>(surv, ns, scratch);
        srt = scratch;
    } else if (ns > NT) {
        srt = block_merge_sort<NT>(surv, ns, scratch);
    } else {
        int P = 64;
        while (P < ns) P <<= 1;
        for (int i = ns + tid; i < P; i += NT) surv[i] = kEmptyEntry;
        __syncthreads();
        block_bitonic_sort<NT>(surv, P);
    }
    int ncl = ns;
    if (unsafe) {
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
                if (lane == 0) *anydup = outp;
            }
            __syncthreads();
            ncl = *anydup;
            if (tid == 0) *dropped += ns - ncl;
        }
    }
    // the first survivor's rank among the old entries bounds the new queue's checked prefix
    if (tid == 0 && ncl > 0) {
        const int p0 = count_below(Q, qlen, srt[0]);
        if (p0 < *first_un) *first_un = p0;
    }
    block_merge_path<NT>(Q, qlen, srt, ncl, Qn, L);
    __syncthreads();  // the new queue is complete; nothing of the old one is read again
    return ncl;
}

}  // namespace ann
