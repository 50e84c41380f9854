// knn.cu -- brute-force k nearest neighbours over BF16 rows, for building the
// similarity graph the search runs on (the paper takes the graph as given:
// Sec. 2.2 builds on proximity graphs such as NSG and HNSW; its k-NN
// candidate lists are the exact Def. 1 neighbours of every base point).
//
// The distance matrix of a brute-force scan is n x n (10^14 entries at 10M
// points), so it must never reach HBM: each CTA holds 128 query rows as
// tensor-core operands in registers, streams the whole base set through
// shared memory in tiles of 128 rows (cp.async, 3-4 tiles in flight), forms each
// 128 x 128 distance tile with mma.sync m16n8k16 (BF16 in, FP32 accumulate)
// and keeps, per query row, its best 64 (key, id) pairs in shared memory.
// A tile's distances pass a per-row threshold (the row's current 64th key)
// into a per-row candidate buffer; a full buffer triggers a merge of the
// buffer into the row's sorted list, after which the tile's remaining
// values are offered again against the tightened threshold.
//
// BF16 x BF16 products are exact in FP32; sums are FP32. Keys are the FP32
// distance (squared l2, or -<q, x>) under an order-preserving map to
// unsigned, so (key, id) sorts like (distance, id).
#include <cuda_bf16.h>

#include "ann_internal.cuh"

namespace ann {
namespace {

constexpr int KBM = 128;    // query rows per CTA
constexpr int KBN = 128;    // base rows per tile
constexpr int KLIST = 64;   // list length per query row
constexpr int KCAP = 32;    // candidate buffer per query row
constexpr int KNT = 256;    // 8 warps: 4 along the query rows x 2 along the tile's base rows
constexpr unsigned long long KMAX = ~0ull;

__device__ __forceinline__ uint32_t ord_enc(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ord_dec(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}

__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8x8 BF16 matrices; lane i names row i % 8 of matrix i / 8.
__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], uint32_t saddr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(saddr));
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *gmem, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct KnnSmem {
    unsigned long long *list;  // [KBM][KLIST], ascending
    unsigned long long *cand;  // [KBM][KCAP], unsorted
    __nv_bfloat16 *tile;       // [stages][KBN][pitch]
    float *bnorm;              // [stages][KBN]
    float *qnorm;              // [KBM]
    float *thr;                // [KBM] current 64th key as a distance (+inf while the list is not full)
    float *tfast;              // [KBM] filter bound of the fast test (see knn_fast_bound)
    int *cnt;                  // [KBM] appends since the last merge (may pass KCAP on overflow)
    int *flags;                // [0] overflow in the last pass, [1] merge rounds exhausted
};

__host__ __device__ constexpr int knn_pitch(int d) { return d + 8; }

// Base tiles in flight: four while they fit beside the lists.
__host__ __device__ constexpr int knn_stages(int d) { return d <= 96 ? 4 : 3; }

__host__ __device__ inline size_t knn_smem_bytes(int d) {
    return (size_t)KBM * KLIST * 8 + (size_t)KBM * KCAP * 8 + (size_t)knn_stages(d) * KBN * knn_pitch(d) * 2 +
           knn_stages(d) * KBN * 4 + 4 * KBM * 4 + 16;
}

// The fast test compares fma(-2, v, |x|^2) against thr - |q|^2 without
// forming the key. Rounding can move the two sides apart by a few units in
// the last place of the larger magnitude, so the bound is widened by 8 ulp:
// every value whose key is <= thr passes it (the exact test follows).
__device__ __forceinline__ float knn_fast_bound(float thr, float qn, bool l2) {
    if (!l2) return thr;
    const float t = thr - qn;
    return t + 8.f * 1.1920929e-7f * fmaxf(fabsf(thr), fabsf(qn));
}

// Sort the row's candidates (warp bitonic, one per lane) and merge them into
// its list with a merge-path co-rank search per output; keys are unique
// (every base row is offered once per query row).
__device__ void knn_merge_row(const KnnSmem &s, int row, int lane, bool l2) {
    unsigned long long *L = s.list + (size_t)row * KLIST;
    unsigned long long *C = s.cand + (size_t)row * KCAP;
    const int c = min(s.cnt[row], KCAP);
    unsigned long long x = lane < c ? C[lane] : KMAX;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j >= 1; j >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x, j);
            const bool keep_min = ((lane & k) == 0) == ((lane & j) == 0);
            x = keep_min ? min(x, y) : max(x, y);
        }
    }
    __syncwarp();
    C[lane] = x;
    __syncwarp();
    unsigned long long out[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        int lo = max(0, i - KCAP), hi = min(i, KLIST);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (L[mid] < C[i - 1 - mid]) lo = mid + 1;
            else hi = mid;
        }
        const unsigned long long a = lo < KLIST ? L[lo] : KMAX;
        const unsigned long long b = i - lo < KCAP ? C[i - lo] : KMAX;
        out[h] = min(a, b);
    }
    __syncwarp();
    L[lane] = out[0];
    L[lane + 32] = out[1];
    __syncwarp();
    if (lane == 0) {
        const unsigned long long last = L[KLIST - 1];
        const float thr = last == KMAX ? __int_as_float(0x7F800000) : ord_dec((uint32_t)(last >> 32));
        s.thr[row] = thr;
        s.tfast[row] = knn_fast_bound(thr, s.qnorm[row], l2);
        s.cnt[row] = 0;
    }
    __syncwarp();
}

// Offer a thread's tile values (acc) to the candidate buffers by their exact
// key. A thread holds 16 values of each of 4 query rows (row group
// rg = 2 mi + h). rows != 0: the first offer, of every value of the row
// groups set in rows; rows == 0: offer again only the values flagged in pend
// (their row's buffer was full when they were offered).
template <bool L2>
__device__ __forceinline__ void knn_offer(const KnnSmem &s, const float (&acc)[2][8][4], unsigned long long &pend,
                                       unsigned rows, int stage, int64_t col0, int64_t n, int64_t m0, int64_t nq,
                                       int64_t self0, int warp_m, int warp_n, int g, int t) {
    const bool first = rows != 0;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int rg = mi * 2 + h;
            if (first ? !((rows >> rg) & 1u) : ((pend >> (rg * 16)) & 0xFFFFull) == 0) continue;
            const int row = warp_m * 32 + mi * 16 + h * 8 + g;
            const float thr = s.thr[row];
            const float qn = L2 ? s.qnorm[row] : 0.f;
            const int64_t self = self0 >= 0 ? self0 + m0 + row : -1;
            const bool rv = m0 + row < nq;
#pragma unroll
            for (int ni = 0; ni < 8; ++ni) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int bit = ((mi * 2 + h) * 8 + ni) * 2 + e;
                    const unsigned long long m = 1ull << bit;
                    if (!first && !(pend & m)) continue;
                    const int cl = warp_n * 64 + ni * 8 + 2 * t + e;
                    const int64_t col = col0 + cl;
                    const float v = acc[mi][ni][h * 2 + e];
                    const float dist = L2 ? fmaxf(fmaf(-2.f, v, s.bnorm[stage * KBN + cl]) + qn, 0.f) : -v;
                    if (dist <= thr && rv && col < n && col != self) {
                        const unsigned long long key = ((unsigned long long)ord_enc(dist) << 32) | (uint32_t)col;
                        const int slot = atomicAdd(&s.cnt[row], 1);
                        if (slot < KCAP) {
                            s.cand[(size_t)row * KCAP + slot] = key;
                            pend &= ~m;
                        } else {
                            pend |= m;
                            s.flags[0] = 1;
                        }
                    } else {
                        pend &= ~m;
                    }
                }
            }
        }
    }
}

template <int KS, bool L2>
__global__ void __launch_bounds__(KNT, 1)
    knn_bf16_kernel(const __nv_bfloat16 *__restrict__ base, const float *__restrict__ bnorm_g, int64_t n,
                    const __nv_bfloat16 *__restrict__ queries, int64_t nq, int64_t self0, int k,
                    int32_t *__restrict__ out_ids, float *__restrict__ out_d, int *__restrict__ err) {
    constexpr int D = KS * 16;
    constexpr int P = knn_pitch(D);
    constexpr int CPR = D / 8;  // 16-byte chunks per row
    constexpr int TILE_BYTES = KBN * P * 2;
    constexpr int KSTAGES = knn_stages(D);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    KnnSmem s;
    {
        unsigned char *p = smem_raw;
        s.list = reinterpret_cast<unsigned long long *>(p);
        p += (size_t)KBM * KLIST * 8;
        s.cand = reinterpret_cast<unsigned long long *>(p);
        p += (size_t)KBM * KCAP * 8;
        s.tile = reinterpret_cast<__nv_bfloat16 *>(p);
        p += (size_t)KSTAGES * TILE_BYTES;
        s.bnorm = reinterpret_cast<float *>(p);
        p += KSTAGES * KBN * 4;
        s.qnorm = reinterpret_cast<float *>(p);
        p += KBM * 4;
        s.thr = reinterpret_cast<float *>(p);
        p += KBM * 4;
        s.tfast = reinterpret_cast<float *>(p);
        p += KBM * 4;
        s.cnt = reinterpret_cast<int *>(p);
        p += KBM * 4;
        s.flags = reinterpret_cast<int *>(p);
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int warp_m = warp & 3, warp_n = warp >> 2;
    const int g = lane >> 2, t = lane & 3;
    const int64_t m0 = (int64_t)blockIdx.x * KBM;
    const int64_t ntiles = (n + KBN - 1) / KBN;
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(s.tile);
    const uint32_t bnorm_s = (uint32_t)__cvta_generic_to_shared(s.bnorm);

    // Tiles past the end are committed as empty groups so that the
    // wait_group count stays uniform.
    auto load_tile = [&](int64_t j) {
        if (j < ntiles) {
            const int stage = (int)(j % KSTAGES);
            const uint32_t dst = tile_s + stage * TILE_BYTES;
            for (int c = tid; c < KBN * CPR; c += KNT) {
                const int r = c / CPR, ch = c - r * CPR;
                const int64_t br = j * KBN + r;
                const bool ok = br < n;
                cp_async16(dst + (r * P + ch * 8) * 2, base + (ok ? br : 0) * D + ch * 8, ok);
            }
            if (L2 && tid < KBN / 4)
                cp_async16(bnorm_s + (stage * KBN + tid * 4) * 4, bnorm_g + j * KBN + tid * 4, true);
        }
        cp_async_commit();
    };

#pragma unroll
    for (int j = 0; j < KSTAGES - 1; ++j) load_tile(j);

    // Query operands (A fragments of m16n8k16, row-major) stay in registers.
    uint32_t a[2][KS][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int64_t r0 = m0 + warp_m * 32 + mi * 16 + g, r1 = r0 + 8;
        const uint32_t *q0 = reinterpret_cast<const uint32_t *>(queries + (r0 < nq ? r0 : 0) * D);
        const uint32_t *q1 = reinterpret_cast<const uint32_t *>(queries + (r1 < nq ? r1 : 0) * D);
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
            a[mi][ks][0] = r0 < nq ? q0[ks * 8 + t] : 0u;
            a[mi][ks][1] = r1 < nq ? q1[ks * 8 + t] : 0u;
            a[mi][ks][2] = r0 < nq ? q0[ks * 8 + 4 + t] : 0u;
            a[mi][ks][3] = r1 < nq ? q1[ks * 8 + 4 + t] : 0u;
        }
    }
    for (int r = tid; r < KBM; r += KNT) {
        float acc = 0.f;
        if (L2 && m0 + r < nq) {
            const __nv_bfloat16 *q = queries + (m0 + r) * D;
            for (int i = 0; i < D; ++i) {
                const float v = __bfloat162float(q[i]);
                acc = fmaf(v, v, acc);
            }
        }
        s.qnorm[r] = acc;
        s.thr[r] = __int_as_float(0x7F800000);
        s.tfast[r] = __int_as_float(0x7F800000);
        s.cnt[r] = 0;
    }
    for (int i = tid; i < KBM * KLIST; i += KNT) s.list[i] = KMAX;
    if (tid == 0) s.flags[0] = s.flags[1] = 0;

    // ldmatrix row address of this lane: matrix q = lane / 8 covers base
    // rows (q / 2) * 8 .. +7 of an n-tile pair and k-half q % 2.
    const uint32_t lm_off =
        (uint32_t)(((warp_n * 64 + (lane >> 4) * 8 + (lane & 7)) * P + ((lane >> 3) & 1) * 8) * 2);

    // Query rows whose own base row may fall inside a tile, ragged tiles and
    // the last CTA's missing rows go through the exact offer for every value.
    const int64_t self_lo = self0 >= 0 ? self0 + m0 : -1;

    float acc[2][8][4];
    unsigned long long pend = 0;
    int prev_stage = 0;
    int64_t prev_col0 = 0;

    // Overflow of the previous tile: merge the fuller rows, then offer the
    // values that found no slot again. Each round empties every overflowed
    // row and a row is offered at most KBN values per tile, so KBN / KCAP
    // rounds suffice; the bound only guards against a broken invariant.
    auto drain = [&]() {
        for (int round = 0; s.flags[0]; ++round) {
            __syncthreads();
            if (round > KBN / KCAP + 1) {
                if (tid == 0) s.flags[1] = 1;
                break;
            }
            if (tid == 0) s.flags[0] = 0;
            for (int row = warp; row < KBM; row += KNT / 32)
                if (s.cnt[row] >= KCAP / 2) knn_merge_row(s, row, lane, L2);
            __syncthreads();
            if (pend)
                knn_offer<L2>(s, acc, pend, 0u, prev_stage, prev_col0, n, m0, nq, self0, warp_m, warp_n, g, t);
            __syncthreads();
        }
    };

    for (int64_t j = 0; j < ntiles; ++j) {
        const int stage = (int)(j % KSTAGES);
        cp_async_wait<KSTAGES - 2>();
        __syncthreads();
        drain();
        load_tile(j + KSTAGES - 1);  // into the stage of tile j - 1, no longer read

#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int ni = 0; ni < 8; ++ni)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[mi][ni][c] = 0.f;
        const uint32_t tb = tile_s + stage * TILE_BYTES + lm_off;
#pragma unroll
        for (int ks = 0; ks < KS; ++ks) {
#pragma unroll
            for (int np = 0; np < 4; ++np) {
                uint32_t b[4];
                ldmatrix_x4(b, tb + (np * 16 * P + ks * 16) * 2);
                mma_bf16_16816(acc[0][2 * np], a[0][ks], b[0], b[1]);
                mma_bf16_16816(acc[1][2 * np], a[1][ks], b[0], b[1]);
                mma_bf16_16816(acc[0][2 * np + 1], a[0][ks], b[2], b[3]);
                mma_bf16_16816(acc[1][2 * np + 1], a[1][ks], b[2], b[3]);
            }
        }

        const int64_t col0 = j * KBN;
        const bool check = (col0 + KBN > n) || m0 + KBM > nq ||
                           (self_lo >= 0 && col0 < self_lo + KBM && self_lo < col0 + KBN);
        // Fast test per row group: the smallest of its 16 values (a min tree)
        // against the row's widened bound.
        unsigned hit = check ? 0xFu : 0u;
        if (!check) {
            float bn[16];
#pragma unroll
            for (int ni = 0; ni < 8; ++ni) {
                if (L2) {
                    const float2 b2 =
                        *reinterpret_cast<const float2 *>(s.bnorm + stage * KBN + warp_n * 64 + ni * 8 + 2 * t);
                    bn[2 * ni] = b2.x;
                    bn[2 * ni + 1] = b2.y;
                } else {
                    bn[2 * ni] = bn[2 * ni + 1] = 0.f;
                }
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float tf = s.tfast[warp_m * 32 + mi * 16 + h * 8 + g];
                    float x[16];
#pragma unroll
                    for (int ni = 0; ni < 8; ++ni)
#pragma unroll
                        for (int e = 0; e < 2; ++e)
                            x[2 * ni + e] = L2 ? fmaf(-2.f, acc[mi][ni][h * 2 + e], bn[2 * ni + e])
                                               : -acc[mi][ni][h * 2 + e];
#pragma unroll
                    for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
                        for (int i = 0; i < w; ++i) x[i] = fminf(x[i], x[i + w]);
                    hit |= (x[0] <= tf ? 1u : 0u) << (mi * 2 + h);
                }
            }
        }
        pend = 0;
        if (hit) knn_offer<L2>(s, acc, pend, hit, stage, col0, n, m0, nq, self0, warp_m, warp_n, g, t);
        prev_stage = stage;
        prev_col0 = col0;
    }
    cp_async_wait<0>();
    __syncthreads();
    drain();

    for (int row = warp; row < KBM; row += KNT / 32)
        if (s.cnt[row] > 0) knn_merge_row(s, row, lane, L2);
    __syncthreads();
    if (tid == 0 && s.flags[1]) atomicExch(err, 1);
    for (int i = tid; i < KBM * k; i += KNT) {
        const int row = i / k, c = i - row * k;
        if (m0 + row >= nq) continue;
        const unsigned long long key = s.list[(size_t)row * KLIST + c];
        const size_t o = (size_t)(m0 + row) * k + c;
        if (key == KMAX) {
            out_ids[o] = -1;
            out_d[o] = __int_as_float(0x7F800000);
        } else {
            out_ids[o] = (int32_t)(uint32_t)key;
            out_d[o] = ord_dec((uint32_t)(key >> 32));
        }
    }
}

// Squared norms of BF16 rows in FP32 (the same sum order as the kernel's
// query norms), zero for the padding rows up to n_pad.
__global__ void bf16_row_norms(const __nv_bfloat16 *__restrict__ x, int64_t n, int64_t n_pad, int d,
                               float *__restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    float acc = 0.f;
    if (r < n) {
        const __nv_bfloat16 *p = x + r * d;
        for (int i = 0; i < d; ++i) {
            const float v = __bfloat162float(p[i]);
            acc = fmaf(v, v, acc);
        }
    }
    out[r] = acc;
}

template <int KS, bool L2>
cudaError_t launch_knn_t(const void *base, const float *norms, int64_t n, const void *queries, int64_t nq,
                         int64_t self0, int k, int32_t *ids, float *dists, int *err, cudaStream_t stream) {
    const size_t smem = knn_smem_bytes(KS * 16);
    cudaError_t e = cudaFuncSetAttribute(knn_bf16_kernel<KS, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = (nq + KBM - 1) / KBM;
    knn_bf16_kernel<KS, L2><<<(unsigned)grid, KNT, smem, stream>>>(
        reinterpret_cast<const __nv_bfloat16 *>(base), norms, n, reinterpret_cast<const __nv_bfloat16 *>(queries),
        nq, self0, k, ids, dists, err);
    return cudaGetLastError();
}

}  // namespace

int64_t knn_norms_rows(int64_t n) { return (n + KBN - 1) / KBN * KBN; }

cudaError_t launch_knn_bf16(const void *base, int64_t n, int d, const void *queries, int64_t nq, int64_t self0,
                            int metric, int k, int32_t *ids, float *dists, float *norms, int *err,
                            cudaStream_t stream) {
    const bool l2 = metric == ANN_METRIC_L2;
    if (l2) {
        const int64_t np = knn_norms_rows(n);
        bf16_row_norms<<<(unsigned)((np + 255) / 256), 256, 0, stream>>>(
            reinterpret_cast<const __nv_bfloat16 *>(base), n, np, d, norms);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
#define ANN_KNN_CASE(KS)                                                                                   \
    case KS:                                                                                               \
        return l2 ? launch_knn_t<KS, true>(base, norms, n, queries, nq, self0, k, ids, dists, err, stream) \
                  : launch_knn_t<KS, false>(base, norms, n, queries, nq, self0, k, ids, dists, err, stream);
    switch (d / 16) {
        ANN_KNN_CASE(2)
        ANN_KNN_CASE(4)
        ANN_KNN_CASE(6)
        ANN_KNN_CASE(8)
        default: return cudaErrorInvalidValue;
    }
#undef ANN_KNN_CASE
}

}  // namespace ann
