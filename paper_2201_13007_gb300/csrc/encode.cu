// encode.cu -- index-build kernels: FP32 rows -> stored rows (FP32, BF16,
// FP16, or FP8 E4M3 with a per-vector scale max|x|/448), zero padded to
// d_pad elements; a range check of the adjacency ids; in-degrees and the
// neighbour-group copies of ann_index_group_neighbors.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "ann_internal.cuh"

namespace ann {

// One warp per row.
template <int STORE>
__global__ void encode_rows(const float *__restrict__ src, int64_t n, int32_t d, void *__restrict__ dst,
                            int32_t d_pad, float *__restrict__ scales) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (row >= n) return;
    const float *x = src + (size_t)row * d;
    if (STORE == ANN_STORE_F32) {
        float *y = reinterpret_cast<float *>(dst) + (size_t)row * d_pad;
        for (int i = lane; i < d_pad; i += 32) y[i] = i < d ? x[i] : 0.f;
    } else if (STORE == ANN_STORE_BF16) {
        __nv_bfloat16 *y = reinterpret_cast<__nv_bfloat16 *>(dst) + (size_t)row * d_pad;
        for (int i = lane; i < d_pad; i += 32) y[i] = __float2bfloat16_rn(i < d ? x[i] : 0.f);
    } else if (STORE == ANN_STORE_F16) {
        __half *y = reinterpret_cast<__half *>(dst) + (size_t)row * d_pad;
        for (int i = lane; i < d_pad; i += 32) y[i] = __float2half_rn(i < d ? x[i] : 0.f);
    } else {
        float mx = 0.f;
        for (int i = lane; i < d; i += 32) mx = fmaxf(mx, fabsf(x[i]));
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
        const float s = mx > 0.f ? __fdiv_rn(mx, 448.0f) : 1.0f;
        if (lane == 0) scales[row] = s;
        __nv_fp8_storage_t *y = reinterpret_cast<__nv_fp8_storage_t *>(dst) + (size_t)row * d_pad;
        for (int i = lane; i < d_pad; i += 32) {
            const float v = i < d ? __fdiv_rn(x[i], s) : 0.f;
            y[i] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
        }
    }
}

cudaError_t launch_encode(const float *src, int64_t n, int32_t d, int storage, void *dst, int32_t d_pad,
                          float *scales, cudaStream_t stream) {
    const int threads = 256;
    const int64_t blocks = (n + 7) / 8;
    switch (storage) {
        case ANN_STORE_F32: encode_rows<ANN_STORE_F32><<<blocks, threads, 0, stream>>>(src, n, d, dst, d_pad, scales); break;
        case ANN_STORE_BF16: encode_rows<ANN_STORE_BF16><<<blocks, threads, 0, stream>>>(src, n, d, dst, d_pad, scales); break;
        case ANN_STORE_F16: encode_rows<ANN_STORE_F16><<<blocks, threads, 0, stream>>>(src, n, d, dst, d_pad, scales); break;
        case ANN_STORE_E4M3: encode_rows<ANN_STORE_E4M3><<<blocks, threads, 0, stream>>>(src, n, d, dst, d_pad, scales); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

__global__ void count_bad_adj(const int32_t *__restrict__ adj, int64_t count, int64_t n,
                              unsigned long long *bad) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = adj[i];
        local += (v < -1 || (int64_t)v >= n) ? 1ull : 0ull;
    }
    if (local) atomicAdd(bad, local);
}

cudaError_t launch_count_bad_adj(const int32_t *adj, int64_t count, int64_t n, unsigned long long *bad,
                                 cudaStream_t stream) {
    count_bad_adj<<<1024, 256, 0, stream>>>(adj, count, n, bad);
    return cudaGetLastError();
}

// In-degree of every vertex: deg[u] += 1 for each edge v -> u.
__global__ void count_in_degree(const int32_t *__restrict__ adj, int64_t count, int32_t *__restrict__ deg) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = adj[i];
        if (u >= 0) atomicAdd(deg + u, 1);
    }
}

cudaError_t launch_count_in_degree(const int32_t *adj, int64_t count, int32_t *deg, cudaStream_t stream) {
    count_in_degree<<<1024, 256, 0, stream>>>(adj, count, deg);
    return cudaGetLastError();
}

// Neighbour groups: row n + s * R + r of rows[] becomes a copy of the row of
// the r-th neighbour of hot vertex hot[s] (zeros, scale 1, for a -1 slot).
// One warp per group row, 16-byte copies.
__global__ void fill_groups(unsigned char *__restrict__ rows, float *__restrict__ scales,
                            const int32_t *__restrict__ adj, const int32_t *__restrict__ hot, int64_t n_hot,
                            int32_t R, int64_t n, int32_t row_bytes) {
    const int lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    if (g >= n_hot * R) return;
    const int64_t s = g / R, r = g - s * R;
    const int32_t u = adj[(size_t)hot[s] * R + r];
    uint4 *dst = reinterpret_cast<uint4 *>(rows + (size_t)(n + g) * row_bytes);
    const uint4 *src = reinterpret_cast<const uint4 *>(rows + (size_t)(u >= 0 ? u : 0) * row_bytes);
    for (int c = lane; c < row_bytes / 16; c += 32) dst[c] = u >= 0 ? src[c] : make_uint4(0u, 0u, 0u, 0u);
    if (scales && lane == 0) scales[n + g] = u >= 0 ? scales[u] : 1.0f;
}

cudaError_t launch_fill_groups(unsigned char *rows, float *scales, const int32_t *adj, const int32_t *hot,
                               int64_t n_hot, int32_t R, int64_t n, int32_t row_bytes, cudaStream_t stream) {
    const int64_t warps = n_hot * R;
    if (warps == 0) return cudaSuccess;
    fill_groups<<<(unsigned)((warps + 7) / 8), 256, 0, stream>>>(rows, scales, adj, hot, n_hot, R, n, row_bytes);
    return cudaGetLastError();
}

}  // namespace ann
