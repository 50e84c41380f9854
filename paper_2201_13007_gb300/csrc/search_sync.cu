// search_sync.cu -- storage-type dispatch of the one-CTA sync search (the
// kernel itself is in search_sync.cuh, instantiated per storage type in
// search_sync_<storage>.cu so the types compile in parallel).
#include "ann_internal.cuh"

namespace ann {

template <int STORE>
cudaError_t launch_sync_store(const SearchArgs &a, int threads, int smem, int grid, cudaStream_t s);
template <int STORE>
cudaError_t occupancy_sync_store(int metric, int threads, int smem, int *bps);

cudaError_t launch_sync_search(const SearchArgs &a, int storage, int threads, int smem, int grid,
                               cudaStream_t s) {
    switch (storage) {
        case ANN_STORE_F32: return launch_sync_store<ANN_STORE_F32>(a, threads, smem, grid, s);
        case ANN_STORE_BF16: return launch_sync_store<ANN_STORE_BF16>(a, threads, smem, grid, s);
        case ANN_STORE_F16: return launch_sync_store<ANN_STORE_F16>(a, threads, smem, grid, s);
        case ANN_STORE_E4M3: return launch_sync_store<ANN_STORE_E4M3>(a, threads, smem, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t sync_search_occupancy(int storage, int metric, int threads, int smem, int *bps) {
    switch (storage) {
        case ANN_STORE_F32: return occupancy_sync_store<ANN_STORE_F32>(metric, threads, smem, bps);
        case ANN_STORE_BF16: return occupancy_sync_store<ANN_STORE_BF16>(metric, threads, smem, bps);
        case ANN_STORE_F16: return occupancy_sync_store<ANN_STORE_F16>(metric, threads, smem, bps);
        case ANN_STORE_E4M3: return occupancy_sync_store<ANN_STORE_E4M3>(metric, threads, smem, bps);
    }
    return cudaErrorInvalidValue;
}

}  // namespace ann
