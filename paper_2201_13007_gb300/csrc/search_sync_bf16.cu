// search_sync_bf16.cu -- the one-CTA sync search kernels for BF16 storage (see search_sync.cuh).
#include "search_sync.cuh"

namespace ann {

template cudaError_t launch_sync_store<ANN_STORE_BF16>(const SearchArgs &, int, int, int, cudaStream_t);
template cudaError_t occupancy_sync_store<ANN_STORE_BF16>(int, int, int, int *);

}  // namespace ann
