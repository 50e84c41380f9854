// search_sync_f32.cu -- the one-CTA sync search kernels for F32 storage (see search_sync.cuh).
#include "search_sync.cuh"

namespace ann {

template cudaError_t launch_sync_store<ANN_STORE_F32>(const SearchArgs &, int, int, int, cudaStream_t);
template cudaError_t occupancy_sync_store<ANN_STORE_F32>(int, int, int, int *);

}  // namespace ann
