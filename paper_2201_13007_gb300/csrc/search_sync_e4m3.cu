// search_sync_e4m3.cu -- the one-CTA sync search kernels for E4M3 storage (see search_sync.cuh).
#include "search_sync.cuh"

namespace ann {

template cudaError_t launch_sync_store<ANN_STORE_E4M3>(const SearchArgs &, int, int, int, cudaStream_t);
template cudaError_t occupancy_sync_store<ANN_STORE_E4M3>(int, int, int, int *);

}  // namespace ann
