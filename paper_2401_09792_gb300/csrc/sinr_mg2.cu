// Template instances of the SINR kernels for groups of 2 lanes (m <= 2).
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
template cudaError_t run_precoder<2, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<2, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<2, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<2, 2>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<2, 2>(const SinrArgs&, bool, cudaStream_t);
}  // namespace detail
}  // namespace ts
