// Template instances of the SINR kernels for groups of 4 lanes (m <= 4).
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
template cudaError_t run_precoder<4, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<4, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<4, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<4, 2>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<4, 2>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_precoder<4, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<4, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<4, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<4, 4>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<4, 4>(const SinrArgs&, bool, cudaStream_t);
}  // namespace detail
}  // namespace ts
