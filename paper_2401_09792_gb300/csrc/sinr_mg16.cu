// Template instances of the SINR kernels for groups of 16 lanes (m <= 16).
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
template cudaError_t run_precoder<16, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<16, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<16, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<16, 4>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<16, 4>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_precoder<16, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<16, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<16, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<16, 8>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<16, 8>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_precoder<16, 16>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<16, 16>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<16, 16>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<16, 16>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<16, 16>(const SinrArgs&, bool, cudaStream_t);
}  // namespace detail
}  // namespace ts
