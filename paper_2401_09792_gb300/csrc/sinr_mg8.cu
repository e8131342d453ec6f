// Template instances of the SINR kernels for groups of 8 lanes (m <= 8).
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
template cudaError_t run_precoder<8, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<8, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<8, 2>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<8, 2>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<8, 2>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_precoder<8, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<8, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<8, 4>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<8, 4>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<8, 4>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_precoder<8, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_serving<8, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_rebuild<8, 8>(const SinrArgs&, cudaStream_t);
template cudaError_t run_links<8, 8>(const SinrArgs&, bool, cudaStream_t);
template cudaError_t run_finalize<8, 8>(const SinrArgs&, bool, cudaStream_t);
}  // namespace detail
}  // namespace ts
