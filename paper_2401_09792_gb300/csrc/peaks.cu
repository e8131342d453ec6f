// Device throughput microbenchmarks: FP32 FMA, TF32 tensor-core MMA
// (tcgen05, M = 128, N = 256, K = 8 per instruction, TMEM accumulator) and
// FP64 FMA, each timed with CUDA events over a fixed amount of work sized to
// run for some milliseconds on every SM.  They give the measured ceilings
// the roofline fractions are compared with.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tuckersinr.h"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(float* out, int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 0.001f * (threadIdx.x + c);
  const float x = 0.9999f, y = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double* out, int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 0.001 * (threadIdx.x + c);
  const double x = 0.9999, y = 1e-7;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// One CTA per SM: A (128 x 8) and B (256 x 8) TF32 tiles of zeros in shared
// memory, `iters` MMAs accumulating into one TMEM tile, one commit, one
// bounded wait.
__global__ void __launch_bounds__(128) k_peak_tf32(int iters, int* status) {
  __shared__ __align__(1024) unsigned char tiles[(128 + 256) * 32];
  __shared__ uint64_t bar;
  __shared__ uint32_t slot;
  const int tid = threadIdx.x;
  for (int i = tid; i < (128 + 256) * 32 / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(tiles)[i] = 0u;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(&slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = slot;
  if (tid == 0) {
    // K-major, no swizzle, 32-byte rows: core matrices K-adjacent 128 B apart,
    // row groups 256 B apart
    auto desc = [](uint32_t addr) {
      uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
      d |= (uint64_t)(128 >> 4) << 16;
      d |= (uint64_t)(256 >> 4) << 32;
      d |= (uint64_t)1 << 46;
      return d;
    };
    const uint64_t ad = desc(smem_u32(tiles)), bd = desc(smem_u32(tiles + 128 * 32));
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
    for (int it = 0; it < iters; ++it) {
      const uint32_t acc = it > 0;
      asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                   "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                   "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&bar))
                 : "memory");
  }
  uint32_t done = 0;
  for (long it = 0; it < (1L << 26) && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(smem_u32(&bar)), "r"(0u) : "memory");
  if (!done && tid == 0) atomicExch(status, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

}  // namespace

extern "C" int ts_device_peaks(double* fp32_tflops, double* tf32_tflops, double* fp64_tflops,
                               void* stream) {
  if (fp32_tflops == nullptr || tf32_tflops == nullptr || fp64_tflops == nullptr) return TS_ERR_NULL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  void* scratch = nullptr;   // never written unless the sums hit the sentinel
  int* status = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&scratch, (size_t)sms * 8 * 256 * sizeof(double) + 256);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    status = reinterpret_cast<int*>(static_cast<char*>(scratch) + (size_t)sms * 8 * 256 * sizeof(double));
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
  }
  auto timed = [&](auto launch, double flops, double* out) {
    if (e != cudaSuccess) return;
    launch();                                    // warm-up
    e = cudaEventRecord(a, s);
    if (e == cudaSuccess) launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess) *out = flops / (ms * 1e-3) / 1e12;
  };
  const int blocks = sms * 8, threads = 256;
  const int fiters = 1 << 14, diters = 1 << 9, titers = 1 << 13;
  timed([&] { k_peak_ffma<<<blocks, threads, 0, s>>>(static_cast<float*>(scratch), fiters, 1.f); },
        2.0 * kChains * fiters * (double)blocks * threads, fp32_tflops);
  timed([&] { k_peak_dfma<<<blocks, threads, 0, s>>>(static_cast<double*>(scratch), diters, 1.0); },
        2.0 * kChains * diters * (double)blocks * threads, fp64_tflops);
  timed([&] { k_peak_tf32<<<sms, 128, 0, s>>>(titers, status); },
        2.0 * 128 * 256 * 8 * (double)titers * sms, tf32_tflops);
  int st_host = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&st_host, status, sizeof(int), cudaMemcpyDeviceToHost);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (scratch) cudaFree(scratch);
  if (e != cudaSuccess) return ts::record_cuda_error(e);
  return st_host == 0 ? TS_OK : TS_ERR_CUDA;
}
