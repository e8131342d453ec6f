// Host-side view of the SINR kernels (launchers, argument block, smem plans).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace ts {

// Everything a SINR kernel reads, as raw device pointers (float2 = complex).
struct SinrArgs {
  int J, m, n, p, P, K, L;
  int coef_mode;                    // 0 dense, 1 paths
  bool identity_C;                  // dense-channel comparator: C = I (p = P), G = X
  const float2* G;                  // [J*J][p][m][n]
  const float2* C;                  // [J*J][P][p]
  const float2* coef;               // dense: [J*J][K][P]; paths: alpha [J*J][P]
  const unsigned long long* turns;  // paths: [J*J][P] df*tau in 2^-64 turns
  float2* V;                        // svd: precoders [J][K][n][L] (workspace)
  uint8_t* pflag;                   // svd: precoder flags [J][K] (workspace)
  float2* Eserv;                    // wideband: serving effective channels [J][K][m][L] (workspace)
  float2* Hserv;                    // svd: serving compressed channels [J][K][m][n] (workspace)
  float2* Rpart;                    // partial covariances [J][J-1][K][m][m] (workspace)
  const float2* F;                  // mmse: G_ik x_2 Pt_k^T, [J*J][p][m][L] (workspace)
  const float* sigma2;              // [J]
  float* sinr;                      // [J][K][L]
  uint8_t* flags;                   // [J][K] or nullptr
};

// Launchers; each picks the template instance for (m, L) and returns the
// launch status.  `smem_*` report the dynamic shared memory of a launch.
cudaError_t launch_turns(const float* tau, float df, int count, unsigned long long* turns,
                         cudaStream_t s);
cudaError_t launch_coefficients(const float2* alpha, const float* tau, float df, int nch, int K,
                                int P, float2* c, cudaStream_t s);
cudaError_t launch_project_precoder(const float2* B, const float2* Pfull, int J, int N, int n,
                                    int L, float2* Pt, cudaStream_t s);
cudaError_t launch_mmse_fold(const float2* G, const float2* Pt, int J, int m, int n, int p,
                             int L, float2* F, cudaStream_t s);
cudaError_t launch_sinr_serving(const SinrArgs& a, cudaStream_t s);
cudaError_t launch_svd_precoder(const SinrArgs& a, cudaStream_t s);
cudaError_t launch_sinr_links(const SinrArgs& a, bool svd, cudaStream_t s);
cudaError_t launch_sinr_finalize(const SinrArgs& a, bool svd, cudaStream_t s);

// Store a CUDA error for ts_last_cuda_error() and return TS_ERR_CUDA.
int record_cuda_error(cudaError_t e);

// Largest m and L the kernels support.
constexpr int kMaxRankM = 16;

}  // namespace ts
