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
  const float2* coef;               // dense: [J*J][Kc][P]; paths: alpha [J*J][P]
  int kap_off;                      // subcarrier index of local subcarrier 0 (a range call)
  int Kc;                           // subcarriers of the dense coefficient array (its stride)
  const unsigned long long* turns;  // paths: [J*J][P] df*tau in 2^-64 turns
  float2* V;                        // svd: precoders [J][K][n][L] (workspace)
  uint8_t* pflag;                   // svd: precoder flags [J][K] (workspace)
  float2* Eserv;                    // wideband: serving effective channels [J][K][m][L] (workspace)
  float2* Hserv;                    // svd with large cores: serving compressed channels
                                    // [J][K][m][n] (workspace), or all links
                                    // [J*J][K][m][n] (adjoint)
  int serv_stride;                  // serving link k at Hserv[(k * serv_stride) * K + kappa]
  int fuse_serve;                   // svd precoder forms H~_kk itself (Hserv unused)
  float2* Wserv;                    // wide cores: serving links' projections c* C,
                                    // [J][K][p] (workspace), or nullptr
  float2* Ueig;                     // svd, two-phase precoder: Gram eigenvectors [J][K][MG][MG]
                                    // (row a of U in row a) and
  float* lam_eig;                   //   their eigenvalues [J][K][MG] (unit-trace Gram), and
  uint8_t* conv_eig;                //   the Jacobi's convergence [J][K] (workspace)
  float2* Uout;                     // adjoint: left singular vectors [J][K][m][m] (or nullptr)
  float* Sout;                      // adjoint: singular values [J][K][m]
  float2* Vmout;                    // adjoint: right singular vectors [J][K][n][m]
  float2* Eint;                     // interfering effective channels E_ik, k != i,
                                    // [J][J-1][K][m][L] (workspace)
  const float2* F;                  // mmse: G_ik x_2 Pt_k^T, [J*J][p][m][L] (workspace)
  const float* sigma2;              // [J]
  float* sinr;                      // [J][K][L]
  uint8_t* flags;                   // [J][K] or nullptr
  int* rlist;                       // units (i K + kappa) to refine (workspace) or nullptr;
                                    // in the precoder phase, units (k K + kappa) whose
                                    // precoder is recomputed in FP64
  int* rcount;                      // length of rlist (workspace, zeroed before finalize)
  float refine_sens;                // refine units whose SINR sensitivity to R exceeds this
  int list_close;                   // svd precoders: list units with a close pair (below)
  float2* Uclose;                   // the listed units' left singular vectors of ranks
                                    // 0 .. min(L + 1, m) - 1, [J*K][min(L+1,m)][m] (workspace)
  int* close_mask;                  // and their close pairs, bit r for (r, r + 1) [J*K]
  // launch-shape choices (0: the default heuristics; set by the autotuner)
  int link_variant;                 // svd links: 1 blocked two-row kernel, 2 one-row kernel
  int precoder_split;               // precoder tile: subcarriers per CTA divided by 2^split
};

// Host-side hooks of the batch planner (api.cu): launch-shape choices applied
// to the SINR calls that follow on this host thread, and a switch that makes
// those calls ignore the ts_set_timing_events pair (while capturing a graph).
struct Tuning {
  int link_variant;
  int precoder_split;
};
void set_tuning(Tuning t);
void suspend_timing(bool suspended);

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
cudaError_t launch_svd_precoder(const SinrArgs& a, cudaStream_t s);
cudaError_t launch_sinr_links(const SinrArgs& a, bool svd, cudaStream_t s);
cudaError_t launch_sinr_finalize(const SinrArgs& a, bool svd, cudaStream_t s);
// FP64-residual refinement of the units the finalize kernel listed (refine.cu)
cudaError_t launch_sinr_refine(const SinrArgs& a, bool svd, cudaStream_t s);

// Close pairs of the SVD precoders.  Two adjacent eigenvalues lambda_r,
// lambda_r+1 of the Gram H~ H~* (r < L, the first discarded one included)
// less than kPolishWindow lambda_1 apart get one more rotation from their
// rows of W = U* H~; less than kPrecoderCloseGap lambda_1 apart, the unit is
// listed (when SinrArgs::list_close is set, m <= 16) with its vectors in
// Uclose, and its precoder refined from H~ formed in double-float
// (precoder_refine.cu).
// Pairs whose smaller eigenvalue is below kPrecoderWeak lambda_1 are not
// refined (their vectors' absolute FP32 error, not the pair's mixing, is
// what limits such streams).
constexpr float kPolishWindow = 0.15f;
constexpr float kPrecoderCloseGap = 5e-3f;
constexpr float kPrecoderWeak = 1e-2f;
cudaError_t launch_precoder_refine(const SinrArgs& a, cudaStream_t s);

// Buffers of the adjoint pipeline (adjoint.cu); Pt == nullptr selects SVD
// precoders (read from SinrArgs::Vmout/Uout/Sout).
struct AdjointWork {
  const float2* Pt;        // wideband: projected precoders [J][n][L]
  const float* dsinr;      // [J][K][L]
  float* sinr;             // forward SINR [J][K][L] (optional)
  float2* W;               // w = c* C   [J*J][K][p]
  float2* E;               // E_ik       [J*J][K][m][L]
  float2* gE;              // dl/dE_ik   [J*J][K][m][L]
  float2* gH;              // dl/dH~_ik  [J*J][K][m][n]
  float2* gV;              // dl/dV_k    [J][K][n][L]
  float2* gw;              // dl/dw      [J*J][K][p]
  float2* dG;              // [J*J][p][m][n]
  float2* dC;              // [J*J][P][p]
  float2* dPt;             // [J][n][L] (wideband)
  float2* part;            // split-K partial sums of dG and dC (adjoint_part_elems)
};
// Split of the subcarrier sums of dl/dG and dl/dC over CTAs, so that small
// systems still fill the GPU (partial sums are added in a fixed order).
struct AdjointSplit {
  int kg, kc;              // subcarrier splits of the dl/dG and dl/dC sums
};
inline AdjointSplit adjoint_split(int J, int m, int n, int p, int P, int K) {
  const long nch = (long)J * J;
  const long g_tiles = nch * ((m * n + 127) / 128), c_tiles = nch * ((P + 31) / 32);
  auto pick = [&](long tiles) {
    long s = (608 + tiles - 1) / tiles;             // at least four CTAs per SM
    const long smax = (K + 63) / 64;                // at least 64 subcarriers per CTA
    if (s > smax) s = smax;
    if (s > 16) s = 16;
    return (int)(s < 1 ? 1 : s);
  };
  return AdjointSplit{pick(g_tiles), pick(c_tiles)};
}
inline size_t adjoint_part_elems(int J, int m, int n, int p, int P, int K) {
  const AdjointSplit sp = adjoint_split(J, m, n, p, P, K);
  const size_t nch = (size_t)J * J;
  const size_t g = sp.kg > 1 ? (size_t)sp.kg * nch * p * m * n : 0;
  const size_t c = sp.kc > 1 ? (size_t)sp.kc * nch * P * p : 0;
  return g > c ? g : c;
}
cudaError_t launch_sinr_rebuild(const SinrArgs& a, cudaStream_t s);
cudaError_t launch_sinr_serving(const SinrArgs& a, cudaStream_t s);
// Tensor-core interfering-link pass (reduced-precision modes, sinr_tc.cu):
// shape support, bytes of the operands (the rewritten core of every link,
// the projections of the interfering links' subcarrier tiles, the tiled
// precoder rows, and in TF32X3 the projections of the serving links'
// tiles), their preparation into `prep` once per call (launch_core_prep:
// operands then precoder rows; or launch_tc_operands before the precoders,
// with `serving` for launch_serving_tc, and launch_tc_vtiles after them),
// the link kernel, and the TF32X3 serving pass writing H~_kk to Hserv.
bool tc_supported(int m, int L, int p);
size_t tc_prep_bytes(int J, int m, int L, int n, int p, int K, int prec);
cudaError_t launch_core_prep(const SinrArgs& a, int prec, void* prep, cudaStream_t s);
cudaError_t launch_tc_operands(const SinrArgs& a, int prec, bool serving, void* prep, cudaStream_t s);
cudaError_t launch_tc_vtiles(const SinrArgs& a, int prec, void* prep, cudaStream_t s);
cudaError_t launch_sinr_links_tc(const SinrArgs& a, int prec, const void* prep, cudaStream_t s);
cudaError_t launch_serving_tc(const SinrArgs& a, const void* prep, cudaStream_t s);
// Widest serving channel (columns n) the register precoder stages whole.
constexpr int kMaxNRegisterPrecoder = 512;
// The SVD precoder forms H~_kk itself (re-reading the core G_kk once per
// subcarrier tile from L2) when the core is at most 64 KB; larger cores (the
// dense-channel comparator) go through a separate serving-link pass.
inline bool precoder_fuses_serve(int m, int n, int p) {
  return (long long)m * n * p <= 8192 && n <= kMaxNRegisterPrecoder;
}
// SVD precoders of units whose serving channels (m <= 16 rows, n columns)
// do not fit the register precoder's shared-memory staging: the
// shared-memory precoder of the large-m path, one CTA per (BS, subcarrier),
// reading H~_kk from the serving pass's workspace (sinr_large.cu).
cudaError_t launch_precoder_staged(const SinrArgs& a, cudaStream_t s);
// Cores the narrow link kernels cannot stage (C_ik and a full core column
// chunk in shared memory): the SVD path runs the wide-core kernel, which
// streams the core in slabs and reads C_ik from L2.
__host__ __device__ inline bool wide_core(int P, int p) { return p > 32 || (long long)P * p > 8192; }
// Largest rank p of the wide-core kernel (w [T][p] in shared memory).
constexpr int kMaxRankPWide = 256;
cudaError_t launch_adjoint(const SinrArgs& a, const AdjointWork& w, cudaStream_t s);
cudaError_t launch_project_precoder_adjoint(const float2* Pfull, const float2* dPt, int J, int N,
                                            int n, int L, float2* dB, cudaStream_t s);

// Groupwise Tucker fit (fit.cu).
struct FitDims {
  int J, M, N, P, m, n, p;
  int model;   // TS_MODEL_GROUPWISE, _SHARED or _INDIVIDUAL: which links share A and B
  int iters;   // block subspace iterations per warm eigensolve (three times as many cold)
};
// number of A (B) factors of a model
__host__ __device__ inline int fit_groups(int J, int model) { return model == 1 ? 1 : model == 2 ? J * J : J; }
size_t fit_workspace_bytes(const FitDims& f);
// X^ = G x_1 A x_2 B x_3 C of every link with the model's factors (fit.cu)
size_t reconstruct_workspace_bytes(const FitDims& f);
cudaError_t launch_reconstruct(const FitDims& f, const float2* A, const float2* B, const float2* C,
                               const float2* G, float2* Xhat, void* ws, cudaStream_t s);
cudaError_t launch_fit(const FitDims& f, const float2* X, int S, int init, float2* A, float2* B,
                       float2* C, float2* G, double* g_hist, void* ws, cudaStream_t s);

// Store a CUDA error for ts_last_cuda_error() and return TS_ERR_CUDA.
int record_cuda_error(cudaError_t e);

// Largest m and L the kernels support.
constexpr int kMaxRankM = 16;

}  // namespace ts
