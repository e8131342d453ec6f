// Adjoint (vector-Jacobian product) of the compressed SINR: given dl/dSINR,
// the gradients of l with respect to the cores G, the mode-3 factors C and
// (wideband precoder) the projected precoders P~.  The paper has no adjoint;
// this differentiates its compressed SINR (eq. 15, 23-28).
//
// Per unit (UE i, subcarrier kappa), with D = E_ii* Q~^{-1} E_ii and
// SINR_r = D_rr / (1 - D_rr) (eq. 5 with W~ = Q~^{-1} E_ii):
//   gamma_r = dl/dSINR_r (1 + SINR_r)^2,  Y = Q~^{-1} E_ii,  M = Y Gamma Y*,
//   dl/dE_ik = -2 M E_ik (k != i),  dl/dE_ii = 2 Y Gamma - 2 M E_ii.
// Then E_ik = H~_ik V_k gives dl/dH~_ik = dl/dE_ik V_k* and
// dl/dV_k = sum_i H~_ik* dl/dE_ik; for SVD precoders V_k = top-L right
// singular vectors of H~_kk, whose adjoint adds
//   U_L S_L (Cm V_m* + S_L^{-2} G* (I - V_m V_m*)) + U S Cm* V_L*
// to dl/dH~_kk (G = dl/dV_k, Cm_rs = (g_r* v_s) / (s_r^2 - s_s^2), s != r).
// Finally H~ = sum_q w_q G[q] with w = C^T conj(c) (eq. 15):
//   dl/dG[q] = sum_kappa conj(w_q) dl/dH~,  dl/dw_q = <G[q], dl/dH~>,
//   dl/dC[P][q] = sum_kappa c_P dl/dw_q.
// Gradients follow the convention dl/dRe + i dl/dIm.  The forward quantities
// are recomputed from (G, C, coefficients), not stored by the forward call.
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
namespace {

__device__ __forceinline__ float2 coef_at(const SinrArgs& A, int ch, int kap, int pp) {
  return A.coef_mode == 0 ? A.coef[((size_t)ch * A.K + kap) * A.P + pp]
                          : path_coef(A.coef[(size_t)ch * A.P + pp], A.turns[(size_t)ch * A.P + pp], kap);
}

// w[ch][kappa][q] = sum_P C[ch][P][q] conj(c_P(kappa))   (the row c* C of eq. 15)
__global__ void k_adj_w(const SinrArgs A, float2* W) {
  const size_t total = (size_t)A.J * A.J * A.K * A.p;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % A.p);
    const size_t r = idx / A.p;
    const int kap = (int)(r % A.K);
    const int ch = (int)(r / A.K);
    float2 acc = cz();
    for (int pp = 0; pp < A.P; ++pp)
      cmacc(acc, A.C[((size_t)ch * A.P + pp) * A.p + q], coef_at(A, ch, kap, pp));
    W[idx] = acc;
  }
}

// precoder column l of BS k at subcarrier kappa, row c
__device__ __forceinline__ float2 prec_at(const SinrArgs& A, const float2* Pt, int k, int kap, int c,
                                          int l) {
  return Pt != nullptr ? Pt[((size_t)k * A.n + c) * A.L + l]
                       : A.Vmout[(((size_t)k * A.K + kap) * A.n + c) * A.m + l];
}

// E[ch][kappa][a][l] = sum_c H~[ch][kappa][a][c] V_k(kappa)[c][l]   (eq. 24)
__global__ void k_adj_effective(const SinrArgs A, const float2* Pt, float2* E) {
  const int m = A.m, n = A.n, L = A.L, K = A.K, J = A.J;
  const size_t total = (size_t)J * J * K * m * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % L);
    size_t r = idx / L;
    const int a = (int)(r % m);
    r /= m;
    const int kap = (int)(r % K);
    const int ch = (int)(r / K);
    const int k = ch % J;
    const float2* h = A.Hserv + (((size_t)ch * K + kap) * m + a) * n;
    float2 acc = cz();
    for (int c = 0; c < n; ++c) cmac(acc, h[c], prec_at(A, Pt, k, kap, c, l));
    E[idx] = acc;
  }
}

// One group of MG lanes per (UE i, subcarrier): SINR, gamma, Y, M and
// dl/dE_ik for every link k of the UE.
template <int MG, int LT>
__global__ void __launch_bounds__(kThreads) k_adj_units(const SinrArgs A, const float2* E,
                                                        const float* dsinr, float2* gE,
                                                        float* sinr_out) {
  __shared__ __align__(16) float2 sm_es[kThreads * LT + kThreads];
  const int T = kThreads / MG;
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int i = blockIdx.y;
  const int kap = blockIdx.x * T + g;
  const int J = A.J, m = A.m, L = A.L, K = A.K;
  const int kc = kap < K ? kap : K - 1;     // tail groups recompute the last subcarrier
  float2* Es = sm_es + g * (MG * LT + 2);

  float2 R[MG], Eself[LT];
#pragma unroll
  for (int b = 0; b < MG; ++b) R[b] = cz();
#pragma unroll
  for (int l = 0; l < LT; ++l) Eself[l] = cz();
  if (a < m) {
    for (int k = 0; k < J; ++k) {
      const float2* Ek = E + (((size_t)(i * J + k) * K + kc) * m) * L;
      if (k == i) {
#pragma unroll
        for (int l = 0; l < LT; ++l) Eself[l] = (l < L) ? Ek[a * L + l] : cz();
        continue;
      }
#pragma unroll
      for (int b = 0; b < MG; ++b) {
        if (b >= m) continue;
#pragma unroll
        for (int l = 0; l < LT; ++l)
          if (l < L) cmacc(R[b], Ek[a * L + l], Ek[b * L + l]);
      }
    }
  }
  add_diag(R, a, a < m ? A.sigma2[i] : 1.f);
  float2 Lq[MG], Y[LT];
  float as[LT], xs[LT];
  const bool ok = sinr_core<MG, LT>(R, Eself, Es, a, Lq, Y, as, xs);
  trsv_rows_conjT<MG, MG, LT>(Lq, Y, a);       // Y = Q~^{-1} E_ii
  float gam[LT];
#pragma unroll
  for (int r = 0; r < LT; ++r) {
    const float sv = as[r] / xs[r];
    gam[r] = (r < L && ok) ? dsinr[((size_t)i * K + kc) * L + r] * (1.f + sv) * (1.f + sv) : 0.f;
  }
  if (kap < K && a < L && sinr_out != nullptr)
    sinr_out[((size_t)i * K + kap) * L + a] = ok ? pickf(as, a) / pickf(xs, a) : __int_as_float(0x7fc00000);

  // M = Y Gamma Y*, row a
#pragma unroll
  for (int l = 0; l < LT; ++l) Es[a * LT + l] = Y[l];
  __syncwarp();
  float2 Mrow[MG];
#pragma unroll
  for (int b = 0; b < MG; ++b) {
    Mrow[b] = cz();
#pragma unroll
    for (int l = 0; l < LT; ++l) cmacc(Mrow[b], cscale(Y[l], gam[l]), Es[b * LT + l]);
  }
  __syncwarp();
  if (kap >= K || a >= m) return;
  for (int k = 0; k < J; ++k) {
    const size_t base = ((size_t)(i * J + k) * K + kap) * m;
    const float2* Ek = E + base * L;
    float2 out[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) out[l] = (k == i) ? cscale(Y[l], 2.f * gam[l]) : cz();
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      if (b >= m) continue;
      const float2 mab = cscale(Mrow[b], -2.f);
#pragma unroll
      for (int l = 0; l < LT; ++l)
        if (l < L) cmac(out[l], mab, Ek[b * L + l]);
    }
#pragma unroll
    for (int l = 0; l < LT; ++l)
      if (l < L) gE[(base + a) * L + l] = out[l];
  }
}

// dl/dH~[ch][kappa][a][c] = sum_l dl/dE[a][l] conj(V_k[c][l])
__global__ void k_adj_backH(const SinrArgs A, const float2* Pt, const float2* gE, float2* gH) {
  const int m = A.m, n = A.n, L = A.L, K = A.K, J = A.J;
  const size_t total = (size_t)J * J * K * m * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % n);
    size_t r = idx / n;
    const int a = (int)(r % m);
    r /= m;
    const int kap = (int)(r % K);
    const int ch = (int)(r / K);
    const int k = ch % J;
    const float2* ge = gE + (((size_t)ch * K + kap) * m + a) * L;
    float2 acc = cz();
    for (int l = 0; l < L; ++l) cmacc(acc, ge[l], prec_at(A, Pt, k, kap, c, l));
    gH[idx] = acc;
  }
}

// dl/dV_k(kappa)[c][l] = sum_i sum_a conj(H~_ik[a][c]) dl/dE_ik[a][l]
__global__ void k_adj_gV(const SinrArgs A, const float2* gE, float2* gV) {
  const int m = A.m, n = A.n, L = A.L, K = A.K, J = A.J;
  const size_t total = (size_t)J * K * n * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % L);
    size_t r = idx / L;
    const int c = (int)(r % n);
    r /= n;
    const int kap = (int)(r % K);
    const int k = (int)(r / K);
    float2 acc = cz();
    for (int i = 0; i < J; ++i) {
      const size_t base = ((size_t)(i * J + k) * K + kap) * m;
      for (int a = 0; a < m; ++a)
        cmacc(acc, gE[(base + a) * L + l], A.Hserv[(base + a) * n + c]);
    }
    gV[idx] = acc;
  }
}

// Adjoint of the SVD precoder (one block per (BS k, subcarrier)): adds to
// dl/dH~_kk the term through V_k = top-L right singular vectors of H~_kk.
constexpr int kSvdBackThreads = 64;
__global__ void __launch_bounds__(kSvdBackThreads) k_adj_svd_back(const SinrArgs A, const float2* gV,
                                                                 float2* gH) {
  extern __shared__ __align__(16) float2 sb[];
  const int m = A.m, n = A.n, L = A.L, K = A.K, J = A.J;
  const int kap = blockIdx.x, k = blockIdx.y;
  const size_t base = (size_t)k * K + kap;
  float2* Us = sb;                    // m x m
  float2* GHV = Us + m * m;           // L x m: G* V_m
  float2* Cm = GHV + L * m;           // L x m
  float* sg = reinterpret_cast<float*>(Cm + L * m);   // m
  const float2* Vm = A.Vmout + base * n * m;
  const float2* G = gV + base * n * L;
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) Us[t] = A.Uout[base * m * m + t];
  for (int t = threadIdx.x; t < m; t += blockDim.x) sg[t] = A.Sout[base * m + t];
  for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
    const int r = t / m, s = t - r * m;
    float2 acc = cz();
    for (int c = 0; c < n; ++c) cmacc(acc, Vm[(size_t)c * m + s], G[(size_t)c * L + r]);
    GHV[t] = acc;                     // sum_c conj(G[c][r]) V[c][s]
  }
  __syncthreads();
  for (int t = threadIdx.x; t < L * m; t += blockDim.x) {
    const int r = t / m, s = t - r * m;
    const float lr = sg[r] * sg[r], ls = sg[s] * sg[s];
    const float den = lr - ls;
    Cm[t] = (s != r && den != 0.f) ? cscale(GHV[t], 1.f / den) : cz();
  }
  __syncthreads();
  float2* out = gH + ((size_t)(k * J + k) * K + kap) * m * n;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    float2 A1[16], Bc[16];
    for (int r = 0; r < L; ++r) {
      float2 acc = cz(), proj = cz();
      for (int s = 0; s < m; ++s) {
        const float2 vcs = cconj(Vm[(size_t)c * m + s]);
        cmac(acc, Cm[r * m + s], vcs);
        cmac(proj, GHV[r * m + s], vcs);
      }
      const float lr = sg[r] * sg[r];
      float2 t = cadd(cconj(G[(size_t)c * L + r]), make_float2(-proj.x, -proj.y));
      A1[r] = lr > 0.f ? cadd(acc, cscale(t, 1.f / lr)) : acc;
    }
    for (int s = 0; s < m; ++s) {
      float2 acc = cz();
      for (int r = 0; r < L; ++r) cmac(acc, cconj(Cm[r * m + s]), cconj(Vm[(size_t)c * m + r]));
      Bc[s] = acc;
    }
    for (int a = 0; a < m; ++a) {
      float2 acc = cz();
      for (int r = 0; r < L; ++r) cmac(acc, cscale(Us[a * m + r], sg[r]), A1[r]);
      for (int s = 0; s < m; ++s) cmac(acc, cscale(Us[a * m + s], sg[s]), Bc[s]);
      out[(size_t)a * n + c] = cadd(out[(size_t)a * n + c], acc);
    }
  }
}

// dl/dP~_k[c][l] = sum_kappa dl/dV_k(kappa)[c][l]   (wideband precoder)
__global__ void k_adj_dPt(const SinrArgs A, const float2* gV, float2* dPt) {
  const int n = A.n, L = A.L, K = A.K, J = A.J;
  const int total = J * n * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int cl = idx % (n * L), k = idx / (n * L);
    float2 acc = cz();
    for (int kap = 0; kap < K; ++kap) acc = cadd(acc, gV[((size_t)k * K + kap) * n * L + cl]);
    dPt[idx] = acc;
  }
}

// dl/dG[ch][q][a][c] = sum_kappa conj(w_q(kappa)) dl/dH~(kappa)[a][c]
constexpr int kPMax = 32;
__global__ void k_adj_dG(const SinrArgs A, const float2* W, const float2* gH, float2* dG) {
  const int m = A.m, n = A.n, p = A.p, K = A.K, J = A.J;
  const size_t total = (size_t)J * J * m * n;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int ac = (int)(idx % ((size_t)m * n));
    const int ch = (int)(idx / ((size_t)m * n));
    float2 acc[kPMax];
#pragma unroll
    for (int q = 0; q < kPMax; ++q) acc[q] = cz();
    for (int kap = 0; kap < K; ++kap) {
      const float2 gh = gH[((size_t)ch * K + kap) * m * n + ac];
      const float2* wr = W + ((size_t)ch * K + kap) * p;
#pragma unroll
      for (int q = 0; q < kPMax; ++q)
        if (q < p) cmacc(acc[q], gh, wr[q]);
    }
#pragma unroll
    for (int q = 0; q < kPMax; ++q)
      if (q < p) dG[((size_t)ch * p + q) * m * n + ac] = acc[q];
  }
}

// dl/dw[ch][kappa][q] = sum_{a,c} conj(G[ch][q][a][c]) dl/dH~(kappa)[a][c]
__global__ void k_adj_gw(const SinrArgs A, const float2* gH, float2* gw) {
  const int m = A.m, n = A.n, p = A.p, K = A.K, J = A.J;
  const size_t total = (size_t)J * J * K * p;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % p);
    const size_t r = idx / p;
    const int kap = (int)(r % K);
    const int ch = (int)(r / K);
    const float2* gh = gH + ((size_t)ch * K + kap) * m * n;
    const float2* gq = A.G + ((size_t)ch * p + q) * m * n;
    float2 acc = cz();
    for (int ac = 0; ac < m * n; ++ac) cmacc(acc, gh[ac], gq[ac]);
    gw[idx] = acc;
  }
}

// dl/dC[ch][P][q] = sum_kappa c_P(kappa) dl/dw[ch][kappa][q]
__global__ void k_adj_dC(const SinrArgs A, const float2* gw, float2* dC) {
  const int p = A.p, P = A.P, K = A.K, J = A.J;
  const size_t total = (size_t)J * J * P * p;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(idx % p);
    const size_t r = idx / p;
    const int pp = (int)(r % P);
    const int ch = (int)(r / P);
    float2 acc = cz();
    for (int kap = 0; kap < K; ++kap) cmac(acc, coef_at(A, ch, kap, pp), gw[((size_t)ch * K + kap) * p + q]);
    dC[idx] = acc;
  }
}

// dB[k][N][b] = sum_l conj(Pfull[k][N][l]) dPt[k][b][l]   (adjoint of Pt = B^T P)
__global__ void k_project_precoder_adjoint(const float2* Pfull, const float2* dPt, int J, int N,
                                           int n, int L, float2* dB) {
  const int total = J * N * n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int b = idx % n, r = (idx / n) % N, k = idx / (n * N);
    float2 acc = cz();
    for (int l = 0; l < L; ++l)
      cmacc(acc, dPt[((size_t)k * n + b) * L + l], Pfull[((size_t)k * N + r) * L + l]);
    dB[idx] = acc;
  }
}

int blocks_for(size_t total, int threads = 256) {
  const size_t b = (total + threads - 1) / threads;
  return (int)(b < 152 * 32 ? (b == 0 ? 1 : b) : 152 * 32);
}

template <int MG, int LT>
cudaError_t run_units(const SinrArgs& A, const float2* E, const float* dsinr, float2* gE,
                      float* sinr_out, cudaStream_t s) {
  const int T = kThreads / MG;
  dim3 grid((A.K + T - 1) / T, A.J);
  k_adj_units<MG, LT><<<grid, kThreads, 0, s>>>(A, E, dsinr, gE, sinr_out);
  return cudaGetLastError();
}

}  // namespace

#define TS_DISPATCH_ADJ(FN, ...)                                                    \
  do {                                                                              \
    const int MG_ = A.m <= 2 ? 2 : A.m <= 4 ? 4 : A.m <= 8 ? 8 : 16;                \
    const int LT_ = A.L <= 2 ? 2 : A.L <= 4 ? 4 : A.L <= 8 ? 8 : 16;                \
    if (MG_ == 2) return FN<2, 2>(__VA_ARGS__);                                     \
    if (MG_ == 4) return LT_ <= 2 ? FN<4, 2>(__VA_ARGS__) : FN<4, 4>(__VA_ARGS__);  \
    if (MG_ == 8)                                                                   \
      return LT_ <= 2 ? FN<8, 2>(__VA_ARGS__)                                       \
                      : LT_ <= 4 ? FN<8, 4>(__VA_ARGS__) : FN<8, 8>(__VA_ARGS__);   \
    return LT_ <= 4 ? FN<16, 4>(__VA_ARGS__)                                        \
                    : LT_ <= 8 ? FN<16, 8>(__VA_ARGS__) : FN<16, 16>(__VA_ARGS__);  \
  } while (0)

cudaError_t adjoint_units(const SinrArgs& A, const float2* E, const float* dsinr, float2* gE,
                          float* sinr_out, cudaStream_t s) {
  TS_DISPATCH_ADJ(run_units, A, E, dsinr, gE, sinr_out, s);
}

}  // namespace detail

cudaError_t launch_adjoint(const SinrArgs& A, const AdjointWork& w, cudaStream_t s) {
  using namespace detail;
  const size_t nch = (size_t)A.J * A.J;
  cudaError_t e = cudaSuccess;
  k_adj_w<<<blocks_for(nch * A.K * A.p), 256, 0, s>>>(A, w.W);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_effective<<<blocks_for(nch * A.K * A.m * A.L), 256, 0, s>>>(A, w.Pt, w.E);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = adjoint_units(A, w.E, w.dsinr, w.gE, w.sinr, s)) != cudaSuccess) return e;
  k_adj_backH<<<blocks_for(nch * A.K * A.m * A.n), 256, 0, s>>>(A, w.Pt, w.gE, w.gH);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_gV<<<blocks_for((size_t)A.J * A.K * A.n * A.L), 256, 0, s>>>(A, w.gE, w.gV);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (w.Pt == nullptr) {
    const size_t smem = (size_t)(A.m * A.m + 2 * A.L * A.m) * sizeof(float2) + A.m * sizeof(float);
    k_adj_svd_back<<<dim3(A.K, A.J), kSvdBackThreads, smem, s>>>(A, w.gV, w.gH);
  } else {
    k_adj_dPt<<<blocks_for((size_t)A.J * A.n * A.L), 256, 0, s>>>(A, w.gV, w.dPt);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_dG<<<blocks_for(nch * A.m * A.n, 128), 128, 0, s>>>(A, w.W, w.gH, w.dG);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_gw<<<blocks_for(nch * A.K * A.p), 256, 0, s>>>(A, w.gH, w.gw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_dC<<<blocks_for(nch * A.P * A.p), 256, 0, s>>>(A, w.gw, w.dC);
  return cudaGetLastError();
}

cudaError_t launch_project_precoder_adjoint(const float2* Pfull, const float2* dPt, int J, int N,
                                            int n, int L, float2* dB, cudaStream_t s) {
  const int total = J * N * n;
  if (total == 0) return cudaSuccess;
  detail::k_project_precoder_adjoint<<<detail::blocks_for(total), 256, 0, s>>>(Pfull, dPt, J, N, n, L, dB);
  return cudaGetLastError();
}

}  // namespace ts
