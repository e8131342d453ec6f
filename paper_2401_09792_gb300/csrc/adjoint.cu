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
  float2 Lq[MG], Y[LT], Zr[LT];
  float as[LT], xs[LT];
  const bool ok = sinr_core<MG, LT>(R, Eself, Es, a, Lq, Y, as, xs, Zr);
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

constexpr int kPMax = 32;          // largest core rank p
constexpr int kAdjKChunk = 32;     // subcarriers staged per step

// dl/dG[ch][q][ac] = sum_kappa conj(w[ch][kappa][q]) dl/dH~[ch][kappa][ac]:
// CTA (128 threads) per (column tile of 128, link ch, subcarrier split s),
// thread per column ac with p accumulators; the w rows of each chunk of
// subcarriers staged in shared memory.  Partial sums of split s go to
// out[s][ch][q][ac] (out = dG when there is one split).
__global__ void __launch_bounds__(128) k_adj_dG(const SinrArgs A, const float2* W, const float2* gH,
                                                float2* out, int ksplit) {
  __shared__ float2 ws[kAdjKChunk * kPMax];
  const int m = A.m, n = A.n, p = A.p, K = A.K, mn = m * n;
  const int tid = threadIdx.x, ac = blockIdx.x * 128 + tid;
  const int ch = blockIdx.y, s = blockIdx.z;
  const int kper = (K + ksplit - 1) / ksplit;
  const int k0 = s * kper, k1 = min(K, k0 + kper);
  float2 acc[kPMax];
#pragma unroll
  for (int q = 0; q < kPMax; ++q) acc[q] = cz();
  for (int kc = k0; kc < k1; kc += kAdjKChunk) {
    const int nk = min(kAdjKChunk, k1 - kc);
    __syncthreads();
    for (int idx = tid; idx < nk * p; idx += 128) ws[idx] = W[((size_t)ch * K + kc) * p + idx];
    __syncthreads();
    if (ac < mn) {
      const float2* gh = gH + ((size_t)ch * K + kc) * mn + ac;
#pragma unroll 4
      for (int t = 0; t < nk; ++t) {
        const float2 h = gh[(size_t)t * mn];
#pragma unroll
        for (int q = 0; q < kPMax; ++q) {
          if (q >= p) break;
          cmacc(acc[q], h, ws[t * p + q]);
        }
      }
    }
  }
  if (ac < mn) {
    const size_t nch = (size_t)A.J * A.J;
#pragma unroll
    for (int q = 0; q < kPMax; ++q) {
      if (q >= p) break;
      out[((s * nch + ch) * p + q) * mn + ac] = acc[q];
    }
  }
}

// dl/dw[ch][kappa][q] = sum_ac conj(G[ch][q][ac]) dl/dH~(kappa)[ac]: CTA of
// eight warps per (link ch, tile of eight subcarriers), warp per subcarrier,
// lanes over ac; the core is staged in shared memory 128 columns at a time
// and each warp's p sums are reduced across its lanes by shuffles.
constexpr int kGwCols = 128;
__global__ void __launch_bounds__(256) k_adj_gw(const SinrArgs A, const float2* gH, float2* gw) {
  __shared__ float2 gs[kPMax * kGwCols];
  const int m = A.m, n = A.n, p = A.p, K = A.K, mn = m * n;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int ch = blockIdx.y;
  const int kap = blockIdx.x * 8 + warp;
  const float2* Gc = A.G + (size_t)ch * p * mn;
  const float2* gh = gH + ((size_t)ch * K + (kap < K ? kap : 0)) * mn;
  float2 acc[kPMax];
#pragma unroll
  for (int q = 0; q < kPMax; ++q) acc[q] = cz();
  for (int c0 = 0; c0 < mn; c0 += kGwCols) {
    const int nc = min(kGwCols, mn - c0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < p * kGwCols; idx += 256) {
      const int q = idx / kGwCols, c = idx - q * kGwCols;
      gs[idx] = c < nc ? Gc[(size_t)q * mn + c0 + c] : cz();
    }
    __syncthreads();
    for (int c = lane; c < nc; c += 32) {
      const float2 h = gh[c0 + c];
#pragma unroll
      for (int q = 0; q < kPMax; ++q) {
        if (q >= p) break;
        cmacc(acc[q], h, gs[q * kGwCols + c]);
      }
    }
  }
  float2 mine = cz();
#pragma unroll
  for (int q = 0; q < kPMax; ++q) {
    if (q >= p) break;
    float2 v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(FULL, v.x, o);
      v.y += __shfl_xor_sync(FULL, v.y, o);
    }
    if (lane == q) mine = v;
  }
  if (kap < K && lane < p) gw[((size_t)ch * K + kap) * p + lane] = mine;
}

// dl/dC[ch][P][q] = sum_kappa c_P(kappa) dl/dw[ch][kappa][q]: CTA (256
// threads) per (tile of 32 paths, link ch, subcarrier split s); thread
// (path row, q group) with the q = qg, qg + 8, ... sums; the coefficients
// and dl/dw rows of each chunk of subcarriers staged in shared memory.
__global__ void __launch_bounds__(256) k_adj_dC(const SinrArgs A, const float2* gw, float2* out,
                                                int ksplit) {
  __shared__ float2 cs[kAdjKChunk * 32];
  __shared__ float2 gs[kAdjKChunk * kPMax];
  const int p = A.p, P = A.P, K = A.K;
  const int tid = threadIdx.x, pr = tid / 8, qg = tid % 8;
  const int P0 = blockIdx.x * 32, ch = blockIdx.y, s = blockIdx.z;
  const int kper = (K + ksplit - 1) / ksplit;
  const int k0 = s * kper, k1 = min(K, k0 + kper);
  float2 acc[kPMax / 8];
#pragma unroll
  for (int u = 0; u < kPMax / 8; ++u) acc[u] = cz();
  for (int kc = k0; kc < k1; kc += kAdjKChunk) {
    const int nk = min(kAdjKChunk, k1 - kc);
    __syncthreads();
    for (int idx = tid; idx < nk * 32; idx += 256) {
      const int t = idx / 32, r = idx % 32;
      cs[idx] = P0 + r < P ? coef_at(A, ch, kc + t, P0 + r) : cz();
    }
    for (int idx = tid; idx < nk * p; idx += 256) gs[idx] = gw[((size_t)ch * K + kc) * p + idx];
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
      const float2 c = cs[t * 32 + pr];
#pragma unroll
      for (int u = 0; u < kPMax / 8; ++u) {
        const int q = qg + 8 * u;
        if (q < p) cmac(acc[u], c, gs[t * p + q]);
      }
    }
  }
  if (P0 + pr < P) {
    const size_t nch = (size_t)A.J * A.J;
#pragma unroll
    for (int u = 0; u < kPMax / 8; ++u) {
      const int q = qg + 8 * u;
      if (q < p) out[((s * nch + ch) * P + P0 + pr) * p + q] = acc[u];
    }
  }
}

// out[i] = sum_s part[s][i], s in order
__global__ void k_adj_sum(const float2* part, int splits, size_t count, float2* out) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < count;
       idx += (size_t)gridDim.x * blockDim.x) {
    float2 acc = part[idx];
    for (int s = 1; s < splits; ++s) acc = cadd(acc, part[(size_t)s * count + idx]);
    out[idx] = acc;
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
  const AdjointSplit sp = adjoint_split(A.J, A.m, A.n, A.p, A.P, A.K);
  const size_t ng = nch * A.p * A.m * A.n, nc = nch * A.P * A.p;
  k_adj_dG<<<dim3((A.m * A.n + 127) / 128, (unsigned)nch, sp.kg), 128, 0, s>>>(
      A, w.W, w.gH, sp.kg > 1 ? w.part : w.dG, sp.kg);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (sp.kg > 1) {
    k_adj_sum<<<blocks_for(ng), 256, 0, s>>>(w.part, sp.kg, ng, w.dG);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_adj_gw<<<dim3((A.K + 7) / 8, (unsigned)nch), 256, 0, s>>>(A, w.gH, w.gw);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_adj_dC<<<dim3((A.P + 31) / 32, (unsigned)nch, sp.kc), 256, 0, s>>>(
      A, w.gw, sp.kc > 1 ? w.part : w.dC, sp.kc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (sp.kc > 1) {
    k_adj_sum<<<blocks_for(nc), 256, 0, s>>>(w.part, sp.kc, nc, w.dC);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_project_precoder_adjoint(const float2* Pfull, const float2* dPt, int J, int N,
                                            int n, int L, float2* dB, cudaStream_t s) {
  const int total = J * N * n;
  if (total == 0) return cudaSuccess;
  detail::k_project_precoder_adjoint<<<detail::blocks_for(total), 256, 0, s>>>(Pfull, dPt, J, N, n, L, dB);
  return cudaGetLastError();
}

}  // namespace ts
