// SINR kernels for the groupwise Tucker form (arXiv 2401.09792, Section 3.3).
//
// Work decomposition.  A unit is one (UE i, subcarrier kappa).  A group of MG
// consecutive lanes (MG = next power of two >= m) evaluates one unit, lane a
// owning row a of every m-row matrix: the compressed channel H~_ik(kappa)
// (eq. 15), the effective channel E_ik = H~_ik V_k (eq. 24), the covariance
// Q~_i (eq. 25) and its Cholesky factor.  A CTA holds T = 256 / MG (at most
// 64) consecutive subcarriers of one UE, so that every core G_ik and factor
// C_ik staged in shared memory serves T subcarriers.
//
//   k_svd_precoder       (BS k, subcarrier tile): H~_kk, Gram H~_kk H~_kk*,
//                        Jacobi eigensolve, V~_k = H~_kk* U_L Sigma_L^{-1}
//                        (eq. 7, eq. 23) -> workspace V[k][kappa][n][L]
//   k_sinr_accumulate    (UE i, subcarrier tile): for every BS k,
//                        w = c* C (eq. 15), E_ik = H~_ik V~_k (svd) or
//                        sum_q w_q F_ik[q] (wideband precoder), accumulate
//                        R_i = sum_{k != i} E E* + sigma^2 I; then the SINR
//                        of eq. (5) in a cancellation-free form (below).
//
// SINR form.  With e_r the columns of E_ii and Q~ = R + E_ii E_ii*,
// eq. (5) equals a_r / x_r where a_r = e_r* Q~^{-1} e_r = |L_Q^{-1} e_r|^2 and
// x_r = [(I + Z*Z)^{-1}]_rr = |column r of L_F^{-1}|^2, Z = L_R^{-1} E_ii,
// F = I + Z*Z = L_F L_F*.  Both are sums of squares, and a_r + x_r = 1.
#pragma once

#include "common.cuh"
#include "kernels.h"
#include "tuckersinr.h"

namespace ts {
namespace detail {

constexpr int kThreads = 256;
// dynamic shared memory a SINR launch may use (the per-CTA limit is 227 KB)
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ float2 path_coef(float2 alpha, unsigned long long turn, int kappa) {
  // c_p(kappa) = conj(alpha_p) exp(+j 2 pi kappa df tau_p); the phase is kept
  // modulo one turn in 64-bit fixed point, then mapped to half-turns in [-1, 1)
  const unsigned long long ph = turn * (unsigned long long)kappa;
  const float x = (float)(long long)ph * 0x1p-63f;
  float s, c;
  sincospif(x, &s, &c);
  return make_float2(fmaf(alpha.x, c, alpha.y * s), fmaf(alpha.x, s, -alpha.y * c));
}

// Stage the coefficient tile c[ch][kap0 .. kap0+T)[0 .. P) into cs[T][P]
// (zero beyond K) and project it: ws[t][q] = sum_P conj(c[t][P]) C[P][q]
// (the row vector c* C of eq. 15).  Ends with the block synchronised.
__device__ __forceinline__ void stage_projection(const SinrArgs& A, int ch, int kap0, int T,
                                                 float2* cs, float2* Cs, float2* ws, int wstride) {
  const int P = A.P, p = A.p, K = A.K;
  const int nth = blockDim.x, tid = threadIdx.x;
  for (int idx = tid; idx < T * P; idx += nth) {
    const int t = idx / P, pp = idx - t * P;
    const int kap = kap0 + t;
    float2 v = cz();
    if (kap < K) {
      if (A.coef_mode == 0)
        v = A.coef[((size_t)ch * K + kap) * P + pp];
      else
        v = path_coef(A.coef[(size_t)ch * P + pp], A.turns[(size_t)ch * P + pp], kap);
    }
    cs[idx] = v;
  }
  for (int idx = tid; idx < P * p; idx += nth) Cs[idx] = A.C[(size_t)ch * P * p + idx];
  __syncthreads();
  for (int idx = tid; idx < T * p; idx += nth) {
    const int t = idx / p, q = idx - t * p;
    float2 acc = cz();
    const float2* crow = cs + t * P;
    for (int pp = 0; pp < P; ++pp) cmacc(acc, Cs[pp * p + q], crow[pp]);
    ws[t * wstride + q] = acc;
  }
  __syncthreads();
}

// Stage G_ch[:, 0..m, c0 .. c0+NC) as Gs[q][a][cc] (row stride SG), zero
// padded for a >= m and columns >= n.
template <int MG, int NC>
__device__ __forceinline__ void stage_core_chunk(const SinrArgs& A, int ch, int c0, float2* Gs,
                                                 int SG) {
  const int p = A.p, m = A.m, n = A.n;
  const int nth = blockDim.x, tid = threadIdx.x;
  const float2* Gch = A.G + (size_t)ch * p * m * n;
  for (int idx = tid; idx < p * MG * NC; idx += nth) {
    const int cc = idx % NC;
    const int a = (idx / NC) % MG;
    const int q = idx / (NC * MG);
    const int c = c0 + cc;
    float2 v = cz();
    if (a < m && c < n) v = Gch[((size_t)q * m + a) * n + c];
    Gs[(q * MG + a) * SG + cc] = v;
  }
}

// H~ chunk of row a for one subcarrier: h[cc] = sum_q w_q G[q][a][c0 + cc].
template <int NC>
__device__ __forceinline__ void core_chunk(const float2* wrow, const float2* Gs, int SG, int MG,
                                           int a, int p, float2 (&h)[NC]) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) h[cc] = cz();
  for (int q = 0; q < p; ++q) {
    const float2 w = wrow[q];
    const float4* g4 = reinterpret_cast<const float4*>(Gs + (q * MG + a) * SG);
#pragma unroll
    for (int c2 = 0; c2 < NC / 2; ++c2) {
      const float4 g = g4[c2];
      cmac(h[2 * c2], w, make_float2(g.x, g.y));
      cmac(h[2 * c2 + 1], w, make_float2(g.z, g.w));
    }
  }
}

// ------------------------------------------------------------------ phase 1
// Shared memory plan of k_svd_precoder (float2 units).
struct PrecoderPlan {
  int T, NC, SG, SH, SS, wstride;
  int off_cs, off_Cs, off_ws, off_Gs, off_Hs, off_Ss, off_Us, off_rot, off_sel, total;
};

__host__ __device__ inline PrecoderPlan precoder_plan(int MG, int T, int NC, int P, int p, int n) {
  PrecoderPlan pl;
  pl.T = T;
  pl.NC = NC;
  pl.SG = NC + 2;
  pl.SH = n + 1;
  pl.SS = MG + 1;
  pl.wstride = p + 1;
  int o = 0;
  pl.off_cs = o; o += T * P;
  pl.off_Cs = o; o += P * p;
  pl.off_ws = o; o += T * pl.wstride;
  pl.off_Gs = o; o += p * MG * pl.SG;
  o = (o + 1) & ~1;
  pl.off_Hs = o; o += T * MG * pl.SH;
  pl.off_Ss = o; o += T * MG * pl.SS;
  pl.off_Us = o; o += T * MG * pl.SS;
  o = (o + 1) & ~1;
  pl.off_rot = o; o += T * MG;           // MG/2 float4 per group
  pl.off_sel = o; o += T * MG / 2 + 1;   // MG int per group
  pl.total = o;
  return pl;
}

template <int MG, int LT, int NC>
__global__ void __launch_bounds__(kThreads) k_svd_precoder(const SinrArgs A, const PrecoderPlan pl) {
  extern __shared__ __align__(16) float2 sm[];
  const int T = pl.T;
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int k = blockIdx.y;
  const int ch = k * A.J + k;
  const int kap0 = blockIdx.x * T;
  const int kap = kap0 + g;
  const int m = A.m, n = A.n, p = A.p, L = A.L, K = A.K;
  float2* cs = sm + pl.off_cs;
  float2* Cs = sm + pl.off_Cs;
  float2* ws = sm + pl.off_ws;
  float2* Gs = sm + pl.off_Gs;
  float2* Hs = sm + pl.off_Hs + g * MG * pl.SH;
  float2* Ss = sm + pl.off_Ss + g * MG * pl.SS;
  float2* Us = sm + pl.off_Us + g * MG * pl.SS;
  float4* rot = reinterpret_cast<float4*>(sm + pl.off_rot) + g * (MG / 2);
  int* sel = reinterpret_cast<int*>(sm + pl.off_sel) + g * MG;

  stage_projection(A, ch, kap0, T, cs, Cs, ws, pl.wstride);

  // compressed serving channel H~_kk(kappa), eq. (15), one row per lane
  for (int c0 = 0; c0 < n; c0 += NC) {
    if (c0 > 0) __syncthreads();
    stage_core_chunk<MG, NC>(A, ch, c0, Gs, pl.SG);
    __syncthreads();
    float2 h[NC];
    core_chunk<NC>(ws + g * pl.wstride, Gs, pl.SG, MG, a, p, h);
#pragma unroll
    for (int cc = 0; cc < NC; ++cc)
      if (c0 + cc < n) Hs[a * pl.SH + c0 + cc] = h[cc];
  }
  __syncwarp();

  // Gram S = H~ H~* (m x m, padded to MG with zero rows), U = I
  {
    float2 srow[MG];
#pragma unroll
    for (int b = 0; b < MG; ++b) srow[b] = cz();
    const float2* ha = Hs + a * pl.SH;
    for (int c = 0; c < n; ++c) {
      const float2 x = ha[c];
#pragma unroll
      for (int b = 0; b < MG; ++b) cmacc(srow[b], x, Hs[b * pl.SH + c]);
    }
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      Ss[a * pl.SS + b] = srow[b];
      Us[a * pl.SS + b] = make_float2(b == a ? 1.f : 0.f, 0.f);
    }
  }
  __syncwarp();

  // cyclic Jacobi with a round-robin ordering: MG/2 disjoint rotations per
  // step, MG-1 steps per sweep.  The rotation for pair (p, q) with
  // S_pq = |b| e^{i phi} is J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] (the
  // real symmetric Jacobi rotation of [[S_pp, |b|], [|b|, S_qq]] conjugated
  // by diag(1, e^{-i phi})); S <- J* S J, U <- U J.
  const int max_sweeps = MG <= 8 ? 12 : 16;
  bool converged = false;
  for (int sweep = 0;; ++sweep) {
    float off = 0.f, dia = 0.f;
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      const float v = cabs2(Ss[a * pl.SS + b]);
      if (b == a) dia += v; else off += v;
    }
    off = gsum<MG>(off);
    dia = gsum<MG>(dia);
    // FP32 stopping rule: off-diagonal energy below (8 u)^2 of the total, u = 2^-24
    converged = off <= 2.3e-13f * dia;
    // the decision is taken warp-wide: every group keeps sweeping until all
    // groups of the warp have converged (extra sweeps leave S unchanged)
    if (__all_sync(FULL, converged) || sweep == max_sweeps) break;
#pragma unroll 1
    for (int step = 0; step < MG - 1; ++step) {
      if (a < MG / 2) {
        int pp, qq;
        if (a == 0) { pp = step; qq = MG - 1; }
        else { pp = (step + a) % (MG - 1); qq = (step - a + MG - 1) % (MG - 1); }
        const float app = Ss[pp * pl.SS + pp].x, aqq = Ss[qq * pl.SS + qq].x;
        const float2 b = Ss[pp * pl.SS + qq];
        const float ab = sqrtf(cabs2(b));
        float c = 1.f, s = 0.f;
        float2 e = make_float2(1.f, 0.f);
        if (ab > 1e-30f && ab > 1e-9f * sqrtf(fabsf(app * aqq))) {
          const float tau = (aqq - app) / (2.f * ab);
          const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
          c = 1.f / sqrtf(fmaf(t, t, 1.f));
          s = t * c;
          e = cscale(b, 1.f / ab);
        }
        rot[a] = make_float4(c, s, e.x, e.y);
        sel[2 * a] = pp;
        sel[2 * a + 1] = qq;
      }
      __syncwarp();
      // rows: S <- J* S ; lane = column
#pragma unroll
      for (int j = 0; j < MG / 2; ++j) {
        const float4 r = rot[j];
        const int pp = sel[2 * j], qq = sel[2 * j + 1];
        const float2 e = make_float2(r.z, r.w);
        const float2 x = Ss[pp * pl.SS + a], y = Ss[qq * pl.SS + a];
        float2 nx = cscale(x, r.x), ny = cscale(y, r.x);
        cms(nx, cscale(e, r.y), y);            // c x - s e y
        cmac(ny, cscale(cconj(e), r.y), x);    // s conj(e) x + c y
        Ss[pp * pl.SS + a] = nx;
        Ss[qq * pl.SS + a] = ny;
      }
      __syncwarp();
      // columns: S <- S J and U <- U J ; lane = row
#pragma unroll
      for (int j = 0; j < MG / 2; ++j) {
        const float4 r = rot[j];
        const int pp = sel[2 * j], qq = sel[2 * j + 1];
        const float2 e = make_float2(r.z, r.w);
        {
          const float2 x = Ss[a * pl.SS + pp], y = Ss[a * pl.SS + qq];
          float2 nx = cscale(x, r.x), ny = cscale(y, r.x);
          cms(nx, cscale(cconj(e), r.y), y);   // c x - s conj(e) y
          cmac(ny, cscale(e, r.y), x);         // s e x + c y
          Ss[a * pl.SS + pp] = nx;
          Ss[a * pl.SS + qq] = ny;
        }
        {
          const float2 x = Us[a * pl.SS + pp], y = Us[a * pl.SS + qq];
          float2 nx = cscale(x, r.x), ny = cscale(y, r.x);
          cms(nx, cscale(cconj(e), r.y), y);
          cmac(ny, cscale(e, r.y), x);
          Us[a * pl.SS + pp] = nx;
          Us[a * pl.SS + qq] = ny;
        }
      }
      __syncwarp();
    }
  }

  // order eigenvalues (descending; padded rows last), pick the top L
  const float lam_a = (a < m) ? Ss[a * pl.SS + a].x : -INFINITY;
  int rank = 0;
  float lam_max = 0.f;
#pragma unroll
  for (int b = 0; b < MG; ++b) {
    const float lb = (b < m) ? Ss[b * pl.SS + b].x : -INFINITY;
    lam_max = fmaxf(lam_max, lb);
    rank += (lb > lam_a) || (lb == lam_a && b < a);
  }
  __syncwarp();
  if (rank < MG) sel[rank] = a;
  __syncwarp();
  int idx[LT];
  float inv_sigma[LT];
  bool deficient = false;
#pragma unroll
  for (int r = 0; r < LT; ++r) {
    idx[r] = sel[r < MG ? r : 0];
    const float lam = Ss[idx[r] * pl.SS + idx[r]].x;
    const bool bad = (r < L) && !(lam > 0.f);
    deficient |= bad;
    inv_sigma[r] = (lam > 0.f) ? 1.f / sqrtf(lam) : 0.f;
  }

  // V~[:, r] = H~* u_r / sigma_r; lanes stride over the n columns
  if (kap < K) {
    float2* Vout = A.V + ((size_t)k * K + kap) * n * L;
    for (int c = a; c < n; c += MG) {
      float2 v[LT];
#pragma unroll
      for (int r = 0; r < LT; ++r) v[r] = cz();
      for (int b = 0; b < m; ++b) {
        const float2 hb = cconj(Hs[b * pl.SH + c]);
#pragma unroll
        for (int r = 0; r < LT; ++r) cmac(v[r], hb, Us[b * pl.SS + idx[r]]);
      }
#pragma unroll
      for (int r = 0; r < LT; ++r)
        if (r < L) Vout[(size_t)c * L + r] = cscale(v[r], inv_sigma[r]);
    }
    if (a == 0)
      A.pflag[(size_t)k * K + kap] =
          (deficient ? TS_FLAG_RANK_DEFICIENT : 0) | (converged ? 0 : TS_FLAG_EIG_UNCONVERGED);
  }
}

// ------------------------------------------------------------------ phase 2
struct AccumPlan {
  int T, NC, SG, SV, SF, ES, wstride;
  int off_cs, off_Cs, off_ws, off_Gs, off_Vs, off_Fs, off_Es, total;
};

__host__ __device__ inline AccumPlan accum_plan(int MG, int LT, int T, int NC, int P, int p,
                                                bool svd) {
  AccumPlan pl;
  pl.T = T;
  pl.NC = NC;
  pl.SG = NC + 2;
  pl.SV = NC * LT + 2;
  pl.SF = LT + 2;
  pl.ES = MG * LT + 2;
  pl.wstride = p + 1;
  int o = 0;
  pl.off_cs = o; o += T * P;
  pl.off_Cs = o; o += P * p;
  pl.off_ws = o; o += T * pl.wstride;
  o = (o + 1) & ~1;
  pl.off_Gs = pl.off_Vs = pl.off_Fs = o;
  if (svd) {
    o += p * MG * pl.SG;
    o = (o + 1) & ~1;
    pl.off_Vs = o; o += T * pl.SV;
  } else {
    o += p * MG * pl.SF;
  }
  o = (o + 1) & ~1;
  pl.off_Es = o; o += T * pl.ES;
  pl.total = o;
  return pl;
}

template <int MG, int LT, int NC, bool SVD>
__global__ void __launch_bounds__(kThreads) k_sinr_accumulate(const SinrArgs A, const AccumPlan pl) {
  extern __shared__ __align__(16) float2 sm[];
  const int T = pl.T;
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int i = blockIdx.y;
  const int kap0 = blockIdx.x * T;
  const int kap = kap0 + g;
  const int J = A.J, m = A.m, n = A.n, p = A.p, L = A.L, K = A.K;
  float2* cs = sm + pl.off_cs;
  float2* Cs = sm + pl.off_Cs;
  float2* ws = sm + pl.off_ws;
  float2* Gs = sm + pl.off_Gs;
  float2* Vs = sm + pl.off_Vs;
  float2* Fs = sm + pl.off_Fs;
  float2* Es = sm + pl.off_Es + g * pl.ES;
  const float2* wrow = ws + g * pl.wstride;

  float2 R[MG];      // row a of R_i = sum_{k != i} E_ik E_ik* (+ sigma^2 I later)
  float2 Eself[LT];  // row a of E_ii
#pragma unroll
  for (int b = 0; b < MG; ++b) R[b] = cz();
#pragma unroll
  for (int l = 0; l < LT; ++l) Eself[l] = cz();

  for (int k = 0; k < J; ++k) {
    const int ch = i * J + k;
    __syncthreads();
    if (!SVD) {
      // F_ik[q][a][l] = (G_ik x_2 Pt_k^T)[a][l][q], folded once per call
      const float2* Fch = A.F + (size_t)ch * p * m * L;
      for (int idx = tid; idx < p * MG * LT; idx += blockDim.x) {
        const int l = idx % LT, aa = (idx / LT) % MG, q = idx / (LT * MG);
        Fs[(q * MG + aa) * pl.SF + l] =
            (aa < m && l < L) ? Fch[((size_t)q * m + aa) * L + l] : cz();
      }
    }
    stage_projection(A, ch, kap0, T, cs, Cs, ws, pl.wstride);

    float2 E[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) E[l] = cz();
    if (SVD) {
      for (int c0 = 0; c0 < n; c0 += NC) {
        if (c0 > 0) __syncthreads();
        stage_core_chunk<MG, NC>(A, ch, c0, Gs, pl.SG);
        for (int idx = tid; idx < T * NC * LT; idx += blockDim.x) {
          const int l = idx % LT, cc = (idx / LT) % NC, t = idx / (LT * NC);
          const int kk = kap0 + t, c = c0 + cc;
          float2 v = cz();
          if (kk < K && c < n && l < L) v = A.V[(((size_t)k * K + kk) * n + c) * L + l];
          Vs[t * pl.SV + cc * LT + l] = v;
        }
        __syncthreads();
        float2 h[NC];
        core_chunk<NC>(wrow, Gs, pl.SG, MG, a, p, h);
        const float2* vrow = Vs + g * pl.SV;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
          for (int l = 0; l < LT; ++l) cmac(E[l], h[cc], vrow[cc * LT + l]);
        }
      }
    } else {
      for (int q = 0; q < p; ++q) {
        const float2 w = wrow[q];
        const float2* frow = Fs + (q * MG + a) * pl.SF;
#pragma unroll
        for (int l = 0; l < LT; ++l) cmac(E[l], w, frow[l]);
      }
    }

    if (k == i) {
#pragma unroll
      for (int l = 0; l < LT; ++l) Eself[l] = E[l];
    } else {
#pragma unroll
      for (int l = 0; l < LT; ++l) Es[a * LT + l] = E[l];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < MG; ++b) {
#pragma unroll
        for (int l = 0; l < LT; ++l) cmacc(R[b], E[l], Es[b * LT + l]);
      }
      __syncwarp();
    }
  }

  // noise on the m x m block, identity on the padding rows (eq. 25)
  add_diag(R, a, a < m ? A.sigma2[i] : 1.f);
  // Q~ = R + E_ii E_ii*
  float2 Q[MG];
#pragma unroll
  for (int l = 0; l < LT; ++l) Es[a * LT + l] = Eself[l];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < MG; ++b) {
    Q[b] = R[b];
#pragma unroll
    for (int l = 0; l < LT; ++l) cmacc(Q[b], Eself[l], Es[b * LT + l]);
  }
  __syncwarp();

  bool ok = chol_rows<MG, MG>(R, a);
  ok = chol_rows<MG, MG>(Q, a) && ok;
  float2 Z[LT], Y[LT];
#pragma unroll
  for (int l = 0; l < LT; ++l) Z[l] = Y[l] = Eself[l];
  trsv_rows<MG, MG, LT>(R, Z, a);
  trsv_rows<MG, MG, LT>(Q, Y, a);

  // a_r = |L_Q^{-1} e_r|^2
  float as[LT];
#pragma unroll
  for (int l = 0; l < LT; ++l) as[l] = gsum<MG>(cabs2(Y[l]));

  // F = I + Z*Z (LT x LT), one row per lane a < LT
#pragma unroll
  for (int l = 0; l < LT; ++l) Es[a * LT + l] = Z[l];
  __syncwarp();
  float2 F[LT];
#pragma unroll
  for (int s = 0; s < LT; ++s) F[s] = make_float2(s == a ? 1.f : 0.f, 0.f);
  if (a < LT) {
    for (int b = 0; b < MG; ++b) {
      const float2 zba = cconj(Es[b * LT + a]);
#pragma unroll
      for (int s = 0; s < LT; ++s) cmac(F[s], zba, Es[b * LT + s]);
    }
  }
  __syncwarp();
  ok = chol_rows<MG, LT>(F, a) && ok;
  float2 X[LT];
#pragma unroll
  for (int s = 0; s < LT; ++s) X[s] = make_float2(s == a ? 1.f : 0.f, 0.f);
  trsv_rows<MG, LT, LT>(F, X, a);
  float xs[LT];
#pragma unroll
  for (int s = 0; s < LT; ++s) xs[s] = gsum<MG>(a < LT ? cabs2(X[s]) : 0.f);

  if (kap < K) {
    const float num = pickf(as, a), den = pickf(xs, a);
    float sv = ok ? num / den : __int_as_float(0x7fc00000);
    if (a < L) A.sinr[((size_t)i * K + kap) * L + a] = sv;
    if (A.flags != nullptr && a == 0) {
      uint8_t f = ok ? 0 : TS_FLAG_NOT_PD;
      if (ok && !isfinite(sv)) f |= TS_FLAG_NONFINITE;
      if (SVD)
        for (int k = 0; k < J; ++k) f |= A.pflag[(size_t)k * K + kap];
      A.flags[(size_t)i * K + kap] = f;
    }
  }
}

template <int MG, int LT>
cudaError_t run_precoder(const SinrArgs& A, cudaStream_t s) {
  constexpr int NC = MG >= 16 ? 8 : 16;
  // groups per CTA: as many as fit 96 KB of shared memory, at most 256 / MG
  int T = kThreads / MG;
  PrecoderPlan pl = precoder_plan(MG, T, NC, A.P, A.p, A.n);
  // keep whole warps: the group shuffles and votes use the full lane mask
  while (T * MG > 32 && (size_t)pl.total * sizeof(float2) > 96 * 1024) {
    T /= 2;
    pl = precoder_plan(MG, T, NC, A.P, A.p, A.n);
  }
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget) return cudaErrorInvalidValue;
  auto kern = k_svd_precoder<MG, LT, NC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + T - 1) / T, A.J);
  kern<<<grid, T * MG, smem, s>>>(A, pl);
  return cudaGetLastError();
}

template <int MG, int LT>
cudaError_t run_accumulate(const SinrArgs& A, bool svd, cudaStream_t s) {
  constexpr int NC = MG >= 16 ? 8 : 16;
  int T = (kThreads / MG) > 64 ? 64 : kThreads / MG;
  AccumPlan pl = accum_plan(MG, LT, T, NC, A.P, A.p, svd);
  while (T * MG > 32 && (size_t)pl.total * sizeof(float2) > kSmemBudget) {
    T /= 2;
    pl = accum_plan(MG, LT, T, NC, A.P, A.p, svd);
  }
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget) return cudaErrorInvalidValue;
  dim3 grid((A.K + T - 1) / T, A.J);
  if (svd) {
    auto kern = k_sinr_accumulate<MG, LT, NC, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, T * MG, smem, s>>>(A, pl);
  } else {
    auto kern = k_sinr_accumulate<MG, LT, NC, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, T * MG, smem, s>>>(A, pl);
  }
  return cudaGetLastError();
}

}  // namespace detail
}  // namespace ts
