// Mixed-precision re-evaluation of the SINR of sensitive units (eq. 25-28).
// The finalize kernel forms R = sum_{k != i} E_ik E_ik* + sigma^2 I in FP32
// and lists the units whose SINRs are sensitive to the rounding of R (a
// perturbation of u ||R|| moves them by more than ~2e-6).  FP32 cannot hold
// such an R closely enough: its weak directions, where the serving signal
// lies, are ~sigma^2 while the rounding is ~u ||R||.  Here one warp per
// listed unit (lane a = row a, MG <= 16 lanes in use):
//   1. forms R again from the stored FP32 effective channels, in
//      double-float (each product exact, sums compensated), so R is exact to
//      ~2^-44 ||R|| for the given E;
//   2. factors the leading FP32 part of R, solves Y = R^{-1} E_ii with that
//      factor and refines it three times with residuals E_ii - R Y in FP64
//      against the double-float R (Y kept in FP64);
//   3. forms M = E_ii* Y (L x L) in FP64, factors F = I + M in FP64 (one
//      lane) and evaluates SINR_r = (1 - x_r) / x_r with
//      x_r = [F^{-1}]_rr = |L_F^{-1} e_r|^2 -- the stable form of eq. (5).
// The O(m^3) factorization stays FP32; the products of R and the residuals
// are where the precision goes.  The unit's flags get TS_FLAG_REFINED.
#include "common.cuh"
#include "kernels.h"
#include "tuckersinr.h"

namespace ts {
namespace {

constexpr int kWarps = 4;       // units in flight per CTA

__device__ __forceinline__ double2 dz() { return make_double2(0.0, 0.0); }
// acc += a * b
__device__ __forceinline__ void dmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ double2 d2(float2 v) { return make_double2(v.x, v.y); }

template <int MG, int LT, bool SVD>
__global__ void __launch_bounds__(32 * kWarps) k_sinr_refine(const SinrArgs A) {
  // per warp: E [MG][LT] float2, Y [MG][LT] double2, F [LT][LT] double2
  __shared__ __align__(16) unsigned char smem[kWarps * (MG * LT * 8 + MG * LT * 16 + LT * LT * 16)];
  const int warp = threadIdx.x / 32, a = threadIdx.x % 32;
  unsigned char* mine = smem + warp * (MG * LT * 8 + MG * LT * 16 + LT * LT * 16);
  float2* Es = reinterpret_cast<float2*>(mine);
  double2* Ys = reinterpret_cast<double2*>(mine + MG * LT * 8);
  double2* Fs = reinterpret_cast<double2*>(mine + MG * LT * 8 + MG * LT * 16);
  const int J = A.J, m = A.m, L = A.L, K = A.K;
  const int count = min(*A.rcount, J * K);
  const bool row = a < MG && a < m;
  for (int u = blockIdx.x * kWarps + warp; u < count; u += gridDim.x * kWarps) {
    const int unit = A.rlist[u];
    const int i = unit / K, kap = unit - i * K;
    // 1. R in double-float from the stored effective channels, and E_ii
    float2 Rh[MG], Rl[MG], Eself[LT];
#pragma unroll
    for (int b = 0; b < MG; ++b) Rh[b] = Rl[b] = cz();
#pragma unroll
    for (int l = 0; l < LT; ++l) Eself[l] = cz();
    for (int s = 0; s < J - 1; ++s) {
      float2 Er[LT];
      const float2* Ein = A.Eint + ((((size_t)i * (J - 1) + s) * K + kap) * m + (row ? a : 0)) * L;
#pragma unroll
      for (int l = 0; l < LT; ++l) Er[l] = (row && l < L) ? Ein[l] : cz();
      if (a < MG)
#pragma unroll
        for (int l = 0; l < LT; ++l) Es[a * LT + l] = Er[l];
      __syncwarp();
#pragma unroll
      for (int b = 0; b < MG; ++b)
#pragma unroll
        for (int l = 0; l < LT; ++l) df_cmacc(Rh[b], Rl[b], Er[l], Es[b * LT + l]);
      __syncwarp();
    }
    if (row) {
      const float2* Ein = A.Eserv + (((size_t)i * K + kap) * m + a) * L;
#pragma unroll
      for (int l = 0; l < LT; ++l)
        if (l < L) Eself[l] = Ein[l];
    }
    // noise (exact), identity on the padding rows
#pragma unroll
    for (int b = 0; b < MG; ++b)
      if (b == a) {
        const float sg = row ? A.sigma2[i] : 1.f;
        float sh, sl;
        const float s0 = __fadd_rn(Rh[b].x, sg);
        const float bb = __fsub_rn(s0, Rh[b].x);
        sl = __fadd_rn(__fsub_rn(Rh[b].x, __fsub_rn(s0, bb)), __fsub_rn(sg, bb));
        sh = s0;
        Rh[b].x = sh;
        Rl[b].x = __fadd_rn(Rl[b].x, sl);
      }
    float2 Lr[MG];
#pragma unroll
    for (int b = 0; b < MG; ++b) Lr[b] = Rh[b];
    const bool ok = chol_rows<MG, MG>(Lr, a);
    if (!__all_sync(FULL, ok || a >= MG)) continue;     // keep the FP32 result
    // 2. Y = R^{-1} E_ii, refined with FP64 residuals
    float2 Yf[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) Yf[l] = Eself[l];
    trsv_rows<MG, MG, LT>(Lr, Yf, a);
    trsv_rows_conjT<MG, MG, LT>(Lr, Yf, a);
    double2 Yd[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) Yd[l] = d2(Yf[l]);
    for (int it = 0; it < 3; ++it) {
      if (a < MG)
#pragma unroll
        for (int l = 0; l < LT; ++l) Ys[a * LT + l] = Yd[l];
      __syncwarp();
      float2 Df[LT];
#pragma unroll
      for (int l = 0; l < LT; ++l) {
        double2 r = d2(Eself[l]);
        if (a < MG)
#pragma unroll
          for (int b = 0; b < MG; ++b) {
            const double2 rb = make_double2((double)Rh[b].x + (double)Rl[b].x,
                                            (double)Rh[b].y + (double)Rl[b].y);
            dmac(r, make_double2(-rb.x, -rb.y), Ys[b * LT + l]);
          }
        Df[l] = make_float2((float)r.x, (float)r.y);
      }
      __syncwarp();
      trsv_rows<MG, MG, LT>(Lr, Df, a);
      trsv_rows_conjT<MG, MG, LT>(Lr, Df, a);
#pragma unroll
      for (int l = 0; l < LT; ++l) {
        Yd[l].x += Df[l].x;
        Yd[l].y += Df[l].y;
      }
    }
    // 3. F = I + E_ii* Y (L x L, FP64), row r in lane r
    if (a < MG) {
#pragma unroll
      for (int l = 0; l < LT; ++l) {
        Es[a * LT + l] = Eself[l];
        Ys[a * LT + l] = Yd[l];
      }
    }
    __syncwarp();
    if (a < L) {
      for (int s = 0; s < L; ++s) {
        double2 acc = make_double2(s == a ? 1.0 : 0.0, 0.0);
        for (int b = 0; b < m; ++b) {
          const float2 e = Es[b * LT + a];
          dmac(acc, make_double2(e.x, -e.y), Ys[b * LT + s]);
        }
        Fs[a * LT + s] = acc;
      }
    }
    __syncwarp();
    bool fok = true;
    if (a == 0) {
      // F = L_F L_F* in place (lower triangle), FP64
      for (int j = 0; j < L && fok; ++j) {
        double d = Fs[j * LT + j].x;
        for (int t = 0; t < j; ++t) d -= Fs[j * LT + t].x * Fs[j * LT + t].x + Fs[j * LT + t].y * Fs[j * LT + t].y;
        if (!(d > 0.0)) { fok = false; break; }
        const double ljj = sqrt(d);
        Fs[j * LT + j] = make_double2(ljj, 0.0);
        for (int r = j + 1; r < L; ++r) {
          double2 v = Fs[r * LT + j];
          for (int t = 0; t < j; ++t) {
            // v -= L[r][t] conj(L[j][t])
            const double2 x = Fs[r * LT + t], y = Fs[j * LT + t];
            v.x -= x.x * y.x + x.y * y.y;
            v.y -= x.y * y.x - x.x * y.y;
          }
          Fs[r * LT + j] = make_double2(v.x / ljj, v.y / ljj);
        }
      }
    }
    fok = __shfl_sync(FULL, fok, 0);
    __syncwarp();
    if (!fok) continue;
    if (a < L) {
      // x_r = |L_F^{-1} e_r|^2 by forward substitution from row r
      double2 y[LT];
#pragma unroll
      for (int s = 0; s < LT; ++s) y[s] = dz();
      double x = 0.0;
#pragma unroll
      for (int s = 0; s < LT; ++s) {
        if (s < a || s >= L) continue;
        double2 v = make_double2(s == a ? 1.0 : 0.0, 0.0);
#pragma unroll
        for (int t = 0; t < LT; ++t) {
          if (t < a || t >= s) continue;
          const double2 l = Fs[s * LT + t];
          v.x -= l.x * y[t].x - l.y * y[t].y;
          v.y -= l.x * y[t].y + l.y * y[t].x;
        }
        const double lss = Fs[s * LT + s].x;
        y[s] = make_double2(v.x / lss, v.y / lss);
        x += y[s].x * y[s].x + y[s].y * y[s].y;
      }
      A.sinr[((size_t)i * K + kap) * L + a] = (float)((1.0 - x) / x);
    }
    if (a == 0 && A.flags != nullptr) A.flags[(size_t)i * K + kap] |= TS_FLAG_REFINED;
    __syncwarp();
  }
}

template <int MG, int LT>
cudaError_t run_refine(const SinrArgs& A, bool svd, cudaStream_t s) {
  const int blocks = 152 * 2;
  if (svd)
    k_sinr_refine<MG, LT, true><<<blocks, 32 * kWarps, 0, s>>>(A);
  else
    k_sinr_refine<MG, LT, false><<<blocks, 32 * kWarps, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sinr_refine(const SinrArgs& a, bool svd, cudaStream_t s) {
  const int MG = a.m <= 2 ? 2 : a.m <= 4 ? 4 : a.m <= 8 ? 8 : 16;
  // the stream tiles of the SINR kernels: 16-lane groups start at 4
  const int LT = a.L <= 2 && MG < 16 ? 2 : a.L <= 4 ? 4 : a.L <= 8 ? 8 : 16;
  switch (MG * 100 + LT) {
    case 202: return run_refine<2, 2>(a, svd, s);
    case 402: return run_refine<4, 2>(a, svd, s);
    case 404: return run_refine<4, 4>(a, svd, s);
    case 802: return run_refine<8, 2>(a, svd, s);
    case 804: return run_refine<8, 4>(a, svd, s);
    case 808: return run_refine<8, 8>(a, svd, s);
    case 1604: return run_refine<16, 4>(a, svd, s);
    case 1608: return run_refine<16, 8>(a, svd, s);
    case 1616: return run_refine<16, 16>(a, svd, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ts
