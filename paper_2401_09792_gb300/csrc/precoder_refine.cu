// Refinement of the SVD precoders of units with a close pair of singular
// values (eq. 7 and eq. 23-24 for one BS k and subcarrier kappa, m <= 16).
//
// The per-stream SINRs follow the individual right singular vectors of
// H~_kk(kappa).  When two adjacent squared singular values among the L + 1
// largest are a gap g apart (relative to the largest), a perturbation of
// relative size u in H~ turns their vectors into each other by ~u / g.  In
// the FP32 precoder the rounding of the coefficients c(kappa) and of the sum
// forming H~ is such a perturbation, and for g < kPrecoderCloseGap it alone
// moves the SINRs by more than ~5e-6 (3e-5 at g = 4e-4 on the precision
// workload), however accurately the FP32 eigenvectors are then polished.
// The FP32 precoder lists those units with its left singular vectors
// q_0 .. q_{R-1} of ranks 0 .. R - 1 (R = min(L + 1, m)); here one CTA per
// listed unit
//   1. forms c(kappa) in FP64 from the 64-bit turn count of each path (or
//      takes the given dense coefficients) and w = c* C (eq. 15) in
//      double-float (FP32 pairs: exact products, compensated sums);
//   2. forms H~ = sum_q w_q G[:, :, q] in double-float, one column per
//      thread, and Y = H~* Q (n x R) from it, so that Y* Y = Q* H~ H~* Q
//      holds to ~2^-44 relative for the given Q;
//   3. sweeps twice over the close pairs (r, r + 1) the FP32 precoder
//      marked: the 2 x 2 Gram
//      B = [y_r y_r+1]* [y_r y_r+1] and the metric G = [q_r q_r+1]*
//      [q_r q_r+1] (double-float sums; G = I + E with |E| ~ 1e-7, so the
//      FP32 vectors need not be orthonormal) give the Rayleigh-Ritz pair of
//      B x = lambda G x through the whitening I - E / 2: the difference of
//      the diagonal and the off-diagonal of C = B - (E B + B E) / 2, which
//      carry the pair's separation, come from the double-float sums, the
//      rotation from them in FP32; the columns of Q and Y (double-float)
//      are replaced by Q x and Y x, the larger eigenvalue first (no pair
//      with an eigenvalue below kPrecoderWeak lambda_1 is marked: y = H~* q
//      carries q's absolute FP32 error times sigma_1, too much for a weak
//      vector);
//   4. rewrites, for the columns a rotation touched, V~[:, r] = y_r / |y_r|
//      and E_kk[:, r] = q_r sigma_r / |q_r| with sigma_r = |y_r| / |q_r|
//      (r < L), rounded to FP32 once.
// Inside a pair the rotation now comes from a 2 x 2 problem exact to
// ~2^-44, so the vectors' mixing drops to the FP32 rounding of the output.
// All of it runs on the FP32 pipe except the FP64 sincos of the
// coefficients (this part's FP64 rate is a small fraction of its FP32 one).
// The unit's precoder flags get TS_FLAG_PRECODER_REFINED.
#include "common.cuh"
#include "kernels.h"
#include "tuckersinr.h"

namespace ts {
namespace {

constexpr int kThreads = 128;
constexpr int kPasses = 2;         // sweeps over the adjacent pairs
constexpr int kMaxL = 16;          // streams

// ------------------------------------------------------- double-float types
struct cdf {                       // complex double-float: value h + l
  float2 h, l;
};
__device__ __forceinline__ cdf cdz() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }
__device__ __forceinline__ void fast_two_sum(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}
__device__ __forceinline__ void cdf_norm(cdf& a) {
  fast_two_sum(a.h.x, a.l.x);
  fast_two_sum(a.h.y, a.l.y);
}
__device__ __forceinline__ cdf cdf_of(double2 v) {
  cdf a;
  a.h = make_float2((float)v.x, (float)v.y);
  a.l = make_float2((float)(v.x - (double)a.h.x), (float)(v.y - (double)a.h.y));
  return a;
}
// acc += w g   (w double-float, g FP32)
__device__ __forceinline__ void cdf_mac_f(cdf& acc, const cdf& w, float2 g) {
  df_add_prod(acc.h.x, acc.l.x, w.h.x, g.x);
  df_add_prod(acc.h.x, acc.l.x, -w.h.y, g.y);
  df_add_prod(acc.h.y, acc.l.y, w.h.x, g.y);
  df_add_prod(acc.h.y, acc.l.y, w.h.y, g.x);
  acc.l.x = fmaf(w.l.x, g.x, fmaf(-w.l.y, g.y, acc.l.x));
  acc.l.y = fmaf(w.l.x, g.y, fmaf(w.l.y, g.x, acc.l.y));
}
// acc += conj(a) q   (a double-float, q FP32)
__device__ __forceinline__ void cdf_conj_mac_f(cdf& acc, const cdf& a, float2 q) {
  df_add_prod(acc.h.x, acc.l.x, a.h.x, q.x);
  df_add_prod(acc.h.x, acc.l.x, a.h.y, q.y);
  df_add_prod(acc.h.y, acc.l.y, a.h.x, q.y);
  df_add_prod(acc.h.y, acc.l.y, -a.h.y, q.x);
  acc.l.x = fmaf(a.l.x, q.x, fmaf(a.l.y, q.y, acc.l.x));
  acc.l.y = fmaf(a.l.x, q.y, fmaf(-a.l.y, q.x, acc.l.y));
}
// acc += a b   (both double-float; the l l term is below the result's accuracy)
__device__ __forceinline__ void cdf_mac(cdf& acc, const cdf& a, const cdf& b) {
  df_add_prod(acc.h.x, acc.l.x, a.h.x, b.h.x);
  df_add_prod(acc.h.x, acc.l.x, -a.h.y, b.h.y);
  df_add_prod(acc.h.y, acc.l.y, a.h.x, b.h.y);
  df_add_prod(acc.h.y, acc.l.y, a.h.y, b.h.x);
  acc.l.x = fmaf(a.h.x, b.l.x, fmaf(-a.h.y, b.l.y, fmaf(a.l.x, b.h.x, fmaf(-a.l.y, b.h.y, acc.l.x))));
  acc.l.y = fmaf(a.h.x, b.l.y, fmaf(a.h.y, b.l.x, fmaf(a.l.x, b.h.y, fmaf(a.l.y, b.h.x, acc.l.y))));
}
// acc += conj(a) b   (both double-float)
__device__ __forceinline__ void cdf_conj_mac(cdf& acc, const cdf& a, const cdf& b) {
  df_add_prod(acc.h.x, acc.l.x, a.h.x, b.h.x);
  df_add_prod(acc.h.x, acc.l.x, a.h.y, b.h.y);
  df_add_prod(acc.h.y, acc.l.y, a.h.x, b.h.y);
  df_add_prod(acc.h.y, acc.l.y, -a.h.y, b.h.x);
  acc.l.x = fmaf(a.h.x, b.l.x, fmaf(a.h.y, b.l.y, fmaf(a.l.x, b.h.x, fmaf(a.l.y, b.h.y, acc.l.x))));
  acc.l.y = fmaf(a.h.x, b.l.y, fmaf(-a.h.y, b.l.x, fmaf(a.l.x, b.h.y, fmaf(-a.l.y, b.h.x, acc.l.y))));
}

// --------------------------------------------------------- FP64 complex
__device__ __forceinline__ double2 d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }

// c_p(kappa) of link ch in FP64: the dense coefficients as given, or the
// path form conj(alpha_p) exp(+j 2 pi kappa df tau_p) with the phase from the
// full 64-bit turn count (half-turns in [-1, 1) at 2^-63 resolution)
__device__ double2 coef64(const SinrArgs& A, int ch, int pp, int kap) {
  const int kg = A.kap_off + kap;
  if (A.coef_mode == 0) return d2(A.coef[((size_t)ch * A.Kc + kg) * A.P + pp]);
  const double2 al = d2(A.coef[(size_t)ch * A.P + pp]);
  const unsigned long long ph = A.turns[(size_t)ch * A.P + pp] * (unsigned long long)kg;
  const double x = (double)(long long)ph * 0x1p-63;
  double sn, cs;
  sincospi(x, &sn, &cs);
  return make_double2(fma(al.x, cs, al.y * sn), fma(al.x, sn, -al.y * cs));
}

// Sum over the CTA of NV double-float reals held per thread (in place in
// h[], l[]); thread 0 gets the totals in h[], l[].  red: 4 x NV x 2 floats
// (four warps).
template <int NV>
__device__ void block_sum_df(float* h, float* l, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int v = 0; v < NV; ++v)
      df_add(h[v], l[v], __shfl_xor_sync(FULL, h[v], o), __shfl_xor_sync(FULL, l[v], o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      red[(warp * NV + v) * 2] = h[v];
      red[(warp * NV + v) * 2 + 1] = l[v];
    }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      h[v] = red[v * 2];
      l[v] = red[v * 2 + 1];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        df_add(h[v], l[v], red[(w * NV + v) * 2], red[(w * NV + v) * 2 + 1]);
    }
}

// Shared-memory plan (bytes).
struct Plan {
  int R;
  size_t off_c, off_w, off_Q, off_Y, off_red, off_X, off_t, off_sc, total;
};

Plan make_plan(int m, int n, int p, int P, int L) {
  Plan pl;
  pl.R = L + 1 < m ? L + 1 : m;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = (o + bytes + 15) & ~(size_t)15;
    return at;
  };
  pl.off_c = take((size_t)P * sizeof(cdf));            // conj(c(kappa))
  pl.off_w = take((size_t)p * sizeof(cdf));            // w = c* C
  pl.off_Q = take((size_t)pl.R * m * sizeof(cdf));     // the vectors q_j (double-float)
  pl.off_Y = take((size_t)pl.R * n * sizeof(cdf));     // Y = H~* Q
  pl.off_red = take(4 * 8 * 2 * sizeof(float));
  pl.off_X = take(4 * sizeof(float2) + 16);
  pl.off_t = take((size_t)pl.R * sizeof(int));          // columns a pair rotation touched
  pl.off_sc = take(2 * kMaxL * sizeof(float));
  pl.total = o;
  return pl;
}

// One CTA per listed unit.  H~ and Y: SPLIT threads per column of H~, each
// on MG / SPLIT rows (so that narrow H~ still occupies the CTA), Y summed over
// the SPLIT lanes by shuffles.
template <int MG, int SPLIT>
__global__ void __launch_bounds__(kThreads) k_precoder_refine(const SinrArgs A, const Plan pl) {
  constexpr int RPT = MG / SPLIT;                   // rows of H~ per thread
  extern __shared__ __align__(16) unsigned char sm[];
  const int J = A.J, m = A.m, n = A.n, p = A.p, P = A.P, K = A.K, L = A.L, R = pl.R;
  const int tid = threadIdx.x, nth = blockDim.x;
  cdf* cc = reinterpret_cast<cdf*>(sm + pl.off_c);
  cdf* ws = reinterpret_cast<cdf*>(sm + pl.off_w);
  cdf* Q = reinterpret_cast<cdf*>(sm + pl.off_Q);           // [R][m]
  cdf* Y = reinterpret_cast<cdf*>(sm + pl.off_Y);           // [R][n]
  float* red = reinterpret_cast<float*>(sm + pl.off_red);
  float2* Xs = reinterpret_cast<float2*>(sm + pl.off_X);    // X00 X10 X01 X11
  int* xok = reinterpret_cast<int*>(sm + pl.off_X + 4 * sizeof(float2));
  int* touched = reinterpret_cast<int*>(sm + pl.off_t);     // [R]
  float* sc = reinterpret_cast<float*>(sm + pl.off_sc);     // [L] V and [L] E scales
  const int count = min(*A.rcount, J * K);
  for (int u = blockIdx.x; u < count; u += gridDim.x) {
    const int unit = A.rlist[u];
    const int mask = A.close_mask[u];
    const int k = unit / K, kap = unit - k * K;
    const int ch = k * J + k;
    __syncthreads();                                  // the previous unit's data consumed
    // 1. conj(c(kappa)) in FP64 -> double-float; the listed vectors
    for (int pp = tid; pp < P; pp += nth) cc[pp] = cdf_of(dconj(coef64(A, ch, pp, kap)));
    for (int i2 = tid; i2 < R * m; i2 += nth) {
      cdf q = cdz();
      q.h = A.Uclose[(size_t)u * R * m + i2];
      Q[i2] = q;
    }
    for (int j = tid; j < R; j += nth) touched[j] = 0;
    __syncthreads();
    // w_q = sum_p conj(c_p) C[p][q] (w = conj(c) when C = I)
    for (int q = tid; q < p; q += nth) {
      cdf acc = cdz();
      if (A.identity_C) {
        acc = cc[q];
      } else {
        const float2* Cq = A.C + (size_t)ch * P * p + q;
        for (int pp = 0; pp < P; ++pp) cdf_mac_f(acc, cc[pp], __ldg(Cq + (size_t)pp * p));
        cdf_norm(acc);
      }
      ws[q] = acc;
    }
    __syncthreads();
    // 2. H~[:, c] = sum_q w_q G[:, c, q] and Y[c][j] = sum_b conj(H~[b][c]) q_j[b]
    {
      const int sp = tid % SPLIT, b0 = sp * RPT;
      const float2* Gch = A.G + (size_t)ch * p * m * n;
      for (int cb = 0; cb < n; cb += nth / SPLIT) {     // uniform trip count (shuffles below)
        const int c = cb + tid / SPLIT;
        const bool act = c < n;
        cdf h[RPT];
#pragma unroll
        for (int bb = 0; bb < RPT; ++bb) h[bb] = cdz();
        if (act) {
          const float2* g = Gch + c;
          for (int q = 0; q < p; ++q) {
            const cdf wq = ws[q];
            float2 gv[RPT];
#pragma unroll
            for (int bb = 0; bb < RPT; ++bb)
              gv[bb] = b0 + bb < m ? __ldg(g + ((size_t)q * m + b0 + bb) * n) : make_float2(0.f, 0.f);
#pragma unroll
            for (int bb = 0; bb < RPT; ++bb) cdf_mac_f(h[bb], wq, gv[bb]);
          }
        }
#pragma unroll
        for (int bb = 0; bb < RPT; ++bb) cdf_norm(h[bb]);
        for (int j = 0; j < R; ++j) {
          cdf y = cdz();
#pragma unroll
          for (int bb = 0; bb < RPT; ++bb)
            if (b0 + bb < m) cdf_conj_mac_f(y, h[bb], Q[j * m + b0 + bb].h);
#pragma unroll
          for (int o = 1; o < SPLIT; o <<= 1) {
            df_add(y.h.x, y.l.x, __shfl_xor_sync(FULL, y.h.x, o), __shfl_xor_sync(FULL, y.l.x, o));
            df_add(y.h.y, y.l.y, __shfl_xor_sync(FULL, y.h.y, o), __shfl_xor_sync(FULL, y.l.y, o));
          }
          cdf_norm(y);
          if (act && sp == 0) Y[j * n + c] = y;
        }
      }
    }
    __syncthreads();
    // 3. Rayleigh-Ritz on the close pairs (r, s = r + 1).  With the metric
    // G = I + E (|E| ~ 1e-7: the vectors are orthonormal to FP32 rounding)
    // the whitening W = I - E / 2 satisfies W* G W = I + O(E^2), so
    // C = W* B W = B - (E B + B E) / 2 and X = W Z, Z the 2 x 2 eigenvectors
    // of C.  c_ss - c_rr and c_rs carry the pair's separation and are formed
    // from double-float B and E; the rotation itself is FP32.
    for (int pass = 0; pass < kPasses; ++pass) {
      for (int r = 0; r + 1 < R; ++r) {
        if (!((mask >> r) & 1)) continue;               // uniform over the CTA
        const int s2 = r + 1;
        // B: b_rr, b_ss, b_rs (re, im); E + I: g_rr, g_ss, g_rs (re, im)
        float vh[8], vl[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) vh[v] = vl[v] = 0.f;
        for (int c = tid; c < n; c += nth) {
          const cdf y1 = Y[r * n + c], y2 = Y[s2 * n + c];
          cdf a11 = cdz(), a22 = cdz(), a12 = cdz();
          cdf_conj_mac(a11, y1, y1);
          cdf_conj_mac(a22, y2, y2);
          cdf_conj_mac(a12, y1, y2);
          df_add(vh[0], vl[0], a11.h.x, a11.l.x);
          df_add(vh[1], vl[1], a22.h.x, a22.l.x);
          df_add(vh[2], vl[2], a12.h.x, a12.l.x);
          df_add(vh[3], vl[3], a12.h.y, a12.l.y);
        }
        for (int b = tid; b < m; b += nth) {
          const cdf q1 = Q[r * m + b], q2 = Q[s2 * m + b];
          cdf a11 = cdz(), a22 = cdz(), a12 = cdz();
          cdf_conj_mac(a11, q1, q1);
          cdf_conj_mac(a22, q2, q2);
          cdf_conj_mac(a12, q1, q2);
          df_add(vh[4], vl[4], a11.h.x, a11.l.x);
          df_add(vh[5], vl[5], a22.h.x, a22.l.x);
          df_add(vh[6], vl[6], a12.h.x, a12.l.x);
          df_add(vh[7], vl[7], a12.h.y, a12.l.y);
        }
        block_sum_df<8>(vh, vl, red);
        if (tid == 0) {
          // E = G - I (the high parts of g_rr, g_ss are within [1/2, 2] of 1,
          // so their difference from 1 is exact)
          const float e11 = __fadd_rn(__fsub_rn(vh[4], 1.f), vl[4]);
          const float e22 = __fadd_rn(__fsub_rn(vh[5], 1.f), vl[5]);
          const float2 e12 = make_float2(vh[6] + vl[6], vh[7] + vl[7]);
          const float b11 = vh[0] + vl[0], b22 = vh[1] + vl[1];
          const float2 b12 = make_float2(vh[2] + vl[2], vh[3] + vl[3]);
          // b_ss - b_rr from the double-float parts (the high parts of two
          // close eigenvalues differ exactly)
          const float db = __fadd_rn(__fsub_rn(vh[1], vh[0]), __fsub_rn(vl[1], vl[0]));
          // C = B - (E B + B E) / 2 to first order in E
          const float dc = db - (e22 * b22 - e11 * b11);                    // c_ss - c_rr
          const float2 c12 = make_float2(
              b12.x - 0.5f * ((e11 + e22) * b12.x + e12.x * (b11 + b22)),
              b12.y - 0.5f * ((e11 + e22) * b12.y + e12.y * (b11 + b22)));
          const float ab = sqrtf(fmaf(c12.x, c12.x, c12.y * c12.y));
          float cz_ = 1.f, sz = 0.f, t = 0.f;
          float2 e = make_float2(1.f, 0.f);
          if (ab > 0.f) {
            const float tau = dc / (2.f * ab);
            t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
            cz_ = 1.f / sqrtf(fmaf(t, t, 1.f));
            sz = t * cz_;
            e = make_float2(c12.x / ab, c12.y / ab);
          }
          // Z = [c  s e; -s conj(e)  c]: eigenvalues c_rr - t |c_rs| and
          // c_ss + t |c_rs|; the larger one first
          float2 z00 = make_float2(cz_, 0.f), z10 = make_float2(-sz * e.x, sz * e.y);
          float2 z01 = make_float2(sz * e.x, sz * e.y), z11 = make_float2(cz_, 0.f);
          if (dc + 2.f * t * ab > 0.f) {
            float2 tmp = z00; z00 = z01; z01 = tmp;
            tmp = z10; z10 = z11; z11 = tmp;
          }
          // X = (I - E / 2) Z
          const float2 e21 = make_float2(e12.x, -e12.y);
          auto col = [&](float2 za, float2 zb, float2& xa, float2& xb) {
            xa = make_float2(za.x - 0.5f * (e11 * za.x + (e12.x * zb.x - e12.y * zb.y)),
                             za.y - 0.5f * (e11 * za.y + (e12.x * zb.y + e12.y * zb.x)));
            xb = make_float2(zb.x - 0.5f * ((e21.x * za.x - e21.y * za.y) + e22 * zb.x),
                             zb.y - 0.5f * ((e21.x * za.y + e21.y * za.x) + e22 * zb.y));
          };
          float2 x00, x10, x01, x11;
          col(z00, z10, x00, x10);
          col(z01, z11, x01, x11);
          Xs[0] = x00; Xs[1] = x10; Xs[2] = x01; Xs[3] = x11;
          // (the FP32 precoder marks no pair with a member below
          // kPrecoderWeak lambda_1: for such a vector y = H~* q carries q's
          // absolute FP32 error times sigma_1, more than the pair's mixing)
          const bool ok = vh[4] > 0.f && vh[5] > 0.f;
          *xok = ok;
          if (ok) touched[r] = touched[s2] = 1;
        }
        __syncthreads();
        if (*xok) {
          const float2 x00 = Xs[0], x10 = Xs[1], x01 = Xs[2], x11 = Xs[3];
          for (int c = tid; c < n; c += nth) {
            const cdf y1 = Y[r * n + c], y2 = Y[s2 * n + c];
            cdf n1 = cdz(), n2 = cdz();
            cdf_mac_f(n1, y1, x00);
            cdf_mac_f(n1, y2, x10);
            cdf_mac_f(n2, y1, x01);
            cdf_mac_f(n2, y2, x11);
            cdf_norm(n1);
            cdf_norm(n2);
            Y[r * n + c] = n1;
            Y[s2 * n + c] = n2;
          }
          for (int b = tid; b < m; b += nth) {
            const cdf q1 = Q[r * m + b], q2 = Q[s2 * m + b];
            cdf n1 = cdz(), n2 = cdz();
            cdf_mac_f(n1, q1, x00);
            cdf_mac_f(n1, q2, x10);
            cdf_mac_f(n2, q1, x01);
            cdf_mac_f(n2, q2, x11);
            cdf_norm(n1);
            cdf_norm(n2);
            Q[r * m + b] = n1;
            Q[s2 * m + b] = n2;
          }
        }
        __syncthreads();
      }
    }
    // 4. for the touched columns r < L: sigma_r = |y_r| / |q_r|,
    // V~[:, r] = y_r / |y_r|, E_kk[:, r] = q_r sigma_r / |q_r|; the others keep
    // the FP32 precoder's output
    bool deficient = false;
    for (int r = 0; r < L; ++r) {
      if (!touched[r]) continue;                        // uniform over the CTA
      float vh[2] = {0.f, 0.f}, vl[2] = {0.f, 0.f};
      for (int c = tid; c < n; c += nth) {
        const cdf y = Y[r * n + c];
        cdf a = cdz();
        cdf_conj_mac(a, y, y);
        df_add(vh[0], vl[0], a.h.x, a.l.x);
      }
      for (int b = tid; b < m; b += nth) {
        const cdf q = Q[r * m + b];
        cdf a = cdz();
        cdf_conj_mac(a, q, q);
        df_add(vh[1], vl[1], a.h.x, a.l.x);
      }
      block_sum_df<2>(vh, vl, red);
      if (tid == 0) {
        const float yn = vh[0] + vl[0], qn = vh[1] + vl[1];
        const bool pos = yn > 0.f && qn > 0.f;
        deficient |= !pos;
        sc[r] = pos ? 1.f / sqrtf(yn) : 0.f;                   // V scale
        sc[kMaxL + r] = pos ? sqrtf(yn) / qn : 0.f;            // E scale: sigma / |q|
      }
      __syncthreads();                                  // red reused by the next column
    }
    if (tid == 0) {
      const uint8_t old = A.pflag[(size_t)k * K + kap];
      A.pflag[(size_t)k * K + kap] =
          (uint8_t)(old | TS_FLAG_PRECODER_REFINED | (deficient ? TS_FLAG_RANK_DEFICIENT : 0));
    }
    float2* Vout = A.V + ((size_t)k * K + kap) * n * L;
    for (int i2 = tid; i2 < n * L; i2 += nth) {
      const int c = i2 / L, r = i2 - c * L;
      if (!touched[r]) continue;
      const cdf y = Y[r * n + c];
      Vout[i2] = make_float2((y.h.x + y.l.x) * sc[r], (y.h.y + y.l.y) * sc[r]);
    }
    float2* Eout = A.Eserv + ((size_t)k * K + kap) * m * L;
    for (int i2 = tid; i2 < m * L; i2 += nth) {
      const int a = i2 / L, r = i2 - a * L;
      if (!touched[r]) continue;
      const cdf q = Q[r * m + a];
      Eout[i2] = make_float2((q.h.x + q.l.x) * sc[kMaxL + r], (q.h.y + q.l.y) * sc[kMaxL + r]);
    }
  }
}

template <int MG, int SPLIT>
cudaError_t run(const SinrArgs& A, const Plan& pl, cudaStream_t s) {
  auto kern = k_precoder_refine<MG, SPLIT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.total);
  if (e != cudaSuccess) return e;
  // a fixed grid whose CTAs take the listed units in turn (the list is
  // short: a few in a hundred units)
  kern<<<152 * 4, kThreads, pl.total, s>>>(A, pl);
  return cudaGetLastError();
}

template <int MG>
cudaError_t run_split(const SinrArgs& A, const Plan& pl, cudaStream_t s) {
  // SPLIT threads per column of H~ keep a narrow H~ on every warp of the CTA
  if (MG >= 4 && A.n <= kThreads / 4) return run<MG, (MG >= 4 ? 4 : 1)>(A, pl, s);
  if (MG >= 2 && A.n <= kThreads / 2) return run<MG, (MG >= 2 ? 2 : 1)>(A, pl, s);
  return run<MG, 1>(A, pl, s);
}

}  // namespace

cudaError_t launch_precoder_refine(const SinrArgs& a, cudaStream_t s) {
  if (!a.list_close || a.rlist == nullptr || a.rcount == nullptr || a.Uclose == nullptr)
    return cudaSuccess;
  if (a.m > 16 || a.L > kMaxL) return cudaErrorInvalidValue;
  const Plan pl = make_plan(a.m, a.n, a.p, a.P, a.L);
  if (pl.total > 227 * 1024) return cudaErrorInvalidValue;
  if (a.m <= 2) return run_split<2>(a, pl, s);
  if (a.m <= 4) return run_split<4>(a, pl, s);
  if (a.m <= 8) return run_split<8>(a, pl, s);
  return run_split<16>(a, pl, s);
}

}  // namespace ts
