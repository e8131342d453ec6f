// SINR kernels for the groupwise Tucker form (arXiv 2401.09792, Section 3.3).
//
// Work decomposition.  A unit is one (UE i, subcarrier kappa).  A group of MG
// consecutive lanes (MG = next power of two >= m) evaluates one unit, lane a
// owning row a of every m-row matrix: the compressed channel H~_ik(kappa)
// (eq. 15), the effective channel E_ik = H~_ik V~_k (eq. 24), the covariance
// Q~_i (eq. 25) and its Cholesky factor.  A CTA of 128 threads holds
// T = 128 / MG consecutive subcarriers of one UE (or BS).
//
//   k_svd_precoder       (BS k, subcarrier tile): H~_kk, Gram H~_kk H~_kk*,
//                        Jacobi eigensolve, V~_k = H~_kk* U_L Sigma_L^{-1}
//                        (eq. 7, eq. 23) and the serving effective channel
//                        E_kk = H~_kk V~_k = U_L Sigma_L -> workspace
//   k_sinr_link_blk      (subcarrier tile, UE i, interfering link k), SVD
//                        precoders: w = c* C (eq. 15), E_ik = H~_ik V~_k and
//                        the partial covariance E_ik E_ik* -> workspace, two
//                        subcarriers and two rows per lane.  The core and
//                        precoder column chunks are staged through a
//                        double-buffered cp.async pipeline, one chunk ahead
//                        of the arithmetic.
//   k_sinr_link          the same, one row per lane (m <= 2, large dense
//                        coefficient tiles), the wideband-precoder fold
//                        E_ik = sum_q w_q F_ik[q], the serving links H~_kk
//                        when the cores are too large to re-read per
//                        precoder tile, and the rebuild of every H~_ik for
//                        the adjoint.
//   k_sinr_finalize      (UE i, subcarrier): R_i = sum_{k != i} E E* +
//                        sigma^2 I, Q~_i = R_i + E_ii E_ii* (eq. 25), then the
//                        SINR of eq. (5) in a cancellation-free form (below).
//   k_sinr_link_wide     the interfering and serving links when the core does
//                        not fit the staging above (p > 32 or P p > 8192),
//                        in sinr_wide.cuh.
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

constexpr int kThreads = 128;
// dynamic shared memory a SINR launch may use (the per-CTA limit is 227 KB)
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ float2 path_coef(float2 alpha, unsigned long long turn, int kappa) {
  // c_p(kappa) = conj(alpha_p) exp(+j 2 pi kappa df tau_p); the phase is kept
  // modulo one turn in 64-bit fixed point, then mapped to half-turns in [-1, 1)
  // from its upper 32 bits (a 2^-31 half-turn step, far below FP32 sincos
  // accuracy; a 64-bit integer conversion would run on the FP64 pipe)
  const unsigned long long ph = turn * (unsigned long long)kappa;
  const float x = (float)(int)(unsigned)(ph >> 32) * 0x1p-31f;
  float s, c;
  sincospif(x, &s, &c);
  return make_float2(fmaf(alpha.x, c, alpha.y * s), fmaf(alpha.x, s, -alpha.y * c));
}

// 8-byte asynchronous global->shared copy; `valid == false` writes zeros and
// reads nothing (the source operand then only needs to be a global address).
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int nbytes = valid ? 8 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes)
               : "memory");
}
// 16-byte asynchronous copy (both addresses 16-byte aligned); `valid ==
// false` writes zeros and reads nothing.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int nbytes = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(nbytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// H~ chunk of row a for one subcarrier: h[cc] = sum_q w_q G[q][a][cc] from a
// shared-memory chunk with row stride SG (float2 units, even).
template <int NC>
__device__ __forceinline__ void core_chunk(const float2* wrow, const float2* Gs, int SG, int MG,
                                           int a, int p, float2 (&h)[NC]) {
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) h[cc] = cz();
#pragma unroll 4
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

// One step of cyclic two-sided Jacobi on the Hermitian MG x MG matrix S
// (row a of S and of the accumulated rotation U in lane a of the group), with
// the round-robin ordering: in step t (0 <= t < MG-1) lane MG-1 pairs with
// lane t, and lanes t+j, t-j (mod MG-1) pair for 1 <= j < MG/2.  For a pair
// (p, q) with S_pq = |b| e^{i phi} the rotation is
// J = [[c, s e^{i phi}], [-s e^{-i phi}, c]] -- the real symmetric Jacobi
// rotation of [[S_pp, |b|], [|b|, S_qq]] conjugated by diag(1, e^{-i phi}) --
// and S <- J* S J, U <- U J.  Both lanes of a pair compute the rotation from
// the same three numbers (lane p's S_pq and the two diagonals), so they agree
// bit for bit; rows are exchanged by shuffles, columns rotate in registers.
// The diagonal entry of the lane's row is tracked in `dg` (S_pp - t|b|,
// S_qq + t|b|), which spares a register select per step.  The rotation uses
// hardware reciprocal square roots: any (c, s) with c^2 + s^2 = 1 to a few
// ulps is a valid Jacobi rotation, and the iteration still drives the
// off-diagonal to zero.  S is expected to be scaled to unit trace.
template <int MG>
__device__ __forceinline__ void jacobi_step(const int t, float2 (&S)[MG], float2 (&U)[MG],
                                            float& dg, int a) {
  int b;
  bool is_p;
  if (a == MG - 1) { b = t; is_p = false; }
  else if (a == t) { b = MG - 1; is_p = true; }
  else {
    const int d = (a - t + (MG - 1)) % (MG - 1);
    is_p = d < MG / 2;
    b = (2 * t - a + 2 * (MG - 1)) % (MG - 1);
  }
  const float d_other = __shfl_sync(FULL, dg, b, MG);
  const float2 mine = pick(S, b);
  const float2 theirs = gshfl<MG>(mine, b);
  const float app = is_p ? dg : d_other, aqq = is_p ? d_other : dg;
  const float2 bpq = is_p ? mine : theirs;
  const float ab2 = cabs2(bpq);
  float c = 1.f;
  float2 se = cz();                        // s e^{i phi}
  if (ab2 > 1e-36f && ab2 > 1e-18f * fabsf(app * aqq)) {
    const float r = rsqrtf(ab2);           // 1 / |b|
    const float tau = 0.5f * (aqq - app) * r;
    const float at = fabsf(tau);
    const float h = fmaf(tau, tau, 1.f);
    // t = sign(tau) / (|tau| + sqrt(1 + tau^2)), the smaller root
    const float tm = at > 1e15f ? __fdividef(0.5f, at) : __fdividef(1.f, at + h * rsqrtf(h));
    const float tt = copysignf(tm, tau);
    c = rsqrtf(fmaf(tt, tt, 1.f));
    se = cscale(bpq, tt * c * r);
    const float tb = tt * (ab2 * r);
    dg = is_p ? app - tb : aqq + tb;
  }
  // rows: S <- J* S (row p' = c p - s e q, row q' = s conj(e) p + c q)
  {
    const float2 f = is_p ? make_float2(-se.x, -se.y) : cconj(se);
#pragma unroll
    for (int k = 0; k < MG; ++k) {
      const float2 other = gshfl<MG>(S[k], b);
      float2 v = cscale(S[k], c);
      cmac(v, f, other);
      S[k] = v;
    }
  }
  // columns: S <- S J and U <- U J, every pair of this step
#pragma unroll
  for (int j = 0; j < MG / 2; ++j) {
    const int pj = j == 0 ? t : (t + j) % (MG - 1);
    const int qj = j == 0 ? MG - 1 : (t - j + MG - 1) % (MG - 1);
    const float cj = __shfl_sync(FULL, c, pj, MG);
    const float2 se_j = gshfl<MG>(se, pj), sec_j = cconj(se_j);
    {
      const float2 x = S[pj], y = S[qj];
      float2 nx = cscale(x, cj), ny = cscale(y, cj);
      cms(nx, sec_j, y);     // c x - s conj(e) y
      cmac(ny, se_j, x);     // s e x + c y
      S[pj] = nx;
      S[qj] = ny;
    }
    {
      const float2 x = U[pj], y = U[qj];
      float2 nx = cscale(x, cj), ny = cscale(y, cj);
      cms(nx, sec_j, y);
      cmac(ny, se_j, x);
      U[pj] = nx;
      U[qj] = ny;
    }
  }
}

// The same sweep for 16 rows in a "conveyor" ordering whose code does not
// depend on the step.  Register slot s of every lane holds column
// cv_col(s, t) at step t, and the pairs of step t are the columns in slots
// (2j, 2j + 1); after each step the slot contents move one place along the
// 15-cycle of slots other than slot 1 (a circle-method round robin: every
// pair of columns meets once in 15 steps).  Three steps are unrolled, their
// pair slots fixed at compile time relative to the layout at the start of
// the three, which is then rotated in registers; the whole sweep is a loop
// of five such bodies (15 unrolled steps would not fit the instruction
// cache).  Slots and columns coincide at the start of every sweep.
__host__ __device__ constexpr int cv_cyc(int k) { return k == 0 ? 0 : k <= 7 ? 2 * k + 1 : 2 * (15 - k); }
__host__ __device__ constexpr int cv_pos(int s) { return s == 0 ? 0 : (s & 1) ? (s - 1) / 2 : 15 - s / 2; }
__host__ __device__ constexpr int cv_col(int s, int t) {
  return s == 1 ? 1 : cv_cyc(((cv_pos(s) - t) % 15 + 15) % 15);
}
__host__ __device__ constexpr int cv_slot(int c, int t) { return c == 1 ? 1 : cv_cyc((cv_pos(c) + t) % 15); }

template <int TT>
__device__ __forceinline__ void conveyor_step16(const int t0, float2 (&S)[16], float2 (&U)[16],
                                                float& dg, int a) {
  constexpr int MG = 16;
  const int t = t0 + TT;
  const int sa = cv_slot(a, t);
  const int b = cv_col(sa ^ 1, t);                // partner row
  const bool is_p = (sa & 1) == 0;
  const float d_other = __shfl_sync(FULL, dg, b, MG);
  const float2 mine = pick(S, cv_slot(b, t0));    // S_ab in the layout of step t0
  const float2 theirs = gshfl<MG>(mine, b);
  const float app = is_p ? dg : d_other, aqq = is_p ? d_other : dg;
  const float2 bpq = is_p ? mine : theirs;
  const float ab2 = cabs2(bpq);
  float c = 1.f;
  float2 se = cz();                        // s e^{i phi}
  if (ab2 > 1e-36f && ab2 > 1e-18f * fabsf(app * aqq)) {
    const float r = rsqrtf(ab2);           // 1 / |b|
    const float tau = 0.5f * (aqq - app) * r;
    const float at = fabsf(tau);
    const float h = fmaf(tau, tau, 1.f);
    const float tm = at > 1e15f ? __fdividef(0.5f, at) : __fdividef(1.f, at + h * rsqrtf(h));
    const float tt = copysignf(tm, tau);
    c = rsqrtf(fmaf(tt, tt, 1.f));
    se = cscale(bpq, tt * c * r);
    const float tb = tt * (ab2 * r);
    dg = is_p ? app - tb : aqq + tb;
  }
  {
    const float2 f = is_p ? make_float2(-se.x, -se.y) : cconj(se);
#pragma unroll
    for (int k = 0; k < MG; ++k) {
      const float2 other = gshfl<MG>(S[k], b);
      float2 v = cscale(S[k], c);
      cmac(v, f, other);
      S[k] = v;
    }
  }
#pragma unroll
  for (int j = 0; j < MG / 2; ++j) {
    const int ps = cv_col(2 * j, TT), qs = cv_col(2 * j + 1, TT);   // slots (compile time)
    const int src = cv_col(2 * j, t);                                // lane p of the pair
    const float cj = __shfl_sync(FULL, c, src, MG);
    const float2 se_j = gshfl<MG>(se, src), sec_j = cconj(se_j);
    {
      const float2 x = S[ps], y = S[qs];
      float2 nx = cscale(x, cj), ny = cscale(y, cj);
      cms(nx, sec_j, y);
      cmac(ny, se_j, x);
      S[ps] = nx;
      S[qs] = ny;
    }
    {
      const float2 x = U[ps], y = U[qs];
      float2 nx = cscale(x, cj), ny = cscale(y, cj);
      cms(nx, sec_j, y);
      cmac(ny, se_j, x);
      U[ps] = nx;
      U[qs] = ny;
    }
  }
}

// slot contents three places along the conveyor cycle (slot 1 stays)
__device__ __forceinline__ void conveyor_rotate3(float2 (&X)[16]) {
  float2 tmp[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) tmp[s] = X[s];
#pragma unroll
  for (int k = 0; k < 15; ++k) X[cv_cyc((k + 3) % 15)] = tmp[cv_cyc(k)];
}

__device__ __forceinline__ void jacobi_sweep16(float2 (&S)[16], float2 (&U)[16], float& dg, int a) {
#pragma unroll 1
  for (int t0 = 0; t0 < 15; t0 += 3) {
    conveyor_step16<0>(t0, S, U, dg, a);
    conveyor_step16<1>(t0, S, U, dg, a);
    conveyor_step16<2>(t0, S, U, dg, a);
    conveyor_rotate3(S);
    conveyor_rotate3(U);
  }
}

// ------------------------------------------------------------------ phase 1
// k_svd_precoder: one group of MG lanes per (BS k, subcarrier).  Forms the
// serving link's compressed channel H~_kk (or reads it from workspace: large
// cores, and the all-link rebuild of the adjoint), the Gram S = H~ H~*, diagonalises it by cyclic
// Jacobi, rotates the rows W = U* H~, refines them by one-sided Jacobi when a
// kept singular value is small, and writes the top-L right singular vectors
// V~ (normalised rows of W, in order of decreasing row norm = singular value).
struct PrecoderPlan {
  int T, SH, SS;
  int off_Hs, off_Ss, off_Us, off_cs, off_w, off_sel, total;
};

// coefficient chunk of the fused H~_kk evaluation
constexpr int kServePC = 32;

__host__ __device__ inline PrecoderPlan precoder_plan(int MG, int T, int n, int p, bool fused) {
  PrecoderPlan pl;
  pl.T = T;
  pl.SH = n + 1;
  pl.SS = MG + 1;
  int o = 0;
  pl.off_Hs = o; o += T * MG * pl.SH;
  // S and U scratch; before the Gram it holds the coefficient chunk and the
  // projections w of the fused H~_kk evaluation
  int r = 2 * T * MG * pl.SS;
  if (fused && T * (kServePC + p) > r) r = T * (kServePC + p);
  pl.off_Ss = o;
  pl.off_Us = o + T * MG * pl.SS;
  pl.off_cs = o;
  pl.off_w = o + T * kServePC;
  o += r;
  pl.off_sel = o; o += T * MG / 2 + 1;   // MG int per group
  pl.total = o;
  return pl;
}

// H~_kk(kappa) = sum_q w_q G_kk[:, :, q] with w = C_kk^T conj(c(kappa))
// (eq. 15, link (k, k)) for the T subcarriers of a precoder CTA, written to
// the rows of Hs (zero rows for a >= m and for kappa >= K).
template <int MG>
__device__ __forceinline__ void serve_channels(const SinrArgs& A, const PrecoderPlan& pl, int k,
                                               int kap0, float2* sm) {
  const int T = pl.T, nth = blockDim.x, tid = threadIdx.x;
  const int J = A.J, m = A.m, n = A.n, p = A.p, P = A.P, K = A.K;
  const int ch = k * J + k;
  float2* cs = sm + pl.off_cs;
  float2* w = sm + pl.off_w;
  const float2* Cch = A.C + (size_t)ch * P * p;
  const unsigned long long* turns = A.turns + (size_t)ch * P;
  auto coef_at = [&](int t, int pp) -> float2 {
    const int kk = kap0 + t;
    if (kk >= K) return cz();
    return A.coef_mode == 0 ? A.coef[((size_t)ch * A.Kc + A.kap_off + kk) * P + pp]
                            : path_coef(A.coef[(size_t)ch * P + pp], turns[pp], A.kap_off + kk);
  };
  if (A.identity_C) {                      // dense channel: C = I, p = P
    for (int idx = tid; idx < T * p; idx += nth) w[idx] = cconj(coef_at(idx / p, idx % p));
  } else {
    for (int idx = tid; idx < T * p; idx += nth) w[idx] = cz();
    for (int P0 = 0; P0 < P; P0 += kServePC) {
      const int pc = min(kServePC, P - P0);
      __syncthreads();                     // previous chunk consumed
      for (int idx = tid; idx < T * kServePC; idx += nth) {
        const int t = idx / kServePC, pp = idx % kServePC;
        cs[idx] = pp < pc ? coef_at(t, P0 + pp) : cz();
      }
      __syncthreads();
      for (int idx = tid; idx < T * p; idx += nth) {
        const int t = idx / p, q = idx - t * p;
        float2 acc = w[idx];
        const float2* crow = cs + t * kServePC;
        for (int pp = 0; pp < pc; ++pp) cmacc(acc, Cch[(size_t)(P0 + pp) * p + q], crow[pp]);
        w[idx] = acc;
      }
    }
  }
  __syncthreads();
  // rows: thread per (row a, column c), eight subcarriers at a time
  constexpr int TB = 8;
  const float2* Gch = A.G + (size_t)ch * p * m * n;
  for (int idx = tid; idx < MG * n; idx += nth) {
    const int aa = idx / n, c = idx - aa * n;
    for (int t0 = 0; t0 < T; t0 += TB) {
      float2 acc[TB];
#pragma unroll
      for (int u = 0; u < TB; ++u) acc[u] = cz();
      if (aa < m) {
        // eight independent core loads in flight per step
        const float2* g = Gch + (size_t)aa * n + c;
        const size_t qs = (size_t)m * n;
        for (int q0 = 0; q0 < p; q0 += 8) {
          float2 gv[8];
#pragma unroll
          for (int v = 0; v < 8; ++v) gv[v] = q0 + v < p ? __ldg(g + (q0 + v) * qs) : cz();
#pragma unroll
          for (int v = 0; v < 8; ++v) {
            if (q0 + v < p) {
#pragma unroll
              for (int u = 0; u < TB; ++u)
                if (t0 + u < T) cmac(acc[u], w[(t0 + u) * p + q0 + v], gv[v]);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < TB; ++u)
        if (t0 + u < T) sm[pl.off_Hs + ((t0 + u) * MG + aa) * pl.SH + c] = acc[u];
    }
  }
}

// PHASE 0: the whole precoder in one kernel.  PHASE 1 (serving channels
// from the serving pass): Gram, Jacobi and Gram-Schmidt only, the Gram
// accumulated over column chunks of H~ staged a chunk at a time, so that a
// CTA holds little shared memory and many units hide the Jacobi's latency;
// U and the eigenvalues go to workspace.  PHASE 2: the rest from the stored
// U (W = U* H~, refinement, close pairs, V~, E_kk), with H~ staged whole.
constexpr int kEigChunk = 16;   // columns of H~ per staged chunk in PHASE 1

template <int MG, int LT, int PHASE>
__global__ void __launch_bounds__(kThreads) k_svd_precoder(const SinrArgs A, const PrecoderPlan pl) {
  extern __shared__ __align__(16) float2 sm[];
  const int T = pl.T;
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int nth = blockDim.x;
  const int k = blockIdx.y;
  const int kap0 = blockIdx.x * T;
  const int kap = kap0 + g;
  const int m = A.m, n = A.n, L = A.L, K = A.K;
  float2* Hs = sm + pl.off_Hs + g * MG * pl.SH;
  float2* Ss = sm + pl.off_Ss + g * MG * pl.SS;
  float2* Us = sm + pl.off_Us + g * MG * pl.SS;
  int* sel = reinterpret_cast<int*>(sm + pl.off_sel) + g * MG;

  float2 S[MG], U[MG];
  bool converged = false;
  if (PHASE == 1) {
    // Gram over column chunks: chunk [t][row][kEigChunk + 1] in the Hs region
#pragma unroll
    for (int b = 0; b < MG; ++b) S[b] = cz();
    const int CS = kEigChunk + 1;
    float2* ch = sm + pl.off_Hs;
    for (int c0 = 0; c0 < n; c0 += kEigChunk) {
      __syncthreads();                               // previous chunk consumed
      for (int idx = tid; idx < T * MG * kEigChunk; idx += nth) {
        const int c = idx % kEigChunk, aa = (idx / kEigChunk) % MG, t = idx / (kEigChunk * MG);
        const int kk = kap0 + t;
        float2 v = cz();
        if (aa < m && kk < K && c0 + c < n)
          v = A.Hserv[(((size_t)k * A.serv_stride * K + kk) * m + aa) * n + c0 + c];
        ch[(t * MG + aa) * CS + c] = v;
      }
      __syncthreads();
      const float2* cg = ch + g * MG * CS;
#pragma unroll 4
      for (int c = 0; c < kEigChunk; ++c) {
        const float2 x = cg[a * CS + c];
#pragma unroll
        for (int b = 0; b < MG; ++b) cmacc(S[b], x, cg[b * CS + c]);
      }
    }
  }
  // H~_kk rows of the T subcarriers (zero rows for a >= m and beyond K),
  // formed here or read from the all-link rebuild of the adjoint
  if (PHASE == 1) {
  } else if (A.fuse_serve) {
    serve_channels<MG>(A, pl, k, kap0, sm);
  } else {
    for (int idx = tid; idx < T * MG * n; idx += nth) {
      const int c = idx % n, aa = (idx / n) % MG, t = idx / (n * MG);
      const int kk = kap0 + t;
      float2 v = cz();
      if (aa < m && kk < K) v = A.Hserv[(((size_t)k * A.serv_stride * K + kk) * m + aa) * n + c];
      sm[pl.off_Hs + (t * MG + aa) * pl.SH + c] = v;
    }
  }
  __syncthreads();

  // Gram S = H~ H~* (m x m, padded to MG with zero rows), row a in lane a
#pragma unroll
  for (int b = 0; b < MG; ++b) U[b] = make_float2(b == a ? 1.f : 0.f, 0.f);
  if (PHASE == 0) {
#pragma unroll
    for (int b = 0; b < MG; ++b) S[b] = cz();
    const float2* ha = Hs + a * pl.SH;
    for (int c = 0; c < n; ++c) {
      const float2 x = ha[c];
#pragma unroll
      for (int b = 0; b < MG; ++b) cmacc(S[b], x, Hs[b * pl.SH + c]);
    }
  }
  if (PHASE != 2) {

  // scale S to unit trace (eigenvectors and eigenvalue ratios are unchanged;
  // the singular values are taken from W below)
  {
    const float tr = gsum<MG>(pick(S, a).x);
    const float sc = tr > 0.f ? 1.f / tr : 1.f;
#pragma unroll
    for (int b = 0; b < MG; ++b) S[b] = cscale(S[b], sc);
  }
  // Cyclic Jacobi on S held in registers (see jacobi_step), until the
  // relative off-diagonal norm is below ~5e-7, then one more sweep: Jacobi
  // converges quadratically, so that sweep takes the off-diagonal from
  // ~5e-7 to rounding level.  Without it a pair of eigenvalues a relative
  // gap g apart keeps its eigenvectors mixed by ~5e-7 / g (up to 3e-4 in
  // the per-stream SINR for g ~ 1e-3); with it the mixing is the FP32
  // Gram's own ~u / g.  The stopping decision is taken warp-wide (extra
  // sweeps leave a converged S unchanged).
  const int max_sweeps = MG <= 8 ? 11 : 13;
  bool polish = false;
  for (int sweep = 0;; ++sweep) {
    float off = 0.f, dia = 0.f;
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      const float v = cabs2(S[b]);
      if (b == a) dia += v; else off += v;
    }
    off = gsum<MG>(off);
    dia = gsum<MG>(dia);
    converged = off <= 2.3e-13f * dia;
    const bool all = __all_sync(FULL, converged);
    if ((all && polish) || sweep == max_sweeps) break;
    polish = all;
    float dg = pick(S, a).x;
    if constexpr (MG == 16) {
      jacobi_sweep16(S, U, dg, a);
    } else {
#pragma unroll
      for (int t = 0; t < MG - 1; ++t) jacobi_step<MG>(t, S, U, dg, a);
    }
  }
  // The rotations come from hardware reciprocal square roots and each is
  // applied in FP32, so U leaves the sweeps unitary only to ~1e-7 .. 1e-6:
  // its columns drift from unit norm (the serving effective channel
  // E_kk = U_L Sigma_L below scales with them) and from each other (which
  // the close-pair rotation below would amplify by lambda / gap).  One pass
  // of modified Gram-Schmidt over the columns makes U unitary to rounding;
  // it moves each column by the size of its defect only.
  {
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      const float nb = gsum<MG>(cabs2(U[b]));
      U[b] = cscale(U[b], nb > 0.f ? 1.f / sqrtf(nb) : 1.f);
#pragma unroll
      for (int b2 = b + 1; b2 < MG; ++b2) {
        // U[:, b2] -= (U[:, b]* U[:, b2]) U[:, b]
        float2 pr = cz();
        cmacc(pr, U[b2], U[b]);                     // U_ab2 conj(U_ab)
        pr.x = gsum<MG>(pr.x);
        pr.y = gsum<MG>(pr.y);
        cms(U[b2], pr, U[b]);
      }
    }
  }
  }  // PHASE != 2
  const size_t ueig = ((size_t)k * K + (kap < K ? kap : K - 1)) * MG;
  if (PHASE == 1) {
    // U (row a in lane a), the eigenvalues and the convergence to workspace
    if (kap < K) {
#pragma unroll
      for (int b = 0; b < MG; ++b) A.Ueig[(ueig + a) * MG + b] = U[b];
      A.lam_eig[ueig + a] = pick(S, a).x;
      if (a == 0) A.conv_eig[(size_t)k * K + kap] = converged ? 1 : 0;
    }
    return;
  }
  if (PHASE == 2) {
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      U[b] = A.Ueig[(ueig + a) * MG + b];
      S[b] = cz();
    }
    add_diag(S, a, A.lam_eig[ueig + a]);                     // only the diagonal is read below
    converged = A.conv_eig[(size_t)k * K + (kap < K ? kap : K - 1)] != 0;
  }
  // The eigenvectors of the Gram are accurate unless a kept singular value is
  // small: refine with one-sided sweeps (below) when lambda_L < 1e-4 lambda_1
  // in any group of the warp.  `erank` (the eigenvalue's rank) and `lam`
  // also select the close pairs polished after them.
  bool need_refine;
  int erank;
  float lam, lmax;
  {
    lam = (a < m) ? pick(S, a).x : -INFINITY;
    lmax = lam;
#pragma unroll
    for (int o = 1; o < MG; o <<= 1) lmax = fmaxf(lmax, __shfl_xor_sync(FULL, lmax, o, MG));
    // rank of this lane's eigenvalue; the L-th largest decides
    erank = 0;
#pragma unroll
    for (int b = 0; b < MG; ++b) {
      const float lb = __shfl_sync(FULL, lam, b, MG);
      erank += (lb > lam) || (lb == lam && b < a);
    }
    const bool small_kept = (a < m) && (erank < L) && !(lam >= 1e-4f * lmax);
    need_refine = __any_sync(FULL, small_kept);
  }
#pragma unroll
  for (int b = 0; b < MG; ++b) Us[a * pl.SS + b] = U[b];
  __syncwarp();

  // W = U* H~ in place of H~ (rows ~ sigma_r v_r*), column block by block
  {
    constexpr int CW = 32 / MG;
    for (int c0 = 0; c0 < n; c0 += CW) {
      float2 hb[MG][CW];
#pragma unroll
      for (int b = 0; b < MG; ++b)
#pragma unroll
        for (int cc = 0; cc < CW; ++cc) hb[b][cc] = (c0 + cc < n) ? Hs[b * pl.SH + c0 + cc] : cz();
      __syncwarp();
#pragma unroll
      for (int cc = 0; cc < CW; ++cc) {
        float2 acc = cz();
#pragma unroll
        for (int b = 0; b < MG; ++b) cmacc(acc, hb[b][cc], Us[b * pl.SS + a]);
        if (c0 + cc < n) Hs[a * pl.SH + c0 + cc] = acc;
      }
      __syncwarp();
    }
  }
  // One-sided (Hestenes) Jacobi sweeps on the rows of W: the rotation of rows
  // (p, q) is the two-sided rotation of their 2 x 2 Gram block, now formed
  // from W itself, so small singular values keep their relative accuracy
  // (the Gram of H~ squares the condition number).  The same rotations are
  // applied to the columns of U, so that H~ = U W holds throughout.  Two
  // lanes per pair, each on half of the columns of W and half of the rows of
  // U.  Sweeps repeat (at most 3) until every pair is orthogonal to 1e-6
  // relative, decided warp-wide.
  bool refined = !need_refine;
  {
    const int j = a >> 1, half = a & 1;
    const int nh = (n + 1) >> 1;
    const int c_lo = half * nh, c_hi = min(n, c_lo + nh);
    const int r_lo = half * (MG / 2), r_hi = r_lo + MG / 2;
    for (int sweep = 0; sweep < (need_refine ? 3 : 0); ++sweep) {
      float worst = 0.f;
#pragma unroll 1
      for (int step = 0; step < MG - 1; ++step) {
        int pp, qq;
        if (j == 0) { pp = step; qq = MG - 1; }
        else { pp = (step + j) % (MG - 1); qq = (step - j + MG - 1) % (MG - 1); }
        float al = 0.f, be = 0.f;
        float2 ga = cz();
        for (int c = c_lo; c < c_hi; ++c) {
          const float2 x = Hs[pp * pl.SH + c], y = Hs[qq * pl.SH + c];
          al += cabs2(x);
          be += cabs2(y);
          cmacc(ga, x, y);
        }
        al += __shfl_xor_sync(FULL, al, 1, MG);
        be += __shfl_xor_sync(FULL, be, 1, MG);
        ga.x += __shfl_xor_sync(FULL, ga.x, 1, MG);
        ga.y += __shfl_xor_sync(FULL, ga.y, 1, MG);
        const float g2 = cabs2(ga);
        if (al > 0.f && be > 0.f) worst = fmaxf(worst, g2 / (al * be));
        const float ab = sqrtf(g2);
        if (ab > 1e-30f && ab > 1e-9f * sqrtf(al * be)) {
          const float tau = (be - al) / (2.f * ab);
          const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
          const float cr = 1.f / sqrtf(fmaf(t, t, 1.f));
          const float sr = t * cr;
          const float2 e = cscale(ga, 1.f / ab);
          const float2 se = cscale(e, sr), sec = cscale(cconj(e), sr);
          for (int c = c_lo; c < c_hi; ++c) {        // W <- J* W (rows p, q)
            const float2 x = Hs[pp * pl.SH + c], y = Hs[qq * pl.SH + c];
            float2 nx = cscale(x, cr), ny = cscale(y, cr);
            cms(nx, se, y);                          // c x - s e y
            cmac(ny, sec, x);                        // s conj(e) x + c y
            Hs[pp * pl.SH + c] = nx;
            Hs[qq * pl.SH + c] = ny;
          }
          for (int r = r_lo; r < r_hi; ++r) {        // U <- U J (columns p, q)
            const float2 x = Us[r * pl.SS + pp], y = Us[r * pl.SS + qq];
            float2 nx = cscale(x, cr), ny = cscale(y, cr);
            cms(nx, sec, y);                         // c x - s conj(e) y
            cmac(ny, se, x);                         // s e x + c y
            Us[r * pl.SS + pp] = nx;
            Us[r * pl.SS + qq] = ny;
          }
        }
        __syncwarp();
      }
      worst = fmaxf(worst, __shfl_xor_sync(FULL, worst, 1, MG));
#pragma unroll
      for (int o = 2; o < MG; o <<= 1) worst = fmaxf(worst, __shfl_xor_sync(FULL, worst, o, MG));
      refined = worst <= 1e-12f;
      if (__all_sync(FULL, refined)) break;
    }
  }

  // Close pairs.  Two eigenvalues of rank r and r + 1 (r < L) within
  // kPolishWindow lambda_1 of each other are mixed by the Gram's FP32
  // rounding by about u lambda_1 / (lambda_r - lambda_r+1), and the
  // per-stream SINRs follow that mixing (~0.5 per rad; ~7 u lambda_1 / gap in
  // the SINR without this step).  Each such pair of rows of W is rotated once
  // more, with the 2 x 2 Gram of the rows accumulated in double-float (the
  // rotation angle then comes with FP32 relative accuracy), so that the
  // mixing drops to what the FP32 rounding of H~ itself leaves, ~0.4 u
  // lambda_1 / gap in the SINR.  Pairs closer than kPrecoderCloseGap
  // lambda_1 (where even that exceeds ~5e-6) list the unit for the FP64
  // precoder.
  int close_mask = 0;                       // bit r: the pair (r, r + 1) is close
  {
    const int gb = (threadIdx.x & 31) / MG * MG;            // group's first lane in the warp
    const unsigned gmask = MG == 32 ? FULL : ((1u << MG) - 1u) << gb;
    for (int r = 0; r < L && r + 1 < m; ++r) {
      const unsigned bp = __ballot_sync(FULL, a < m && erank == r) & gmask;
      const unsigned bq = __ballot_sync(FULL, a < m && erank == r + 1) & gmask;
      const int pp = bp ? __ffs(bp) - 1 - gb : 0, qq = bq ? __ffs(bq) - 1 - gb : 0;
      const float lp = __shfl_sync(FULL, lam, pp, MG), lq = __shfl_sync(FULL, lam, qq, MG);
      const bool close = bp && bq && (lp - lq) < kPolishWindow * lmax;
      if (bp && bq && (lp - lq) < kPrecoderCloseGap * lmax && lq >= kPrecoderWeak * lmax)
        close_mask |= 1 << r;
      if (!__any_sync(FULL, close)) continue;
      float alh = 0.f, all = 0.f, beh = 0.f, bel = 0.f;
      float2 gah = cz(), gal = cz();
      if (close)
        for (int c = a; c < n; c += MG) {
          const float2 x = Hs[pp * pl.SH + c], y = Hs[qq * pl.SH + c];
          df_add_prod(alh, all, x.x, x.x);
          df_add_prod(alh, all, x.y, x.y);
          df_add_prod(beh, bel, y.x, y.x);
          df_add_prod(beh, bel, y.y, y.y);
          df_cmacc(gah, gal, x, y);                          // sum x conj(y)
        }
      // group sums of the double-float partials (TwoSum on the high parts)
#pragma unroll
      for (int o = 1; o < MG; o <<= 1) {
        df_add(alh, all, __shfl_xor_sync(FULL, alh, o, MG), __shfl_xor_sync(FULL, all, o, MG));
        df_add(beh, bel, __shfl_xor_sync(FULL, beh, o, MG), __shfl_xor_sync(FULL, bel, o, MG));
        df_add(gah.x, gal.x, __shfl_xor_sync(FULL, gah.x, o, MG), __shfl_xor_sync(FULL, gal.x, o, MG));
        df_add(gah.y, gal.y, __shfl_xor_sync(FULL, gah.y, o, MG), __shfl_xor_sync(FULL, gal.y, o, MG));
      }
      // be - al without cancellation (the high parts are within a factor 2
      // of each other for a close pair, so their difference is exact)
      const float dba = __fadd_rn(__fsub_rn(beh, alh), __fsub_rn(bel, all));
      const float gx = gah.x + gal.x, gy = gah.y + gal.y;
      const float ab = sqrtf(fmaf(gx, gx, gy * gy));
      const float scale = sqrtf(alh) * sqrtf(beh);
      if (close && ab > 0.f && ab > 1e-12f * scale) {
        const float tau = dba / (2.f * ab);
        const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
        const float cr = 1.f / sqrtf(fmaf(t, t, 1.f));
        const float sr = t * cr;
        const float2 e = make_float2(gx / ab, gy / ab);
        const float2 se = cscale(e, sr), sec = cscale(cconj(e), sr);
        for (int c = a; c < n; c += MG) {                    // W <- J* W (rows p, q)
          const float2 x = Hs[pp * pl.SH + c], y = Hs[qq * pl.SH + c];
          float2 nx = cscale(x, cr), ny = cscale(y, cr);
          cms(nx, se, y);
          cmac(ny, sec, x);
          Hs[pp * pl.SH + c] = nx;
          Hs[qq * pl.SH + c] = ny;
        }
        {                                                    // U <- U J (columns p, q), row a
          const float2 x = Us[a * pl.SS + pp], y = Us[a * pl.SS + qq];
          float2 nx = cscale(x, cr), ny = cscale(y, cr);
          cms(nx, sec, y);
          cmac(ny, se, x);
          Us[a * pl.SS + pp] = nx;
          Us[a * pl.SS + qq] = ny;
        }
      }
      __syncwarp();
    }
  }

  // singular values = row norms of W; order them (descending; padding last)
  float nrm2 = 0.f;
  for (int c = 0; c < n; ++c) nrm2 += cabs2(Hs[a * pl.SH + c]);
  Ss[a * pl.SS + a].x = (a < m) ? nrm2 : -INFINITY;
  __syncwarp();
  int rank = 0;
#pragma unroll
  for (int b = 0; b < MG; ++b) {
    const float lb = Ss[b * pl.SS + b].x;
    const float la = Ss[a * pl.SS + a].x;
    rank += (lb > la) || (lb == la && b < a);
  }
  __syncwarp();
  if (rank < MG) sel[rank] = a;
  __syncwarp();
  int idx[LT];
  float inv[LT];
  bool deficient = false;
#pragma unroll
  for (int r = 0; r < LT; ++r) {
    idx[r] = sel[r < MG ? r : 0];
    const float s2 = Ss[idx[r] * pl.SS + idx[r]].x;
    deficient |= (r < L) && !(s2 > 0.f);
    inv[r] = (s2 > 0.f) ? 1.f / sqrtf(s2) : 0.f;
  }

  // V~[:, r] = conj(row idx_r of W) / sigma_r; lanes stride over the columns
  if (kap < K) {
    float2* Vout = A.V + ((size_t)k * K + kap) * n * L;
    for (int c = a; c < n; c += MG) {
#pragma unroll
      for (int r = 0; r < LT; ++r)
        if (r < L) Vout[(size_t)c * L + r] = cscale(cconj(Hs[idx[r] * pl.SH + c]), inv[r]);
    }
    // serving effective channel E_kk = H~_kk V~_k = U W W* / sigma = U_L Sigma_L
    if (a < m) {
      float2* Eout = A.Eserv + (((size_t)k * K + kap) * m + a) * L;
#pragma unroll
      for (int r = 0; r < LT; ++r)
        if (r < L) {
          const float sg = Ss[idx[r] * pl.SS + idx[r]].x;
          Eout[r] = cscale(Us[a * pl.SS + idx[r]], sg > 0.f ? sqrtf(sg) : 0.f);
        }
    }
    if (a == 0)
      A.pflag[(size_t)k * K + kap] = (deficient ? TS_FLAG_RANK_DEFICIENT : 0) |
                                     ((converged || refined) ? 0 : TS_FLAG_EIG_UNCONVERGED);

    if (A.Uout != nullptr && a < m) {
      // the full SVD of H~_kk for the adjoint: lane a writes singular triplet a
      const int ia = sel[a];
      const float s2 = Ss[ia * pl.SS + ia].x;
      const float sg = s2 > 0.f ? sqrtf(s2) : 0.f, isg = s2 > 0.f ? 1.f / sg : 0.f;
      const size_t base = (size_t)k * K + kap;
      A.Sout[base * m + a] = sg;
      for (int b = 0; b < m; ++b) A.Uout[(base * m + b) * m + a] = Us[b * pl.SS + ia];
      for (int c = 0; c < n; ++c)
        A.Vmout[(base * n + c) * m + a] = cscale(cconj(Hs[ia * pl.SH + c]), isg);
    }
  }
  // a unit with a close pair: listed with its left singular vectors of ranks
  // 0 .. min(L + 1, m) - 1 for the double-float refinement
  {
    const bool lst = close_mask != 0 && A.list_close && kap < K;
    int pos = -1;
    if (lst && a == 0) pos = atomicAdd(A.rcount, 1);
    pos = __shfl_sync(FULL, pos, 0, MG);
    if (lst && pos >= 0 && pos < A.J * K) {
      const int R = min(L + 1, m);
      if (a < m)
        for (int r = 0; r < R; ++r) A.Uclose[((size_t)pos * R + r) * m + a] = Us[a * pl.SS + sel[r]];
      if (a == 0) {
        A.rlist[pos] = k * K + kap;
        A.close_mask[pos] = close_mask;
      }
    }
  }
}

// ------------------------------------------------------------------ phase 2
// k_sinr_link: one CTA per (subcarrier tile, UE i, link).  It rebuilds
// H~_ik on the T subcarriers of its tile chunk by chunk, forms E_ik and
// writes the partial covariance rows E_ik E_ik* (interfering links) or E_ii
// itself (the serving link of the wideband-precoder variant) to workspace.
// Shared memory plan (float2 units): C_ik, the coefficient tile or path
// form, two stage buffers (core chunk or wideband fold, precoder chunk), the
// projection ws; the per-group scratch Es reuses the stage buffers.
struct LinkPlan {
  int T, NC, SG, SV, SF, ES, wstride, wide;
  int off_Cs, off_cs, off_pa, off_pt, off_ws, off_stage, stage, off_Gs, off_Vs, off_Es, total;
};

__host__ __device__ inline LinkPlan link_plan(int MG, int LT, int T, int NC, int P, int p, int mode) {
  const bool svd = mode != 1;            // chunked modes (svd, serve, rebuild)
  LinkPlan pl;
  pl.T = T;
  pl.NC = NC;
  pl.SG = NC + 2;
  pl.SV = NC * LT + 2;
  pl.SF = LT + 2;
  pl.ES = MG * LT + 2;
  pl.wstride = p + 1;
  pl.wide = 0;
  int o = 0;
  pl.off_Cs = o; o += P * p;
  pl.off_cs = o; o += T * P;
  pl.off_pa = o; o += P;
  pl.off_pt = o; o += P;
  pl.off_ws = o; o += T * pl.wstride;
  o = (o + 1) & ~1;
  pl.off_stage = o;
  int so = 0;
  pl.off_Gs = so; so += svd ? p * MG * pl.SG : p * MG * pl.SF;
  so = (so + 1) & ~1;
  pl.off_Vs = so; if (mode == 0) so += T * pl.SV;
  so = (so + 1) & ~1;
  pl.stage = so;
  const int nbuf = svd ? 2 : 1;
  const int es = T * pl.ES;
  o += (nbuf * so > es ? nbuf * so : es);
  pl.off_Es = pl.off_stage;
  pl.total = o;
  return pl;
}

// Modes of k_sinr_link.
constexpr int kModeSvd = 0;     // interfering link, E = H~ V~ (SVD precoders)
constexpr int kModeFold = 1;    // any link, E = sum_q w_q F[q] (wideband precoder)
constexpr int kModeServe = 2;   // serving links (large cores): write H~_kk rows
constexpr int kModeRebuild = 3; // every link (adjoint): write H~_ik rows

template <int MG, int LT, int NC, int MODE>
__global__ void __launch_bounds__(kThreads) k_sinr_link(const SinrArgs A, const LinkPlan pl) {
  constexpr bool CHUNKED = MODE != kModeFold;
  extern __shared__ __align__(16) float2 sm[];
  const int T = pl.T;
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int nth = blockDim.x;
  const int i = blockIdx.y;
  const int z = blockIdx.z;
  const int kap0 = blockIdx.x * T;
  const int kap = kap0 + g;
  const int J = A.J, m = A.m, n = A.n, p = A.p, L = A.L, K = A.K, P = A.P;
  // svd: z enumerates the interfering links; fold and rebuild: z is the BS
  // index; serve: the serving link
  const int k = MODE == kModeSvd ? (z < i ? z : z + 1) : MODE == kModeServe ? i : z;
  const int ch = i * J + k;
  const int nchunk = CHUNKED ? (n + NC - 1) / NC : 1;
  // the refinement list of the finalize kernel that follows starts empty
  if (MODE != kModeRebuild && A.rcount != nullptr && tid == 0 && blockIdx.x == 0 && i == 0 && z == 0)
    *A.rcount = 0;
  float2* Cs = sm + pl.off_Cs;
  float2* cs = sm + pl.off_cs;
  float2* ws = sm + pl.off_ws;
  float2* stage0 = sm + pl.off_stage;
  const float2* wrow = ws + g * pl.wstride;

  // Staging of one column chunk: G_ik[:, 0..m, c0 .. c0+NC) and (svd) the
  // precoder rows V_k(kappa)[c0 .. c0+NC][0..L) of the tile.  With even n and
  // L (and 16-byte aligned arrays) the copies move complex pairs; each thread
  // walks fixed positions with constant strides.
  const bool wide = pl.wide != 0;
  auto issue_chunk = [&](int cidx) {
    float2* buf = stage0 + (cidx & 1) * pl.stage;
    const int c0 = cidx * NC;
    const float2* Gch = A.G + (size_t)ch * p * m * n;
    if (wide) {
      constexpr int GU = MG * NC / 2;                 // 16-byte units per q slab
      const int cc = 2 * (tid % (NC / 2)), aa = (tid / (NC / 2)) % MG;
      const bool rowok = aa < m && c0 + cc < n;
      const float2* src = Gch + ((size_t)(tid / GU) * m + aa) * n + c0 + cc;
      float2* dst = buf + pl.off_Gs + ((tid / GU) * MG + aa) * pl.SG + cc;
      const size_t sstep = (size_t)(kThreads / GU) * m * n;
      const int dstep = (kThreads / GU) * MG * pl.SG;
      for (int q = tid / GU; q < p; q += kThreads / GU, src += sstep, dst += dstep)
        cp_async16(dst, rowok ? src : A.G, rowok);
      if (MODE == kModeSvd) {
        constexpr int VU = NC * LT / 2;               // 16-byte units per subcarrier
        const int l = 2 * (tid % (LT / 2)), vc = (tid / (LT / 2)) % NC;
        const int t0 = tid / VU;
        const bool colok = c0 + vc < n && l < L;
        for (int t = t0; t < T; t += kThreads / VU) {
          const bool ok = colok && kap0 + t < K;
          cp_async16(buf + pl.off_Vs + t * pl.SV + vc * LT + l,
                     ok ? A.V + (((size_t)k * K + kap0 + t) * n + c0 + vc) * L + l : A.V, ok);
        }
      }
      return;
    }
    for (int idx = tid; idx < p * MG * NC; idx += nth) {
      const int cc = idx % NC, aa = (idx / NC) % MG, q = idx / (NC * MG);
      const int c = c0 + cc;
      const bool ok = aa < m && c < n;
      cp_async8(buf + pl.off_Gs + (q * MG + aa) * pl.SG + cc,
                ok ? Gch + ((size_t)q * m + aa) * n + c : A.G, ok);
    }
    if (MODE == kModeSvd) {
      for (int idx = tid; idx < T * NC * LT; idx += nth) {
        const int l = idx % LT, cc = (idx / LT) % NC, t = idx / (LT * NC);
        const int kk2 = kap0 + t, c = c0 + cc;
        const bool ok = kk2 < K && c < n && l < L;
        cp_async8(buf + pl.off_Vs + t * pl.SV + cc * LT + l,
                  ok ? A.V + (((size_t)k * K + kk2) * n + c) * L + l : A.V, ok);
      }
    }
  };

  // group 0: C_ik, the coefficients of the tile and chunk 0 (or the fold)
  if (!A.identity_C)
    for (int idx = tid; idx < P * p; idx += nth)
      cp_async8(Cs + idx, A.C + (size_t)ch * P * p + idx, true);
  if (A.coef_mode == 0) {
    for (int idx = tid; idx < T * P; idx += nth) {
      const int t = idx / P, pp = idx - t * P;
      const bool ok = kap0 + t < K;
      cp_async8(cs + idx, ok ? A.coef + ((size_t)ch * A.Kc + A.kap_off + kap0 + t) * P + pp : A.coef, ok);
    }
  } else {
    for (int idx = tid; idx < P; idx += nth) {
      cp_async8(sm + pl.off_pa + idx, A.coef + (size_t)ch * P + idx, true);
      cp_async8(sm + pl.off_pt + idx, A.turns + (size_t)ch * P + idx, true);
    }
  }
  if (CHUNKED) {
    issue_chunk(0);
  } else {
    const float2* Fch = A.F + (size_t)ch * p * m * L;
    for (int idx = tid; idx < p * MG * LT; idx += nth) {
      const int l = idx % LT, aa = (idx / LT) % MG, q = idx / (LT * MG);
      const bool ok = aa < m && l < L;
      cp_async8(stage0 + pl.off_Gs + (q * MG + aa) * pl.SF + l,
                ok ? Fch + ((size_t)q * m + aa) * L + l : A.F, ok);
    }
  }
  cp_async_commit();
  if (CHUNKED && nchunk > 1) issue_chunk(1);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();

  // projection w = c* C for the T subcarriers (eq. 15)
  if (A.coef_mode != 0) {
    const float2* pa = sm + pl.off_pa;
    const unsigned long long* pt = reinterpret_cast<const unsigned long long*>(sm + pl.off_pt);
    for (int idx = tid; idx < T * P; idx += nth) {
      const int t = idx / P, pp = idx - t * P;
      cs[idx] = (kap0 + t < K) ? path_coef(pa[pp], pt[pp], A.kap_off + kap0 + t) : cz();
    }
    __syncthreads();
  }
  for (int idx = tid; idx < T * p; idx += nth) {
    const int t = idx / p, q = idx - t * p;
    float2 acc = cz();
    const float2* crow = cs + t * P;
    if (A.identity_C)
      acc = cconj(crow[q]);            // dense channel: C = I, p = P
    else
      for (int pp = 0; pp < P; ++pp) cmacc(acc, Cs[pp * p + q], crow[pp]);
    ws[t * pl.wstride + q] = acc;
  }
  __syncthreads();

  float2 E[LT];   // row a of E_ik
#pragma unroll
  for (int l = 0; l < LT; ++l) E[l] = cz();
  float2* Hrow = nullptr;
  if (MODE == kModeServe)
    Hrow = A.Hserv + (((size_t)i * K + (kap < K ? kap : 0)) * m + (a < m ? a : 0)) * n;
  if (MODE == kModeRebuild)
    Hrow = A.Hserv + (((size_t)ch * K + (kap < K ? kap : 0)) * m + (a < m ? a : 0)) * n;
  const bool hvalid = kap < K && a < m;
  if (CHUNKED) {
    for (int cidx = 0; cidx < nchunk; ++cidx) {
      if (cidx > 0) {
        if (cidx + 1 < nchunk) issue_chunk(cidx + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
      }
      const float2* buf = stage0 + (cidx & 1) * pl.stage;
      float2 h[NC];
      core_chunk<NC>(wrow, buf + pl.off_Gs, pl.SG, MG, a, p, h);
      if (MODE == kModeServe || MODE == kModeRebuild) {
        const int c0 = cidx * NC;
        if (hvalid) {
#pragma unroll
          for (int cc = 0; cc < NC; ++cc)
            if (c0 + cc < n) Hrow[c0 + cc] = h[cc];
        }
      } else {
        const float2* vrow = buf + pl.off_Vs + g * pl.SV;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
          for (int l2 = 0; l2 < LT / 2; ++l2) {
            const float4 v = reinterpret_cast<const float4*>(vrow + cc * LT)[l2];
            cmac(E[2 * l2], h[cc], make_float2(v.x, v.y));
            cmac(E[2 * l2 + 1], h[cc], make_float2(v.z, v.w));
          }
        }
      }
      __syncthreads();   // this buffer is refilled two chunks later
    }
  } else {
    const float2* Fs = stage0 + pl.off_Gs;
#pragma unroll 4
    for (int q = 0; q < p; ++q) {
      const float2 w = wrow[q];
      const float4* f4 = reinterpret_cast<const float4*>(Fs + (q * MG + a) * pl.SF);
#pragma unroll
      for (int l2 = 0; l2 < LT / 2; ++l2) {
        const float4 f = f4[l2];
        cmac(E[2 * l2], w, make_float2(f.x, f.y));
        cmac(E[2 * l2 + 1], w, make_float2(f.z, f.w));
      }
    }
    __syncthreads();     // Es below reuses the stage buffer
  }
  cp_async_wait<0>();

  if (MODE == kModeServe || MODE == kModeRebuild || !hvalid) return;   // nothing below for them
  if (MODE == kModeFold && k == i) {
    // serving effective channel of the wideband-precoder variant
    float2* Eout = A.Eserv + (((size_t)i * K + kap) * m + a) * L;
#pragma unroll
    for (int l = 0; l < LT; ++l)
      if (l < L) Eout[l] = E[l];
    return;
  }
  // row a of the interfering effective channel E_ik (eq. 24); the
  // finalisation forms the covariance of eq. (25) from all of them
  const int slot = MODE == kModeSvd ? z : (z < i ? z : z - 1);
  float2* Eout = A.Eint + ((((size_t)i * (J - 1) + slot) * K + kap) * m + a) * L;
#pragma unroll
  for (int l = 0; l < LT; ++l)
    if (l < L) Eout[l] = E[l];
}

// SINR of one unit from row a of R = interference + noise (padding rows set
// to the identity) and row a of E_ii, with the same arithmetic everywhere it
// is needed (forward and adjoint).  With Q~ = R + E_ii E_ii* (eq. 25):
//   a_r = e_r* Q~^{-1} e_r = |L_Q^{-1} e_r|^2   (as[r], every lane)
//   x_r = [(I + Z*Z)^{-1}]_rr, Z = L_R^{-1} E_ii   (xs[r], every lane)
// and SINR_r = a_r / x_r (eq. 5).  Returns Lq = chol(Q~) row a,
// Zq = L_Q^{-1} E_ii row a and Z = L_R^{-1} E_ii row a; false if a
// factorisation failed.  R is destroyed
// (it holds chol(R) on return); Es is the group's MG x LT shared scratch.
template <int MG, int LT>
__device__ __forceinline__ bool sinr_core(float2 (&R)[MG], const float2 (&Eself)[LT], float2* Es,
                                          int a, float2 (&Lq)[MG], float2 (&Zq)[LT],
                                          float (&as)[LT], float (&xs)[LT], float2 (&Z)[LT]) {
  // Q~ = R + E_ii E_ii*
#pragma unroll
  for (int l = 0; l < LT; ++l) Es[a * LT + l] = Eself[l];
  __syncwarp();
#pragma unroll
  for (int b = 0; b < MG; ++b) {
    Lq[b] = R[b];
#pragma unroll
    for (int l = 0; l < LT; ++l) cmacc(Lq[b], Eself[l], Es[b * LT + l]);
  }
  __syncwarp();

  bool ok = chol_rows<MG, MG>(R, a);
  ok = chol_rows<MG, MG>(Lq, a) && ok;
#pragma unroll
  for (int l = 0; l < LT; ++l) Z[l] = Zq[l] = Eself[l];
  trsv_rows<MG, MG, LT>(R, Z, a);
  trsv_rows<MG, MG, LT>(Lq, Zq, a);

#pragma unroll
  for (int l = 0; l < LT; ++l) as[l] = gsum<MG>(cabs2(Zq[l]));

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
#pragma unroll
  for (int s = 0; s < LT; ++s) xs[s] = gsum<MG>(a < LT ? cabs2(X[s]) : 0.f);
  return ok;
}

// Blocked variant of the interfering-link SVD pass (k_sinr_link, svd mode),
// for MG >= 4.  A group of GL = MG/2 lanes evaluates two subcarriers and lane
// j owns rows j and j + GL of both, so every core element read from shared
// memory feeds two subcarriers and every precoder element two rows (a 128-bit
// shared load costs four wavefronts per warp whether or not lanes share
// addresses, so reuse has to happen in registers).  128 threads, T = 512/MG
// subcarriers per CTA, column chunks of NC = 4.  Path-form coefficients are
// evaluated inside the projection, so only dense coefficients are staged.
// SERVE: the serving links instead (grid z = 1), writing the rows of H~_kk
// to workspace for the precoder (no precoders, no E).
template <int MG, int LT, bool SERVE>
__global__ void __launch_bounds__(kThreads) k_sinr_link_blk(const SinrArgs A, const LinkPlan pl) {
  constexpr int NC = 4;
  constexpr int GL = MG / 2;
  constexpr int T = 2 * kThreads / GL;
  constexpr int QS = kThreads / T;          // threads per subcarrier in the projection
  constexpr int QA = 32 / QS;               // projection accumulators per thread (p <= 32)
  extern __shared__ __align__(16) float2 sm[];
  const int tid = threadIdx.x;
  const int gp = tid / GL, j = tid % GL;
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * T;
  const int J = A.J, m = A.m, n = A.n, p = A.p, L = A.L, K = A.K, P = A.P;
  const int k = SERVE ? i : (z < i ? z : z + 1);
  const int ch = i * J + k;
  const int nchunk = (n + NC - 1) / NC;
  float2* Cs = sm + pl.off_Cs;
  float2* cs = sm + pl.off_cs;
  float2* ws = sm + pl.off_ws;
  float2* stage0 = sm + pl.off_stage;
  const bool wide = pl.wide != 0;
  // the refinement list of the finalize kernel that follows starts empty
  if (!SERVE && A.rcount != nullptr && tid == 0 && blockIdx.x == 0 && i == 0 && z == 0) *A.rcount = 0;

  auto issue_chunk = [&](int cidx) {
    float2* buf = stage0 + (cidx & 1) * pl.stage;
    const int c0 = cidx * NC;
    const float2* Gch = A.G + (size_t)ch * p * m * n;
    if (wide) {
      constexpr int GU = MG * NC / 2;
      const int cc = 2 * (tid % (NC / 2)), aa = (tid / (NC / 2)) % MG;
      const bool rowok = aa < m && c0 + cc < n;
      const float2* src = Gch + ((size_t)(tid / GU) * m + aa) * n + c0 + cc;
      float2* dst = buf + pl.off_Gs + ((tid / GU) * MG + aa) * pl.SG + cc;
      const size_t sstep = (size_t)(kThreads / GU) * m * n;
      const int dstep = (kThreads / GU) * MG * pl.SG;
      for (int q = tid / GU; q < p; q += kThreads / GU, src += sstep, dst += dstep)
        cp_async16(dst, rowok ? src : A.G, rowok);
      if (SERVE) return;
      constexpr int VU = NC * LT / 2;
      const int l = 2 * (tid % (LT / 2)), vc = (tid / (LT / 2)) % NC;
      const bool colok = c0 + vc < n && l < L;
      for (int t = tid / VU; t < T; t += kThreads / VU) {
        const bool ok = colok && kap0 + t < K;
        cp_async16(buf + pl.off_Vs + t * pl.SV + vc * LT + l,
                   ok ? A.V + (((size_t)k * K + kap0 + t) * n + c0 + vc) * L + l : A.V, ok);
      }
      return;
    }
    for (int idx = tid; idx < p * MG * NC; idx += kThreads) {
      const int cc = idx % NC, aa = (idx / NC) % MG, q = idx / (NC * MG);
      const int c = c0 + cc;
      const bool ok = aa < m && c < n;
      cp_async8(buf + pl.off_Gs + (q * MG + aa) * pl.SG + cc,
                ok ? Gch + ((size_t)q * m + aa) * n + c : A.G, ok);
    }
    if (SERVE) return;
    for (int idx = tid; idx < T * NC * LT; idx += kThreads) {
      const int l = idx % LT, cc = (idx / LT) % NC, t = idx / (LT * NC);
      const int kk2 = kap0 + t, c = c0 + cc;
      const bool ok = kk2 < K && c < n && l < L;
      cp_async8(buf + pl.off_Vs + t * pl.SV + cc * LT + l,
                ok ? A.V + (((size_t)k * K + kk2) * n + c) * L + l : A.V, ok);
    }
  };

  // group 0: C_ik, the coefficients (dense tile, or the path form) and chunk 0
  if (!A.identity_C)
    for (int idx = tid; idx < P * p; idx += kThreads)
      cp_async8(Cs + idx, A.C + (size_t)ch * P * p + idx, true);
  if (A.coef_mode == 0) {
    for (int idx = tid; idx < T * P; idx += kThreads) {
      const int t = idx / P, pp = idx - t * P;
      const bool ok = kap0 + t < K;
      cp_async8(cs + idx, ok ? A.coef + ((size_t)ch * A.Kc + A.kap_off + kap0 + t) * P + pp : A.coef, ok);
    }
  } else {
    for (int idx = tid; idx < P; idx += kThreads) {
      cp_async8(sm + pl.off_pa + idx, A.coef + (size_t)ch * P + idx, true);
      cp_async8(sm + pl.off_pt + idx, A.turns + (size_t)ch * P + idx, true);
    }
  }
  issue_chunk(0);
  cp_async_commit();
  if (nchunk > 1) issue_chunk(1);
  cp_async_commit();
  cp_async_wait<1>();
  __syncthreads();

  // projection w[t][q] = sum_P C[P][q] conj(c_P(kappa_t)) (eq. 15): QS threads
  // (consecutive lanes) per subcarrier, thread qs handles q = qs, qs + QS, ...
  // and evaluates the coefficient of every QS-th path, shared by shuffles
  {
    const int t = tid / QS, qs = tid % QS;
    const int kap_t = kap0 + t;
    float2 acc[QA];
#pragma unroll
    for (int u = 0; u < QA; ++u) acc[u] = cz();
    const float2* pa = sm + pl.off_pa;
    const unsigned long long* pt = reinterpret_cast<const unsigned long long*>(sm + pl.off_pt);
    for (int p0 = 0; p0 < P; p0 += QS) {
      float2 mine = cz();
      const int pm = p0 + qs;
      if (kap_t < K && pm < P)
        mine = A.coef_mode == 0 ? cs[t * P + pm] : path_coef(pa[pm], pt[pm], A.kap_off + kap_t);
#pragma unroll
      for (int r = 0; r < QS; ++r) {
        const int pp = p0 + r;
        float2 c = mine;
        if (QS > 1) c = gshfl<QS>(mine, r);
        if (pp >= P) break;                          // uniform over the warp
        if (A.identity_C) {
#pragma unroll
          for (int u = 0; u < QA; ++u)
            if (qs + u * QS == pp) acc[u] = cconj(c);
        } else {
          const float2* crow = Cs + pp * p;
#pragma unroll
          for (int u = 0; u < QA; ++u) {
            if (u * QS >= p) break;                  // uniform over the warp
            if (qs + u * QS < p) cmacc(acc[u], crow[qs + u * QS], c);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < QA; ++u)
      if (qs + u * QS < p) ws[t * pl.wstride + qs + u * QS] = acc[u];
  }
  __syncthreads();

  float2 E[2][2][LT];   // [subcarrier of the pair][row j, j + GL][stream]
#pragma unroll
  for (int x = 0; x < 2; ++x)
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int l = 0; l < LT; ++l) E[x][r][l] = cz();
  const float2* w0 = ws + (2 * gp) * pl.wstride;
  const float2* w1 = w0 + pl.wstride;
  for (int cidx = 0; cidx < nchunk; ++cidx) {
    if (cidx > 0) {
      if (cidx + 1 < nchunk) issue_chunk(cidx + 1);
      cp_async_commit();
      cp_async_wait<1>();
      __syncthreads();
    }
    const float2* buf = stage0 + (cidx & 1) * pl.stage;
    float2 h[2][2][NC];
#pragma unroll
    for (int x = 0; x < 2; ++x)
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) h[x][r][cc] = cz();
    const float2* g0 = buf + pl.off_Gs + j * pl.SG;
    const float2* g1 = g0 + GL * pl.SG;
#pragma unroll 4
    for (int q = 0; q < p; ++q) {
      const float2 wa = w0[q], wb = w1[q];
      const float4* ga = reinterpret_cast<const float4*>(g0 + q * MG * pl.SG);
      const float4* gb = reinterpret_cast<const float4*>(g1 + q * MG * pl.SG);
#pragma unroll
      for (int c2 = 0; c2 < NC / 2; ++c2) {
        const float4 u = ga[c2], v = gb[c2];
        const float2 u0 = make_float2(u.x, u.y), u1 = make_float2(u.z, u.w);
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
        cmac(h[0][0][2 * c2], wa, u0);
        cmac(h[0][0][2 * c2 + 1], wa, u1);
        cmac(h[1][0][2 * c2], wb, u0);
        cmac(h[1][0][2 * c2 + 1], wb, u1);
        cmac(h[0][1][2 * c2], wa, v0);
        cmac(h[0][1][2 * c2 + 1], wa, v1);
        cmac(h[1][1][2 * c2], wb, v0);
        cmac(h[1][1][2 * c2 + 1], wb, v1);
      }
    }
    if (SERVE) {
      // rows j and j + GL of H~_kk for both subcarriers, NC columns each
      const int c0 = cidx * NC;
#pragma unroll
      for (int x = 0; x < 2; ++x) {
        const int kap = kap0 + 2 * gp + x;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int a = j + r * GL;
          if (kap >= K || a >= m) continue;
          float2* Hrow = A.Hserv + (((size_t)i * K + kap) * m + a) * n;
#pragma unroll
          for (int cc = 0; cc < NC; ++cc)
            if (c0 + cc < n) Hrow[c0 + cc] = h[x][r][cc];
        }
      }
      __syncthreads();   // this buffer is refilled two chunks later
      continue;
    }
    const float2* va = buf + pl.off_Vs + (2 * gp) * pl.SV;
    const float2* vb = va + pl.SV;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
      for (int l2 = 0; l2 < LT / 2; ++l2) {
        const float4 x = reinterpret_cast<const float4*>(va + cc * LT)[l2];
        const float4 y = reinterpret_cast<const float4*>(vb + cc * LT)[l2];
        const float2 x0 = make_float2(x.x, x.y), x1 = make_float2(x.z, x.w);
        const float2 y0 = make_float2(y.x, y.y), y1 = make_float2(y.z, y.w);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          cmac(E[0][r][2 * l2], h[0][r][cc], x0);
          cmac(E[0][r][2 * l2 + 1], h[0][r][cc], x1);
          cmac(E[1][r][2 * l2], h[1][r][cc], y0);
          cmac(E[1][r][2 * l2 + 1], h[1][r][cc], y1);
        }
      }
    }
    __syncthreads();   // this buffer is refilled two chunks later
  }
  cp_async_wait<0>();
  if (SERVE) return;

  // rows j and j + GL of the interfering effective channel E_ik (eq. 24) for
  // both subcarriers; the finalisation forms the covariance of eq. (25)
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    const int kap = kap0 + 2 * gp + x;
    if (kap >= K) continue;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int a = j + r * GL;
      if (a >= m) continue;
      float2* Eout = A.Eint + ((((size_t)i * (J - 1) + z) * K + kap) * m + a) * L;
#pragma unroll
      for (int l = 0; l < LT; ++l)
        if (l < L) Eout[l] = E[x][r][l];
    }
  }
}

// k_sinr_finalize: one group of MG lanes per (UE i, subcarrier): sums the
// partial covariances, adds the noise (eq. 25) and evaluates the SINR.
template <int MG, int LT, bool SVD>
__global__ void __launch_bounds__(kThreads) k_sinr_finalize(const SinrArgs A, int T) {
  constexpr int kEsHalf = kThreads * LT + (kThreads / 2) * 2;
  __shared__ __align__(16) float2 sm_es[2 * kEsHalf];
  const int tid = threadIdx.x, g = tid / MG, a = tid % MG;
  const int i = blockIdx.y;
  const int kap = blockIdx.x * T + g;
  const int J = A.J, m = A.m, L = A.L, K = A.K;
  const int kc = kap < K ? kap : K - 1;     // tail groups recompute the last subcarrier
  float2* Es = sm_es + g * (MG * LT + 2);

  // R = sum_{k != i} E_ik E_ik* (eq. 25 without the serving term): the
  // rows of each interfering effective channel through the group's scratch,
  // two buffers, the next link's rows copied (cp.async) while the current
  // one is accumulated; rows a >= m and streams l >= L stay zero
  float2 R[MG], Eself[LT];
#pragma unroll
  for (int b = 0; b < MG; ++b) R[b] = cz();
#pragma unroll
  for (int l = 0; l < LT; ++l) {
    Es[a * LT + l] = cz();
    Es[kEsHalf + a * LT + l] = cz();
  }
  __syncwarp();
  auto fetch = [&](int s) {
    if (a < m) {
      const float2* Ein = A.Eint + ((((size_t)i * (J - 1) + s) * K + kc) * m + a) * L;
      float2* dst = Es + (s & 1) * kEsHalf + a * LT;
      for (int l = 0; l < L; ++l) cp_async8(dst + l, Ein + l, true);
    }
    cp_async_commit();
  };
  if (J > 1) fetch(0);
  for (int s = 0; s < J - 1; ++s) {
    if (s + 1 < J - 1) {
      fetch(s + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const float2* Eb = Es + (s & 1) * kEsHalf;
    float2 Er[LT];
#pragma unroll
    for (int l2 = 0; l2 < LT / 2; ++l2) {
      const float4 e = reinterpret_cast<const float4*>(Eb + a * LT)[l2];
      Er[2 * l2] = make_float2(e.x, e.y);
      Er[2 * l2 + 1] = make_float2(e.z, e.w);
    }
#pragma unroll
    for (int b = 0; b < MG; ++b) {
#pragma unroll
      for (int l2 = 0; l2 < LT / 2; ++l2) {
        const float4 e = reinterpret_cast<const float4*>(Eb + b * LT)[l2];
        cmacc(R[b], Er[2 * l2], make_float2(e.x, e.y));
        cmacc(R[b], Er[2 * l2 + 1], make_float2(e.z, e.w));
      }
    }
    __syncwarp();                                 // buffer read before fetch(s + 2) refills it
  }
  // serving effective channel E_ii (eq. 24), from the precoder phase (svd)
  // or from the serving-link pass of k_sinr_link (wideband precoder)
  {
    const float2* Ein = A.Eserv + (((size_t)i * K + kc) * m + (a < m ? a : 0)) * L;
#pragma unroll
    for (int l = 0; l < LT; ++l) Eself[l] = (a < m && l < L) ? Ein[l] : cz();
  }

  // noise on the m x m block, identity on the padding rows (eq. 25)
  add_diag(R, a, a < m ? A.sigma2[i] : 1.f);
  float Ra2[MG];                                  // |R_ab|^2, for the listing below
#pragma unroll
  for (int b = 0; b < MG; ++b) Ra2[b] = (a < m && b < m) ? cabs2(R[b]) : 0.f;
  float2 Lq[MG], Zq[LT], Zr[LT];
  float as[LT], xs[LT];
  const bool ok = sinr_core<MG, LT>(R, Eself, Es, a, Lq, Zq, as, xs, Zr);
  // Units whose SINRs are sensitive to the FP32 rounding of R are listed for
  // the refinement pass.  To first order SINR_r moves with y_r* dR y_r, where
  // y_r = R^{-1} e_r and e_r* y_r is its scale; the rounding of R perturbs
  // each entry by ~u |R_ab| with uncorrelated signs, so the estimate is
  //   s = max_r sqrt(sum_ab |y_ar|^2 |R_ab|^2 |y_br|^2) / (e_r* y_r)
  // and the relative error is a few u s (at most ~5 u s on the channel
  // models tried: s ~ 1 for the compressed workloads, 1e2 .. 2e2 for
  // low-rank interference on a small noise floor).  Listed when s exceeds
  // the threshold.
  if (A.rlist != nullptr) {
    float2 Y[LT];
#pragma unroll
    for (int l = 0; l < LT; ++l) Y[l] = Zr[l];      // L_R^{-1} E_ii from sinr_core
    trsv_rows_conjT<MG, MG, LT>(R, Y, a);           // Y = R^{-1} E_ii (R holds chol(R) here)
    float sens = 0.f;
#pragma unroll
    for (int l = 0; l < LT; ++l) {
      const float y2 = a < m ? cabs2(Y[l]) : 0.f;
      float t = 0.f;                                // sum_b |R_ab|^2 |y_br|^2
#pragma unroll
      for (int b = 0; b < MG; ++b) t = fmaf(Ra2[b], __shfl_sync(FULL, y2, b, MG), t);
      const float num = gsum<MG>(y2 * t);
      const float den = gsum<MG>(fmaf(Eself[l].x, Y[l].x, Eself[l].y * Y[l].y));
      if (l < L && den > 0.f) sens = fmaxf(sens, sqrtf(num) / den);
    }
    if (ok && kap < K && a == 0 && !(sens <= A.refine_sens)) {
      const int pos = atomicAdd(A.rcount, 1);
      if (pos < A.J * K) A.rlist[pos] = i * K + kap;
    }
  }

  if (kap < K) {
    uint8_t pf = 0;
    if (SVD)
      for (int k = 0; k < J; ++k) pf |= A.pflag[(size_t)k * K + kap];
    const float num = pickf(as, a), den = pickf(xs, a);
    const bool valid = ok && !(pf & TS_FLAG_TIMEOUT);
    const float sv = valid ? num / den : __int_as_float(0x7fc00000);
    if (a < L) A.sinr[((size_t)i * K + kap) * L + a] = sv;
    if (A.flags != nullptr && a == 0) {
      uint8_t f = ok ? 0 : TS_FLAG_NOT_PD;
      if (valid && !isfinite(sv)) f |= TS_FLAG_NONFINITE;
      A.flags[(size_t)i * K + kap] = f | pf;
    }
  }
}

template <int MG, int LT>
cudaError_t run_precoder(const SinrArgs& A, cudaStream_t s) {
  // groups per CTA: 128 / MG, halved while the CTA needs more than 28 KB of
  // shared memory (eight CTAs per SM), keeping whole warps for the group
  // shuffles and votes
  int T = kThreads / MG;
  const bool fused = A.fuse_serve != 0;
  PrecoderPlan pl = precoder_plan(MG, T, A.n, A.p, fused);
  while (T * MG > 32 && (size_t)pl.total * sizeof(float2) > 28 * 1024) {
    T /= 2;
    pl = precoder_plan(MG, T, A.n, A.p, fused);
  }
  for (int sp = 0; sp < A.precoder_split && T * MG > 32; ++sp) {
    T /= 2;
    pl = precoder_plan(MG, T, A.n, A.p, fused);
  }
  const size_t smem = (size_t)pl.total * sizeof(float2);
  // serving channels too wide to stage per group (n up to 1024, read from
  // the serving pass's workspace): the shared-memory precoder
  if (smem > kSmemBudget) return fused ? cudaErrorInvalidValue : launch_precoder_staged(A, s);
  if (!fused && A.Ueig != nullptr) {
    // two phases: the eigensolve with little shared memory per CTA (many
    // units resident), then the rest with H~ staged whole
    const int T1 = kThreads / MG;
    PrecoderPlan p1 = precoder_plan(MG, T1, kEigChunk, A.p, false);
    p1.total = T1 * MG * (kEigChunk + 1);         // PHASE 1 uses the chunk region only
    const size_t smem1 = (size_t)p1.total * sizeof(float2);
    auto k1 = k_svd_precoder<MG, LT, 1>;
    cudaError_t e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
    if (e != cudaSuccess) return e;
    k1<<<dim3((A.K + T1 - 1) / T1, A.J), T1 * MG, smem1, s>>>(A, p1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    auto k2 = k_svd_precoder<MG, LT, 2>;
    if ((e = cudaFuncSetAttribute(k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    k2<<<dim3((A.K + T - 1) / T, A.J), T * MG, smem, s>>>(A, pl);
    return cudaGetLastError();
  }
  auto kern = k_svd_precoder<MG, LT, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + T - 1) / T, A.J);
  kern<<<grid, T * MG, smem, s>>>(A, pl);
  return cudaGetLastError();
}

template <int MG, int LT, int MODE>
cudaError_t launch_link_mode(const SinrArgs& A, int nz, cudaStream_t s) {
  constexpr int NC = 8;
  if (nz == 0) return cudaSuccess;
  int T = kThreads / MG;
  LinkPlan pl = link_plan(MG, LT, T, NC, A.P, A.p, MODE);
  while (T * MG > 32 && (size_t)pl.total * sizeof(float2) > kSmemBudget) {
    T /= 2;
    pl = link_plan(MG, LT, T, NC, A.P, A.p, MODE);
  }
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget) return cudaErrorInvalidValue;
  // pairwise (16-byte) staging needs even n and L, 16-byte aligned G and V and
  // a full 128-thread CTA
  pl.wide = (A.n % 2 == 0) && (A.L % 2 == 0) && LT >= 2 && (T * MG == kThreads) &&
            (((uintptr_t)A.G & 15u) == 0) && (((uintptr_t)A.V & 15u) == 0);
  dim3 grid((A.K + T - 1) / T, A.J, nz);
  auto kern = k_sinr_link<MG, LT, NC, MODE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, T * MG, smem, s>>>(A, pl);
  return cudaGetLastError();
}

template <int MG, int LT, bool SERVE = false>
cudaError_t launch_link_blocked(const SinrArgs& A, cudaStream_t s) {
  constexpr int NC = 4;
  constexpr int T = 2 * kThreads / (MG / 2);
  if (!SERVE && A.J < 2) return cudaSuccess;
  LinkPlan pl = link_plan(MG, LT, T, NC, A.P, A.p, SERVE ? kModeServe : kModeSvd);
  // the coefficient tile is only staged for dense coefficients
  if (A.coef_mode != 0) {
    const int shrink = T * A.P;
    pl.off_pa -= shrink; pl.off_pt -= shrink; pl.off_ws -= shrink; pl.off_stage -= shrink;
    pl.off_Es -= shrink; pl.total -= shrink;
  }
  // scratch of the epilogue (2 MG LT + 2 per pair of subcarriers) must fit
  // in the stage buffers
  const int es = (kThreads / (MG / 2)) * (2 * MG * LT + 2);
  if (es > 2 * pl.stage) pl.total += es - 2 * pl.stage;
  const size_t smem = (size_t)pl.total * sizeof(float2);
  // large dense coefficient tiles: the unblocked kernel shrinks its tile
  if (smem > kSmemBudget)
    return SERVE ? launch_link_mode<MG, LT, kModeServe>(A, 1, s)
                 : launch_link_mode<MG, LT, kModeSvd>(A, A.J - 1, s);
  pl.wide = (A.n % 2 == 0) && (A.L % 2 == 0) && LT >= 2 && (((uintptr_t)A.G & 15u) == 0) &&
            (SERVE || ((uintptr_t)A.V & 15u) == 0);
  dim3 grid((A.K + T - 1) / T, A.J, SERVE ? 1 : A.J - 1);
  auto kern = k_sinr_link_blk<MG, LT, SERVE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(A, pl);
  return cudaGetLastError();
}

}  // namespace detail
}  // namespace ts

#include "sinr_wide.cuh"

namespace ts {
namespace detail {

// svd: interfering links (the blocked kernel for m > 2, the wide-core kernel
// for cores the narrow kernels cannot stage); wideband precoder: every link
template <int MG, int LT>
cudaError_t run_links(const SinrArgs& A, bool svd, cudaStream_t s) {
  if (svd && wide_core(A.P, A.p)) return launch_link_wide<(MG <= 8 ? 8 : 16), LT, false>(A, s);
  if (svd) {
    if (MG >= 4 && A.p <= 32 && A.link_variant != 2)
      return launch_link_blocked<(MG >= 4 ? MG : 4), LT>(A, s);
    return launch_link_mode<MG, LT, kModeSvd>(A, A.J - 1, s);
  }
  return launch_link_mode<MG, LT, kModeFold>(A, A.J, s);
}

// svd with large cores: the serving links' compressed channels H~_kk into
// workspace, for the precoder to read
template <int MG, int LT>
cudaError_t run_serving(const SinrArgs& A, cudaStream_t s) {
  if (wide_core(A.P, A.p)) return launch_link_wide<(MG <= 8 ? 8 : 16), LT, true>(A, s);
  if (MG >= 4 && A.p <= 32 && A.link_variant != 2)
    return launch_link_blocked<(MG >= 4 ? MG : 4), LT, true>(A, s);
  return launch_link_mode<MG, LT, kModeServe>(A, 1, s);
}

// adjoint: rebuild every link's compressed channel H~_ik into workspace
template <int MG, int LT>
cudaError_t run_rebuild(const SinrArgs& A, cudaStream_t s) {
  return launch_link_mode<MG, LT, kModeRebuild>(A, A.J, s);
}

template <int MG, int LT>
cudaError_t run_finalize(const SinrArgs& A, bool svd, cudaStream_t s) {
  const int T = kThreads / MG;
  dim3 grid((A.K + T - 1) / T, A.J);
  if (svd)
    k_sinr_finalize<MG, LT, true><<<grid, kThreads, 0, s>>>(A, T);
  else
    k_sinr_finalize<MG, LT, false><<<grid, kThreads, 0, s>>>(A, T);
  return cudaGetLastError();
}

}  // namespace detail
}  // namespace ts
