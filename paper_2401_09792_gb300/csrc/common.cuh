// Device helpers shared by the SINR kernels: complex float arithmetic and
// small dense linear algebra on matrices held one row per lane inside a
// group of MG consecutive lanes of a warp (MG in {2, 4, 8, 16}).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ts {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float2 cz() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void cmacc(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(a.y, b.x, acc.y);
  acc.y = fmaf(-a.x, b.y, acc.y);
}
// acc -= a * conj(b)
__device__ __forceinline__ void cmsc(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(-a.y, b.x, acc.y);
  acc.y = fmaf(a.x, b.y, acc.y);
}
// acc -= a * b
__device__ __forceinline__ void cms(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(-a.x, b.x, acc.x);
  acc.x = fmaf(a.y, b.y, acc.x);
  acc.y = fmaf(-a.x, b.y, acc.y);
  acc.y = fmaf(-a.y, b.x, acc.y);
}

// Double-float accumulation: a value held as hi + lo, |lo| <~ ulp(hi).
// TwoSum (Knuth) and the FMA product error make each step exact up to the
// rounding of lo, so a sum of products of FP32 numbers keeps ~2^-44 of its
// largest term.  The explicit _rn intrinsics keep the compiler from fusing
// the product into the sum, which would break the error terms.
__device__ __forceinline__ void df_add_prod(float& hi, float& lo, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float pe = fmaf(x, y, -p);                // x y - p, exactly
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // hi + p - s
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}
// (hi, lo) += (h2, l2), both double-float
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));   // hi + h2 - s
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(l2, e));
}
// (hi, lo) += a * conj(b), real and imaginary parts separately
__device__ __forceinline__ void df_cmacc(float2& hi, float2& lo, float2 a, float2 b) {
  df_add_prod(hi.x, lo.x, a.x, b.x);
  df_add_prod(hi.x, lo.x, a.y, b.y);
  df_add_prod(hi.y, lo.y, a.y, b.x);
  df_add_prod(hi.y, lo.y, -a.x, b.y);
}

template <int MG>
__device__ __forceinline__ float2 gshfl(float2 v, int src) {
  return make_float2(__shfl_sync(FULL, v.x, src, MG), __shfl_sync(FULL, v.y, src, MG));
}

// Sum over the MG lanes of the group; every lane gets the total.
template <int MG>
__device__ __forceinline__ float gsum(float v) {
#pragma unroll
  for (int o = MG / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o, MG);
  return v;
}

// Element `idx` (lane-dependent) of a register array, without local memory.
template <int N>
__device__ __forceinline__ float2 pick(const float2 (&v)[N], int idx) {
  float2 r = v[0];
#pragma unroll
  for (int j = 1; j < N; ++j) r = (j == idx) ? v[j] : r;
  return r;
}
template <int N>
__device__ __forceinline__ float pickf(const float (&v)[N], int idx) {
  float r = v[0];
#pragma unroll
  for (int j = 1; j < N; ++j) r = (j == idx) ? v[j] : r;
  return r;
}
template <int N>
__device__ __forceinline__ void add_diag(float2 (&v)[N], int idx, float d) {
#pragma unroll
  for (int j = 0; j < N; ++j)
    if (j == idx) v[j].x += d;
}

// In-place Cholesky A = L L* of a Hermitian positive-definite NN x NN matrix
// (NN <= MG) stored one row per lane of a group of MG lanes: lane a < NN
// holds row a (only entries b <= a are read).  On return lane a holds row a
// of L in entries b <= a.  Lanes a >= NN take part in the shuffles but their
// values are meaningless.  Returns false if a pivot was not positive or not
// finite (the same answer in every lane of the group).
template <int MG, int NN>
__device__ __forceinline__ bool chol_rows(float2 (&A)[NN], int a) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < NN; ++j) {
    const float d = __shfl_sync(FULL, A[j].x, j, MG);
    ok = ok && (d > 0.f) && isfinite(d);
    const float ljj = sqrtf(d);
    const float inv = 1.0f / ljj;
    if (a > j) A[j] = cscale(A[j], inv);
    if (a == j) A[j] = make_float2(ljj, 0.f);
#pragma unroll
    for (int b = j + 1; b < NN; ++b) {
      const float2 lbj = gshfl<MG>(A[j], b);
      if (b <= a) cmsc(A[b], A[j], lbj);
    }
  }
  return ok;
}

// Forward substitution L X = Y for the NN x NN lower-triangular L held one
// row per lane (from chol_rows); Y is NN x NR, one row per lane, and is
// overwritten by X.
template <int MG, int NN, int NR>
__device__ __forceinline__ void trsv_rows(const float2 (&Lr)[NN], float2 (&Y)[NR], int a) {
#pragma unroll
  for (int j = 0; j < NN; ++j) {
    if (a == j) {
      const float inv = 1.0f / Lr[j].x;
#pragma unroll
      for (int r = 0; r < NR; ++r) Y[r] = cscale(Y[r], inv);
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 xj = gshfl<MG>(Y[r], j);
      if (a > j) cms(Y[r], Lr[j], xj);
    }
  }
}

// Back substitution L* X = Y for the NN x NN lower-triangular L held one row
// per lane (from chol_rows); Y (NN x NR, one row per lane) is overwritten by
// X.  Row j of L is broadcast entry by entry, so lane a < j gets L[j][a].
template <int MG, int NN, int NR>
__device__ __forceinline__ void trsv_rows_conjT(const float2 (&Lr)[NN], float2 (&Y)[NR], int a) {
#pragma unroll
  for (int j = NN - 1; j >= 0; --j) {
    if (a == j) {
      const float inv = 1.0f / Lr[j].x;
#pragma unroll
      for (int r = 0; r < NR; ++r) Y[r] = cscale(Y[r], inv);
    }
    float2 lja = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < j; ++c) {
      const float2 v = gshfl<MG>(Lr[c], j);
      if (c == a) lja = v;
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 xj = gshfl<MG>(Y[r], j);
      if (a < j) cmsc(Y[r], xj, lja);     // Y[a] -= conj(L[j][a]) X[j]
    }
  }
}

}  // namespace ts
