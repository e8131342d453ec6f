// Groupwise Tucker fit (Section 3.2, Algorithm 2) on the GPU, in FP64, and
// the same alternating update for the shared (eq. 12: one A, one B) and
// individual (eq. 10: A_ik, B_ik per link) models: every factor is fitted
// from the mode Gram summed over the links that share it.
//
// X_ik ~ G_ik x_1 A_i x_2 B_k x_3 C_ik (eq. 14) with one UE per cell: link
// ch = i*J + k.  After the initialisation (eq. 20-22 with the other factors
// set to the identity), S Gauss-Seidel sweeps update all A_i (eq. 20), then
// all B_k (eq. 21) with the new A, then all C_ik (eq. 22) with the new A, B;
// each factor is the leading eigenvectors of a summed mode Gram.  The core
// (eq. 17) is formed once at the end.  The objective g of eq. (19) after each
// block update is the sum of the kept eigenvalues of that update's Grams.
//
// Tensors are stored mode-3 slowest, mode-2 fastest: T[l][i3][i1][i2] (the
// layout of X [ch][P][M][N] and of the core [ch][p][m][n]).  Factors are
// [dim][rank], row-major.
//
// Eigensolvers: cyclic Jacobi with a round-robin ordering in one CTA for
// dimensions <= kJacobiMax; above that, block subspace iteration with
// Cholesky-QR and a Rayleigh-Ritz step (Jacobi on the block) warm-started
// from the current factor.  Blocks wider than kJacobiMax (ranks above 56)
// keep the Jacobi matrices and the Cholesky factor in global scratch; when
// the block would span the whole space the Gram itself goes to Jacobi.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tuckersinr.h"

namespace ts {
namespace fit {
namespace {

__device__ __forceinline__ double2 dz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 dconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double dabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
__device__ __forceinline__ void dmac(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += a * conj(b)
__device__ __forceinline__ void dmacc(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
}
__device__ __forceinline__ double2 ld(const double2* p, size_t i) { return p[i]; }

int nblocks(size_t total) {
  const size_t b = (total + 255) / 256;
  return (int)(b == 0 ? 1 : (b < 152 * 64 ? b : 152 * 64));
}

// out = in x_mode U^H for every link l: the contracted index i of `mode`
// (0: i1, 1: i2, 2: i3) becomes r, out[..r..] = sum_i conj(U[i][r]) in[..i..].
// Dims of `in`: d1, d2, d3; the factor of link l is U + off(l) * dim * r
// where off(l) is the link's A (fsel 0) or B (fsel 1) factor under `model`,
// or l (C_ik, fsel 2).
__device__ __forceinline__ int factor_of(int l, int J, int fsel, int model) {
  if (fsel == 2 || model == 2) return l;
  if (model == 1) return 0;
  return fsel == 0 ? l / J : l % J;
}

template <typename TIn>
__global__ void k_modeprod(const TIn* in, int nlink, int J, int d1, int d2, int d3, int mode,
                           const double2* U, int fsel, int model, int r, double2* out) {
  const int o1 = mode == 0 ? r : d1, o2 = mode == 1 ? r : d2, o3 = mode == 2 ? r : d3;
  const int dim = mode == 0 ? d1 : mode == 1 ? d2 : d3;
  const size_t per = (size_t)o1 * o2 * o3;
  const size_t total = per * nlink;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx / per);
    size_t t = idx - (size_t)l * per;
    const int j2 = (int)(t % o2);
    t /= o2;
    const int j1 = (int)(t % o1);
    const int j3 = (int)(t / o1);
    const int f = factor_of(l, J, fsel, model);
    const double2* Uf = U + (size_t)f * dim * r;
    const TIn* src = in + (size_t)l * d1 * d2 * d3;
    double2 acc = dz();
    if (mode == 0) {
      for (int i = 0; i < dim; ++i)
        dmacc(acc, ld(src, ((size_t)j3 * d1 + i) * d2 + j2), Uf[(size_t)i * r + j1]);
    } else if (mode == 1) {
      for (int i = 0; i < dim; ++i)
        dmacc(acc, ld(src, ((size_t)j3 * d1 + j1) * d2 + i), Uf[(size_t)i * r + j2]);
    } else {
      for (int i = 0; i < dim; ++i)
        dmacc(acc, ld(src, ((size_t)i * d1 + j1) * d2 + j2), Uf[(size_t)i * r + j3]);
    }
    out[idx] = acc;
  }
}

// Summed mode Gram.  gmode 0: one Gram T_(1) T_(1)^H per A factor, summed
// over the links that share it (groupwise: links (i, k) for fixed i); gmode
// 1: the same for B (groupwise: fixed k); gmode 2: one Gram T_(3) T_(3)^H per
// link.  T is [l][d3][d1][d2].
__global__ void k_gram(const double2* T, int J, int d1, int d2, int d3, int gmode, int model,
                       double2* Gm) {
  const int dim = gmode == 0 ? d1 : gmode == 1 ? d2 : d3;
  const int nmat = gmode == 2 ? J * J : fit_groups(J, model);
  // links of group g: groupwise J of them, shared all J^2, individual one
  const int nsum = gmode == 2 || model == 2 ? 1 : model == 1 ? J * J : J;
  const size_t total = (size_t)nmat * dim * dim;
  const size_t per = (size_t)d1 * d2 * d3;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx % dim);
    const int a = (int)((idx / dim) % dim);
    const int g = (int)(idx / ((size_t)dim * dim));
    double2 acc = dz();
    for (int s = 0; s < nsum; ++s) {
      const int l = gmode == 2 || model == 2 ? g : model == 1 ? s : gmode == 0 ? g * J + s : s * J + g;
      const double2* src = T + (size_t)l * per;
      if (gmode == 0) {
        for (int i3 = 0; i3 < d3; ++i3)
          for (int i2 = 0; i2 < d2; ++i2)
            dmacc(acc, src[((size_t)i3 * d1 + a) * d2 + i2], src[((size_t)i3 * d1 + b) * d2 + i2]);
      } else if (gmode == 1) {
        for (int i3 = 0; i3 < d3; ++i3)
          for (int i1 = 0; i1 < d1; ++i1)
            dmacc(acc, src[((size_t)i3 * d1 + i1) * d2 + a], src[((size_t)i3 * d1 + i1) * d2 + b]);
      } else {
        for (int i1 = 0; i1 < d1; ++i1)
          for (int i2 = 0; i2 < d2; ++i2)
            dmacc(acc, src[((size_t)a * d1 + i1) * d2 + i2], src[((size_t)b * d1 + i1) * d2 + i2]);
      }
    }
    Gm[idx] = acc;
  }
}

// Cyclic Jacobi on one Hermitian D x D matrix per CTA, round-robin
// ordering, FP64.  Writes the r leading eigenvectors (descending
// eigenvalues, each column's largest-modulus entry made real positive) to
// out[mat] ([D][r]) and the sum of the r leading eigenvalues to lsum[mat].
// With `basis` non-null the eigenvectors are mapped through it first:
// out = basis[mat] ([N][D]) * eigvecs (Rayleigh-Ritz), out is [N][r].
// The matrix and its rotation accumulator live in shared memory for
// D <= kJacobiMax, else (GLOB) in the CTA's slice of the global scratch
// `gs` (2 D (D + 1) entries per matrix, L2-resident); the per-pair
// rotations stay in shared memory either way.
constexpr int kJacobiMax = 72;
constexpr int kJacobiThreads = 256;
template <bool GLOB>
__global__ void __launch_bounds__(kJacobiThreads)
k_jacobi(const double2* Sin, int D, int r, double2* out, double* lsum, const double2* basis,
         int N, double2* gs) {
  extern __shared__ __align__(16) double2 js[];
  const int SD = D + 1;
  const int Dcap = GLOB ? D : kJacobiMax;
  const int mat = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  double2* S = GLOB ? gs + (size_t)mat * 2 * D * SD : js;   // D x SD
  double2* U = S + D * SD;                                  // D x SD
  double2* rcs = GLOB ? js : U + D * SD;                    // (c, s) per pair
  double2* rph = rcs + Dcap / 2 + 1;    // e per pair; later the r <= D column phases
  int* pq = reinterpret_cast<int*>(rph + Dcap);
  double* red = reinterpret_cast<double*>(pq + Dcap + 2);
  const double2* src = Sin + (size_t)mat * D * D;
  for (int t = tid; t < D * D; t += nth) {
    const int a = t / D, b = t - a * D;
    S[a * SD + b] = src[t];
    U[a * SD + b] = make_double2(a == b ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const int DE = D + (D & 1);           // padded to even for the pairing
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence: off-diagonal energy vs total
    double off = 0.0, tot = 0.0;
    for (int t = tid; t < D * D; t += nth) {
      const int a = t / D, b = t - a * D;
      const double v = dabs2(S[a * SD + b]);
      tot += v;
      if (a != b) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((tid & 31) == 0) { red[2 * (tid >> 5)] = off; red[2 * (tid >> 5) + 1] = tot; }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, st = 0.0;
      for (int w = 0; w < nth / 32; ++w) { so += red[2 * w]; st += red[2 * w + 1]; }
      red[64] = (so <= 1e-30 * st) ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool done = red[64] != 0.0;
    __syncthreads();
    if (done) break;
    for (int step = 0; step < DE - 1; ++step) {
      for (int j = tid; j < DE / 2; j += nth) {
        int p = j == 0 ? step : (step + j) % (DE - 1);
        int q = j == 0 ? DE - 1 : (step - j + DE - 1) % (DE - 1);
        double c = 1.0, s = 0.0;
        double2 e = make_double2(1.0, 0.0);
        if (p < D && q < D) {
          const double app = S[p * SD + p].x, aqq = S[q * SD + q].x;
          const double2 bpq = S[p * SD + q];
          const double ab = sqrt(dabs2(bpq));
          if (ab > 1e-300 && ab > 1e-17 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * ab);
            const double tt = copysign(1.0, tau) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
            e = dscale(bpq, 1.0 / ab);
          }
        } else {
          p = q = -1;
        }
        rcs[j] = make_double2(c, s);
        rph[j] = e;
        pq[2 * j] = p;
        pq[2 * j + 1] = q;
      }
      __syncthreads();
      // rows: S <- J* S
      for (int t = tid; t < (DE / 2) * D; t += nth) {
        const int j = t / D, col = t - j * D;
        const int p = pq[2 * j], q = pq[2 * j + 1];
        if (p < 0) continue;
        const double2 rr = rcs[j];
        const double2 e = rph[j];
        const double2 x = S[p * SD + col], y = S[q * SD + col];
        S[p * SD + col] = dadd(dscale(x, rr.x), dscale(dmul(e, y), -rr.y));
        S[q * SD + col] = dadd(dscale(dmul(dconj(e), x), rr.y), dscale(y, rr.x));
      }
      __syncthreads();
      // columns: S <- S J, U <- U J
      for (int t = tid; t < (DE / 2) * D; t += nth) {
        const int j = t / D, row = t - j * D;
        const int p = pq[2 * j], q = pq[2 * j + 1];
        if (p < 0) continue;
        const double2 rr = rcs[j];
        const double2 e = rph[j];
        {
          const double2 x = S[row * SD + p], y = S[row * SD + q];
          S[row * SD + p] = dadd(dscale(x, rr.x), dscale(dmul(dconj(e), y), -rr.y));
          S[row * SD + q] = dadd(dscale(dmul(e, x), rr.y), dscale(y, rr.x));
        }
        {
          const double2 x = U[row * SD + p], y = U[row * SD + q];
          U[row * SD + p] = dadd(dscale(x, rr.x), dscale(dmul(dconj(e), y), -rr.y));
          U[row * SD + q] = dadd(dscale(dmul(e, x), rr.y), dscale(y, rr.x));
        }
      }
      __syncthreads();
    }
  }
  // order: rank of each eigenvalue (descending; ties by index)
  for (int a = tid; a < D; a += nth) {
    const double la = S[a * SD + a].x;
    int rk = 0;
    for (int b = 0; b < D; ++b) {
      const double lb = S[b * SD + b].x;
      rk += (lb > la) || (lb == la && b < a);
    }
    pq[rk] = a;
  }
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int j = 0; j < r; ++j) sum += S[pq[j] * SD + pq[j]].x;
    lsum[mat] = sum;
  }
  // phase of each kept column: largest-modulus entry real positive
  for (int j = tid; j < r; j += nth) {
    const int col = pq[j];
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < D; ++a) {
      const double v = dabs2(U[a * SD + col]);
      if (v > bv) { bv = v; best = a; }
    }
    const double2 u = U[best * SD + col];
    const double nu = sqrt(dabs2(u));
    rph[j] = make_double2(nu > 0 ? u.x / nu : 1.0, nu > 0 ? -u.y / nu : 0.0);   // conj phase
  }
  __syncthreads();
  if (basis == nullptr) {
    for (int t = tid; t < D * r; t += nth) {
      const int a = t / r, j = t - a * r;
      out[(size_t)mat * D * r + t] = dmul(U[a * SD + pq[j]], rph[j]);
    }
  } else {
    const double2* Bm = basis + (size_t)mat * N * D;
    for (int t = tid; t < N * r; t += nth) {
      const int a = t / r, j = t - a * r;
      double2 acc = dz();
      for (int b = 0; b < D; ++b) dmac(acc, Bm[(size_t)a * D + b], U[b * SD + pq[j]]);
      out[(size_t)mat * N * r + t] = dmul(acc, rph[j]);
    }
  }
}

// Y[mat] = S[mat] Q[mat]  (N x N times N x c)
__global__ void k_gemm_sq(const double2* S, const double2* Q, int nmat, int N, int c, double2* Y) {
  const size_t total = (size_t)nmat * N * c;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % c);
    const int a = (int)((idx / c) % N);
    const int mat = (int)(idx / ((size_t)N * c));
    const double2* Sr = S + ((size_t)mat * N + a) * N;
    const double2* Qm = Q + (size_t)mat * N * c;
    double2 acc = dz();
    for (int b = 0; b < N; ++b) dmac(acc, Sr[b], Qm[(size_t)b * c + j]);
    Y[idx] = acc;
  }
}

// T[mat] = Q^H S Q  (c x c), with SQ = S Q given
__global__ void k_gemm_qhy(const double2* Q, const double2* Y, int nmat, int N, int c, double2* T) {
  const size_t total = (size_t)nmat * c * c;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % c);
    const int i = (int)((idx / c) % c);
    const int mat = (int)(idx / ((size_t)c * c));
    const double2* Qm = Q + (size_t)mat * N * c;
    const double2* Ym = Y + (size_t)mat * N * c;
    double2 acc = dz();
    for (int a = 0; a < N; ++a) dmacc(acc, Ym[(size_t)a * c + j], Qm[(size_t)a * c + i]);
    T[idx] = acc;
  }
}

// Orthonormalise the columns of Y[mat] (N x c) in place into Q: Cholesky-QR
// (R^H R = Y^H Y, Q = Y R^{-1}); one CTA per matrix.  R in shared memory
// for c <= kJacobiMax, else (GLOB) in the CTA's slice of the global scratch.
template <bool GLOB>
__global__ void __launch_bounds__(kJacobiThreads) k_cholqr(double2* Y, int N, int c, double2* gs) {
  extern __shared__ __align__(16) double2 cs[];
  const int SC = c + 1;
  const int mat = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  double2* R = GLOB ? gs + (size_t)mat * c * SC : cs;     // c x SC
  double2* Ym = Y + (size_t)mat * N * c;
  for (int t = tid; t < c * c; t += nth) {
    const int i = t / c, j = t - i * c;
    double2 acc = dz();
    for (int a = 0; a < N; ++a) dmacc(acc, Ym[(size_t)a * c + j], Ym[(size_t)a * c + i]);
    R[i * SC + j] = acc;                   // (Y^H Y)[i][j]
  }
  __syncthreads();
  // Cholesky Y^H Y = L L^H in place (lower), sequential over columns
  for (int j = 0; j < c; ++j) {
    if (tid == 0) {
      const double d = R[j * SC + j].x;
      R[j * SC + j] = make_double2(d > 0.0 ? sqrt(d) : 1.0, 0.0);
    }
    __syncthreads();
    const double ljj = R[j * SC + j].x;
    for (int i = j + 1 + tid; i < c; i += nth) R[i * SC + j] = dscale(R[i * SC + j], 1.0 / ljj);
    __syncthreads();
    for (int t = tid; t < (c - j - 1) * (c - j - 1); t += nth) {
      const int i = j + 1 + t / (c - j - 1), k = j + 1 + t % (c - j - 1);
      if (k <= i) {
        double2 v = R[i * SC + k];
        const double2 pr = dmul(R[i * SC + j], dconj(R[k * SC + j]));
        R[i * SC + k] = make_double2(v.x - pr.x, v.y - pr.y);
      }
    }
    __syncthreads();
  }
  // Q = Y L^{-H}: each row y (1 x c) solves q L^H = y by forward substitution
  if (GLOB) {
    // in place: q_j overwrites y_j once the q_k, k < j, it needs are written
    for (int a = tid; a < N; a += nth) {
      double2* row = Ym + (size_t)a * c;
      for (int j = 0; j < c; ++j) {
        double2 v = row[j];
        for (int k = 0; k < j; ++k) {
          const double2 pr = dmul(row[k], dconj(R[j * SC + k]));
          v = make_double2(v.x - pr.x, v.y - pr.y);
        }
        row[j] = dscale(v, 1.0 / R[j * SC + j].x);
      }
    }
  } else {
    for (int a = tid; a < N; a += nth) {
      double2 q[kJacobiMax];
      for (int j = 0; j < c; ++j) {
        double2 v = Ym[(size_t)a * c + j];
        for (int k = 0; k < j; ++k) {
          const double2 pr = dmul(q[k], dconj(R[j * SC + k]));
          v = make_double2(v.x - pr.x, v.y - pr.y);
        }
        q[j] = dscale(v, 1.0 / R[j * SC + j].x);
      }
      for (int j = 0; j < c; ++j) Ym[(size_t)a * c + j] = q[j];
    }
  }
}

// Start block: the current factor (warm start) in its r columns, then
// columns of the identity for the oversampling columns.
__global__ void k_start_block(const double2* F, int nmat, int N, int r, int c, double2* Q) {
  const size_t total = (size_t)nmat * N * c;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx % c);
    const int a = (int)((idx / c) % N);
    const int mat = (int)(idx / ((size_t)N * c));
    double2 v;
    if (j < r && F != nullptr)
      v = F[((size_t)mat * N + a) * r + j];
    else {
      // deterministic, well spread start: exp(2 pi i a (j + 1) / N) / sqrt(N)
      double s, co;
      sincospi(2.0 * (double)a * (double)(j + 1) / (double)N, &s, &co);
      v = make_double2(co / sqrt((double)N), s / sqrt((double)N));
    }
    Q[idx] = v;
  }
}

__global__ void k_to_double(const float2* in, size_t count, double2* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2(in[i].x, in[i].y);
}

__global__ void k_to_float(const double2* in, size_t count, float2* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

// g_hist[slot] = sum of lsum[0 .. nmat)
__global__ void k_sum_g(const double* lsum, int nmat, double* g_hist, int slot) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nmat; ++i) s += lsum[i];
    g_hist[slot] = s;
  }
}

// g = sum |core|^2 over all links
__global__ void k_norm2(const double2* T, size_t count, double* g_hist, int slot) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = threadIdx.x; i < count; i += blockDim.x) s += dabs2(T[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    g_hist[slot] = t;
  }
}

}  // namespace

// Columns of the subspace-iteration block for a D x D eigenproblem keeping r
// (0: D <= kJacobiMax, solved directly in shared memory).  Oversampled to
// max(r + 16, 2 r) while that fits the shared-memory block, else to
// kJacobiMax while r + 16 does, else (large ranks) to min(D, max(r + 16,
// 2 r)) with the block kept in global memory.
int eig_block(int D, int r) {
  if (D <= kJacobiMax) return 0;
  int c = r + 16 > 2 * r ? r + 16 : 2 * r;
  if (c > kJacobiMax && r + 16 <= kJacobiMax) c = kJacobiMax;
  return c > D ? D : c;
}

size_t jacobi_smem(int D, bool glob) {
  const int Dcap = glob ? D : kJacobiMax;
  return (glob ? 0 : (size_t)2 * kJacobiMax * (kJacobiMax + 1) * sizeof(double2)) +
         (size_t)(Dcap / 2 + 1 + Dcap) * sizeof(double2) + (size_t)(Dcap + 2) * sizeof(int) +
         80 * sizeof(double);
}

// Entries of the subspace blocks (Q, Y, T each) and of the global Jacobi /
// Cholesky-QR scratch that the fit's three factor updates need.
void eig_sizes(const FitDims& f, size_t& blk, size_t& gsz) {
  const size_t J2 = (size_t)f.J * f.J, nG = fit_groups(f.J, f.model);
  blk = 1;
  gsz = 1;
  auto need = [&](int D, int r, size_t nmat) {
    const int c = eig_block(D, r);
    if (c == 0) return;
    if (c < D && nmat * D * c > blk) blk = nmat * D * c;
    if (c > kJacobiMax && nmat * 2 * c * (c + 1) > gsz) gsz = nmat * 2 * (size_t)c * (c + 1);
  };
  need(f.M, f.m, nG);
  need(f.N, f.n, nG);
  need(f.P, f.p, J2);
}

// Leading r eigenvectors of nmat Hermitian D x D matrices S (FP64) into F
// ([nmat][D][r]), their eigenvalue sums into lsum.  `warm`: F holds a start.
// gscratch: 2 c (c + 1) entries per matrix for blocks beyond kJacobiMax.
cudaError_t leading_eigvecs(const double2* S, int nmat, int D, int r, double2* F, double* lsum,
                            bool warm, double2* Qbuf, double2* Ybuf, double2* Tbuf, int iters,
                            double2* gscratch, cudaStream_t s) {
  const size_t jsm = jacobi_smem(D, false);
  cudaError_t e = cudaFuncSetAttribute(k_jacobi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)jsm);
  if (e != cudaSuccess) return e;
  if (D <= kJacobiMax) {
    k_jacobi<false><<<nmat, kJacobiThreads, jsm, s>>>(S, D, r, F, lsum, nullptr, 0, nullptr);
    return cudaGetLastError();
  }
  const int c = eig_block(D, r);
  const bool glob = c > kJacobiMax;
  if (c == D) {
    // the block would be the whole space: solve S itself
    k_jacobi<true><<<nmat, kJacobiThreads, jacobi_smem(D, true), s>>>(S, D, r, F, lsum, nullptr, 0,
                                                                      gscratch);
    return cudaGetLastError();
  }
  // block subspace iteration on c columns; a cold start (initialisation)
  // runs three times as long
  if (!warm) iters *= 3;
  k_start_block<<<nblocks((size_t)nmat * D * c), 256, 0, s>>>(warm ? F : nullptr, nmat, D, r, c, Qbuf);
  const size_t qsm = glob ? 0 : (size_t)c * (c + 1) * sizeof(double2);
  if (!glob) {
    e = cudaFuncSetAttribute(k_cholqr<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm);
    if (e != cudaSuccess) return e;
  }
  auto cholqr = [&](double2* Yb) {
    if (glob)
      k_cholqr<true><<<nmat, kJacobiThreads, 0, s>>>(Yb, D, c, gscratch);
    else
      k_cholqr<false><<<nmat, kJacobiThreads, qsm, s>>>(Yb, D, c, nullptr);
  };
  cholqr(Qbuf);
  for (int it = 0; it < iters; ++it) {
    k_gemm_sq<<<nblocks((size_t)nmat * D * c), 256, 0, s>>>(S, Qbuf, nmat, D, c, Ybuf);
    cholqr(Ybuf);
    double2* t = Qbuf; Qbuf = Ybuf; Ybuf = t;
  }
  // Rayleigh-Ritz: T = Q^H S Q, eigenvectors of T mapped through Q
  k_gemm_sq<<<nblocks((size_t)nmat * D * c), 256, 0, s>>>(S, Qbuf, nmat, D, c, Ybuf);
  k_gemm_qhy<<<nblocks((size_t)nmat * c * c), 256, 0, s>>>(Qbuf, Ybuf, nmat, D, c, Tbuf);
  if (glob)
    k_jacobi<true><<<nmat, kJacobiThreads, jacobi_smem(c, true), s>>>(Tbuf, c, r, F, lsum, Qbuf, D,
                                                                      gscratch);
  else
    k_jacobi<false><<<nmat, kJacobiThreads, jsm, s>>>(Tbuf, c, r, F, lsum, Qbuf, D, nullptr);
  return cudaGetLastError();
}

}  // namespace fit

namespace fit {
namespace {

// One forward mode product per launch, FP32: out = in x_mode U with U the
// link's factor ([dim_out][r], row-major), in [l][i3][i1][i2] with the
// contracted index of `mode` running over r.
__global__ void k_expand(const float2* in, int nlink, int J, int o1, int o2, int o3, int mode,
                         const float2* U, int fsel, int model, int r, float2* out) {
  const size_t per = (size_t)o1 * o2 * o3;
  const size_t total = per * nlink;
  const int i1n = mode == 0 ? r : o1, i2n = mode == 1 ? r : o2;
  const int dim = mode == 0 ? o1 : mode == 1 ? o2 : o3;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx / per);
    size_t t = idx - (size_t)l * per;
    const int j2 = (int)(t % o2);
    t /= o2;
    const int j1 = (int)(t % o1);
    const int j3 = (int)(t / o1);
    const float2* Uf = U + (size_t)factor_of(l, J, fsel, model) * dim * r;
    const size_t lin = (size_t)l * (mode == 0 ? (size_t)r * o2 * o3 : mode == 1 ? (size_t)o1 * r * o3
                                                                               : (size_t)o1 * o2 * r);
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < r; ++q) {
      const float2 u = Uf[(size_t)(mode == 0 ? j1 : mode == 1 ? j2 : j3) * r + q];
      const size_t src = mode == 0 ? ((size_t)j3 * i1n + q) * i2n + j2
                       : mode == 1 ? ((size_t)j3 * i1n + j1) * i2n + q
                                   : ((size_t)q * i1n + j1) * i2n + j2;
      const float2 v = in[lin + src];
      acc.x = fmaf(u.x, v.x, acc.x);
      acc.x = fmaf(-u.y, v.y, acc.x);
      acc.y = fmaf(u.x, v.y, acc.y);
      acc.y = fmaf(u.y, v.x, acc.y);
    }
    out[idx] = acc;
  }
}

}  // namespace
}  // namespace fit

size_t reconstruct_workspace_bytes(const FitDims& f) {
  const size_t J2 = (size_t)f.J * f.J;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  return al(J2 * f.p * f.M * f.n * sizeof(float2)) + al(J2 * f.p * f.M * f.N * sizeof(float2));
}

cudaError_t launch_reconstruct(const FitDims& f, const float2* A, const float2* B, const float2* C,
                               const float2* G, float2* Xhat, void* ws, cudaStream_t s) {
  using namespace fit;
  const size_t J2 = (size_t)f.J * f.J;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  float2* T1 = static_cast<float2*>(ws);                                   // [l][p][M][n]
  float2* T2 = reinterpret_cast<float2*>(static_cast<char*>(ws) + al(J2 * f.p * f.M * f.n * sizeof(float2)));
  // G [l][p][m][n] x_1 A -> [l][p][M][n] x_2 B -> [l][p][M][N] x_3 C -> [l][P][M][N]
  k_expand<<<nblocks(J2 * f.p * f.M * f.n), 256, 0, s>>>(G, (int)J2, f.J, f.M, f.n, f.p, 0, A, 0, f.model,
                                                         f.m, T1);
  k_expand<<<nblocks(J2 * f.p * f.M * f.N), 256, 0, s>>>(T1, (int)J2, f.J, f.M, f.N, f.p, 1, B, 1, f.model,
                                                         f.n, T2);
  k_expand<<<nblocks(J2 * f.P * f.M * f.N), 256, 0, s>>>(T2, (int)J2, f.J, f.M, f.N, f.P, 2, C, 2, f.model,
                                                         f.p, Xhat);
  return cudaGetLastError();
}

size_t fit_workspace_bytes(const FitDims& f) {
  const size_t J2 = (size_t)f.J * f.J;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t c16 = sizeof(double2);
  size_t tmax = J2 * f.P * f.M * f.N;                         // X in FP64 (largest tensor)
  size_t tb = J2 * f.P * (size_t)(f.M > f.m ? f.M : f.m) * (f.N > f.n ? f.N : f.n);
  const size_t big = (tmax > tb ? tmax : tb) * c16;
  const size_t nG = fit_groups(f.J, f.model);
  const size_t gram = (J2 * f.P * f.P + nG * f.M * f.M + nG * f.N * f.N) * c16;
  size_t blk = 0, gsz = 0;
  fit::eig_sizes(f, blk, gsz);
  return al(J2 * f.P * f.M * f.N * c16) + 2 * al(big) + al(gram) + 3 * al(blk * c16) + al(gsz * c16) +
         al((nG * f.M * f.m + nG * f.N * f.n + J2 * f.P * f.p) * c16) + al(J2 * sizeof(double));
}

cudaError_t launch_fit(const FitDims& f, const float2* X, int S, int init, float2* A, float2* B,
                       float2* C, float2* G, double* g_hist, void* ws, cudaStream_t s) {
  using namespace fit;
  const int J = f.J, M = f.M, N = f.N, P = f.P, m = f.m, n = f.n, p = f.p, model = f.model;
  const size_t J2 = (size_t)J * J;
  const int nG = fit_groups(J, model);       // A and B factors
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  const size_t c16 = sizeof(double2);
  char* base = static_cast<char*>(ws);
  size_t o = 0;
  auto take = [&](size_t bytes) { char* p0 = base + o; o += al(bytes); return p0; };
  size_t tmax = J2 * P * M * N;
  size_t tb = J2 * P * (size_t)(M > m ? M : m) * (N > n ? N : n);
  const size_t big = (tmax > tb ? tmax : tb) * c16;
  double2* Xd = reinterpret_cast<double2*>(take(J2 * P * M * N * c16));
  double2* T1 = reinterpret_cast<double2*>(take(big));
  double2* T2 = reinterpret_cast<double2*>(take(big));
  double2* GC = reinterpret_cast<double2*>(
      take((J2 * P * P + (size_t)nG * M * M + (size_t)nG * N * N) * c16));
  double2* GA = GC + J2 * P * P;
  double2* GB = GA + (size_t)nG * M * M;
  size_t blk = 0, gsz = 0;
  eig_sizes(f, blk, gsz);
  double2* Qb = reinterpret_cast<double2*>(take(blk * c16));
  double2* Yb = reinterpret_cast<double2*>(take(blk * c16));
  double2* Tb = reinterpret_cast<double2*>(take(blk * c16));
  double2* gs = reinterpret_cast<double2*>(take(gsz * c16));
  double2* A64 = reinterpret_cast<double2*>(
      take(((size_t)nG * M * m + (size_t)nG * N * n + J2 * P * p) * c16));
  double2* B64 = A64 + (size_t)nG * M * m;
  double2* C64 = B64 + (size_t)nG * N * n;
  double* lsum = reinterpret_cast<double*>(take(J2 * sizeof(double)));
  const int iters = f.iters > 0 ? f.iters : 40;
  cudaError_t e = cudaSuccess;
#define TS_FIT_CHECK()                            \
  do {                                            \
    if ((e = cudaGetLastError()) != cudaSuccess) \
      return e;                                   \
  } while (0)

  k_to_double<<<nblocks(J2 * P * M * N), 256, 0, s>>>(X, J2 * P * M * N, Xd);
  TS_FIT_CHECK();
  // X x_1 A^H -> [P][m][N]; then x_3 C^H -> [p][m][N] ; Gram over mode 2 (B)
  auto update_B = [&](bool warm) -> cudaError_t {
    k_modeprod<double2><<<nblocks(J2 * P * m * N), 256, 0, s>>>(Xd, (int)J2, J, M, N, P, 0, A64, 0, model, m, T1);
    k_modeprod<double2><<<nblocks(J2 * p * m * N), 256, 0, s>>>(T1, (int)J2, J, m, N, P, 2, C64, 2, model, p, T2);
    k_gram<<<nblocks((size_t)nG * N * N), 256, 0, s>>>(T2, J, m, N, p, 1, model, GB);
    return leading_eigvecs(GB, nG, N, n, B64, lsum, warm, Qb, Yb, Tb, iters, gs, s);
  };
  auto update_A = [&](bool warm) -> cudaError_t {
    k_modeprod<double2><<<nblocks(J2 * P * M * n), 256, 0, s>>>(Xd, (int)J2, J, M, N, P, 1, B64, 1, model, n, T1);
    k_modeprod<double2><<<nblocks(J2 * p * M * n), 256, 0, s>>>(T1, (int)J2, J, M, n, P, 2, C64, 2, model, p, T2);
    k_gram<<<nblocks((size_t)nG * M * M), 256, 0, s>>>(T2, J, M, n, p, 0, model, GA);
    return leading_eigvecs(GA, nG, M, m, A64, lsum, warm, Qb, Yb, Tb, iters, gs, s);
  };
  auto update_C = [&](bool warm) -> cudaError_t {
    k_modeprod<double2><<<nblocks(J2 * P * m * N), 256, 0, s>>>(Xd, (int)J2, J, M, N, P, 0, A64, 0, model, m, T1);
    k_modeprod<double2><<<nblocks(J2 * P * m * n), 256, 0, s>>>(T1, (int)J2, J, m, N, P, 1, B64, 1, model, n, T2);
    k_gram<<<nblocks(J2 * P * P), 256, 0, s>>>(T2, J, m, n, P, 2, model, GC);
    return leading_eigvecs(GC, (int)J2, P, p, C64, lsum, warm, Qb, Yb, Tb, iters, gs, s);
  };
  if (init == 0) {
    // eq. (20)-(22) with the other factors set to the identity
    k_gram<<<nblocks((size_t)nG * M * M), 256, 0, s>>>(Xd, J, M, N, P, 0, model, GA);
    if ((e = leading_eigvecs(GA, nG, M, m, A64, lsum, false, Qb, Yb, Tb, iters, gs, s)) != cudaSuccess) return e;
    k_gram<<<nblocks((size_t)nG * N * N), 256, 0, s>>>(Xd, J, M, N, P, 1, model, GB);
    if ((e = leading_eigvecs(GB, nG, N, n, B64, lsum, false, Qb, Yb, Tb, iters, gs, s)) != cudaSuccess) return e;
    k_gram<<<nblocks(J2 * P * P), 256, 0, s>>>(Xd, J, M, N, P, 2, model, GC);
    if ((e = leading_eigvecs(GC, (int)J2, P, p, C64, lsum, false, Qb, Yb, Tb, iters, gs, s)) != cudaSuccess) return e;
  } else {
    k_to_double<<<nblocks((size_t)nG * M * m), 256, 0, s>>>(A, (size_t)nG * M * m, A64);
    k_to_double<<<nblocks((size_t)nG * N * n), 256, 0, s>>>(B, (size_t)nG * N * n, B64);
    k_to_double<<<nblocks(J2 * P * p), 256, 0, s>>>(C, J2 * P * p, C64);
  }
  TS_FIT_CHECK();
  // core (eq. 17) of the current factors: W = X x_1 A^H x_2 B^H, G = W x_3 C^H
  auto core = [&]() {
    k_modeprod<double2><<<nblocks(J2 * P * m * N), 256, 0, s>>>(Xd, (int)J2, J, M, N, P, 0, A64, 0, model, m, T1);
    k_modeprod<double2><<<nblocks(J2 * P * m * n), 256, 0, s>>>(T1, (int)J2, J, m, N, P, 1, B64, 1, model, n, T2);
    k_modeprod<double2><<<nblocks(J2 * p * m * n), 256, 0, s>>>(T2, (int)J2, J, m, n, P, 2, C64, 2, model, p, T1);
  };
  if (g_hist != nullptr) {
    core();
    k_norm2<<<1, 1024, 0, s>>>(T1, J2 * p * m * n, g_hist, 0);
    TS_FIT_CHECK();
  }
  for (int sw = 0; sw < S; ++sw) {
    if ((e = update_A(true)) != cudaSuccess) return e;
    if (g_hist != nullptr) k_sum_g<<<1, 32, 0, s>>>(lsum, nG, g_hist, 1 + 3 * sw);
    if ((e = update_B(true)) != cudaSuccess) return e;
    if (g_hist != nullptr) k_sum_g<<<1, 32, 0, s>>>(lsum, nG, g_hist, 2 + 3 * sw);
    if ((e = update_C(true)) != cudaSuccess) return e;
    if (g_hist != nullptr) k_sum_g<<<1, 32, 0, s>>>(lsum, (int)J2, g_hist, 3 + 3 * sw);
    TS_FIT_CHECK();
  }
  core();
  k_to_float<<<nblocks(J2 * p * m * n), 256, 0, s>>>(T1, J2 * p * m * n, G);
  k_to_float<<<nblocks((size_t)nG * M * m), 256, 0, s>>>(A64, (size_t)nG * M * m, A);
  k_to_float<<<nblocks((size_t)nG * N * n), 256, 0, s>>>(B64, (size_t)nG * N * n, B);
  k_to_float<<<nblocks(J2 * P * p), 256, 0, s>>>(C64, J2 * P * p, C);
  return cudaGetLastError();
#undef TS_FIT_CHECK
}

}  // namespace ts
