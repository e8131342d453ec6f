// SINR kernels for more than 16 receive rows per unit (m <= 64; e.g. the
// paper's m = 60 of M = 64 receive antennas).  One unit's m x m matrices no
// longer fit a lane group's registers, so the SVD precoder and the
// finalisation hold them in shared memory, one 128-thread CTA per unit; the
// interfering and serving links run the wide-core kernel with 32 or 64 rows
// per lane group (sinr_wide.cuh).  The arithmetic is the narrow kernels':
//   k_svd_precoder_large  Gram S = H~_kk H~_kk* (eq. 23) summed in
//                         double-float and scaled to unit trace, cyclic
//                         Jacobi (round-robin pairs; each rotation by one
//                         thread, its rows and columns by lane j of every
//                         warp), V~ = conj(rows of U_L* H~)
//                         / sigma and E_kk = U_L Sigma_L (eq. 7, eq. 24);
//   k_sinr_finalize_large R = sum_{k != i} E E* + sigma^2 I (eq. 25) in
//                         double-float, Y = R^{-1} E_ii from its FP32
//                         Cholesky factor with FP64-residual refinement,
//                         x_r = [(I + E_ii* Y)^{-1}]_rr in FP64,
//                         SINR_r = (1 - x_r) / x_r (eq. 5).
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
namespace {

constexpr int kLargeThreads = 128;

// sum over the CTA (every thread gets the total); red: 32 floats
__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

// Shared-memory plan of the large precoder (float2 units).
struct LargePrecPlan {
  int SD, DE, off_S, off_U, off_H, off_rot, off_pq, off_red, total;
};

__host__ __device__ inline LargePrecPlan large_prec_plan(int m, int n, int L) {
  LargePrecPlan pl;
  pl.SD = m + 1;
  pl.DE = m + (m & 1);
  int o = 0;
  pl.off_S = o; o += m * pl.SD;
  pl.off_U = o; o += m * pl.SD;
  const int Lw = L < m ? L + 1 : m;                         // W rows: the kept ones and the next
  pl.off_H = o; o += (m * 33 > Lw * n ? m * 33 : Lw * n);  // H~ column chunk, later W rows
  pl.off_rot = o; o += pl.DE;                              // (c, s) and e per pair
  pl.off_pq = o; o += (2 * pl.DE + 2) / 2 + 1;             // ints: pairs, later the order
  pl.off_red = o; o += 20;                                 // 32 floats + a flag
  pl.total = o;
  return pl;
}

template <int MG, int LT>
__global__ void __launch_bounds__(kLargeThreads) k_svd_precoder_large(const SinrArgs A,
                                                                       const LargePrecPlan pl) {
  constexpr int MAXE = (MG * (MG + 1) / 2 + kLargeThreads - 1) / kLargeThreads;
  extern __shared__ __align__(16) float2 sm[];
  const int m = A.m, n = A.n, L = A.L, K = A.K;
  const int kap = blockIdx.x, k = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int SD = pl.SD, DE = pl.DE;
  float2* S = sm + pl.off_S;
  float2* U = sm + pl.off_U;
  float2* Hc = sm + pl.off_H;
  float2* rot = sm + pl.off_rot;                 // [DE/2] (c, s), then [DE/2] e
  int* pq = reinterpret_cast<int*>(sm + pl.off_pq);
  float* red = reinterpret_cast<float*>(sm + pl.off_red);
  const float2* H = A.Hserv + ((size_t)k * A.serv_stride * K + kap) * m * n;   // [m][n]

  // 1. Gram S = H~ H~* (lower triangle, mirrored), H~ staged 32 columns at a
  // time, accumulated in double-float (each product exact, the sums
  // compensated) and rounded once: a plain FP32 sum over n columns carries
  // ~sqrt(n) u ||S|| of rounding (n up to 1024 here), which mixes
  // eigenvectors a relative gap g apart by that over g and moves the
  // per-stream SINRs by up to ~1e-5; one rounding leaves ~u ||S||.
  float2 acc[MAXE], acl[MAXE];
#pragma unroll
  for (int e = 0; e < MAXE; ++e) acc[e] = acl[e] = cz();
  const int ntri = m * (m + 1) / 2;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int cc = min(32, n - c0);
    __syncthreads();
    for (int idx = tid; idx < m * 32; idx += nth) {
      const int a = idx / 32, c = idx % 32;
      Hc[a * 33 + c] = c < cc ? H[(size_t)a * n + c0 + c] : cz();
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < MAXE; ++e) {
      const int t = tid + e * kLargeThreads;
      if (t >= ntri) break;
      // t -> (a, b), b <= a: row a starts at a (a + 1) / 2
      int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
      while (a * (a + 1) / 2 > t) --a;
      while ((a + 1) * (a + 2) / 2 <= t) ++a;
      const int b = t - a * (a + 1) / 2;
      for (int c = 0; c < cc; ++c) df_cmacc(acc[e], acl[e], Hc[a * 33 + c], Hc[b * 33 + c]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int e = 0; e < MAXE; ++e) {
    const int t = tid + e * kLargeThreads;
    if (t >= ntri) break;
    int a = (int)((sqrtf(8.f * t + 1.f) - 1.f) * 0.5f);
    while (a * (a + 1) / 2 > t) --a;
    while ((a + 1) * (a + 2) / 2 <= t) ++a;
    const int b = t - a * (a + 1) / 2;
    const float2 v = make_float2(acc[e].x + acl[e].x, acc[e].y + acl[e].y);
    S[a * SD + b] = v;
    S[b * SD + a] = a == b ? make_float2(v.x, 0.f) : cconj(v);
  }
  for (int idx = tid; idx < m * m; idx += nth) {
    const int a = idx / m, b = idx - a * m;
    U[a * SD + b] = make_float2(a == b ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // unit trace (eigenvectors and eigenvalue ratios unchanged)
  {
    const float tr = block_sum(tid < m ? S[tid * SD + tid].x : 0.f, red);
    const float sc = tr > 0.f ? 1.f / tr : 1.f;
    for (int idx = tid; idx < m * m; idx += nth) {
      const int a = idx / m, b = idx - a * m;
      S[a * SD + b] = cscale(S[a * SD + b], sc);
    }
  }
  __syncthreads();

  // 2. cyclic Jacobi, round-robin pairs (the padding index DE-1 = m when m
  // is odd pairs with nothing), to relative off-diagonal norm ~5e-7.  Pairs
  // whose diagonal entries are both below m u of the trace lie in the
  // numerical null space of the FP32 Gram (rank n < m, or weaker): their
  // rotations only mix null vectors among themselves, at rounding level,
  // and leave the kept eigenvectors alone, so they are neither rotated nor
  // counted (otherwise a null cluster of rank-deficient links converges
  // linearly from rounding noise and exhausts the sweeps).
  const float eps_null = (float)m * 5.9604645e-8f;     // m 2^-24 of the unit trace
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  // Once the threshold is met, one more sweep takes the off-diagonal to
  // rounding level (quadratic convergence), so that nearly equal
  // eigenvalues a relative gap g apart keep only the FP32 Gram's ~u / g
  // mixing of their eigenvectors, not ~5e-7 / g.
  bool converged = false, polish = false;
  for (int sweep = 0; sweep <= 17; ++sweep) {
    float off = 0.f, tot = 0.f;
    for (int idx = tid; idx < m * m; idx += nth) {
      const int a = idx / m, b = idx - a * m;
      const float v = cabs2(S[a * SD + b]);
      tot += v;
      if (a != b && fmaxf(S[a * SD + a].x, S[b * SD + b].x) > eps_null) off += v;
    }
    off = block_sum(off, red);
    tot = block_sum(tot, red);
    converged = off <= 2.3e-13f * tot;
    if ((converged && polish) || sweep == 17) break;
    polish = converged;
    // one step: the DE/2 disjoint pairs of the round-robin ordering; their
    // rotations by one thread each, then the rows of S and the columns of S
    // and U, lane j of every warp on pair j (its rotation loaded once) and
    // the warps over the columns (rows), without index divisions
    for (int step = 0; step < DE - 1; ++step) {
      if (tid < DE / 2) {
        const int j = tid;
        int p = j == 0 ? step : (step + j) % (DE - 1);
        int q = j == 0 ? DE - 1 : (step - j + DE - 1) % (DE - 1);
        float c = 1.f, sn = 0.f;
        float2 e = make_float2(1.f, 0.f);
        bool act = false;
        if (p < m && q < m) {
          const float app = S[p * SD + p].x, aqq = S[q * SD + q].x;
          const float2 bpq = S[p * SD + q];
          const float ab = sqrtf(cabs2(bpq));
          if (ab > 1e-30f && ab > 1e-9f * sqrtf(fabsf(app * aqq)) && fmaxf(app, aqq) > eps_null) {
            const float tau = (aqq - app) / (2.f * ab);
            const float tt = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
            c = 1.f / sqrtf(fmaf(tt, tt, 1.f));
            sn = tt * c;
            e = cscale(bpq, 1.f / ab);
            act = true;
          }
        }
        rot[j] = make_float2(c, sn);
        rot[DE / 2 + j] = e;
        pq[2 * j] = act ? p : -1;
        pq[2 * j + 1] = q;
      }
      __syncthreads();
      const int j = lane;
      const bool mine = j < DE / 2 && pq[2 * j] >= 0;
      int p = 0, q = 0;
      float c = 1.f;
      float2 se = cz(), sec = cz();
      if (mine) {
        p = pq[2 * j];
        q = pq[2 * j + 1];
        const float2 cs = rot[j], e = rot[DE / 2 + j];
        c = cs.x;
        se = cscale(e, cs.y);
        sec = cscale(cconj(e), cs.y);
      }
      // rows: S <- J* S (row p' = c p - s e q, row q' = s conj(e) p + c q)
      if (mine)
        for (int col = warp; col < m; col += nwarp) {
          const float2 x = S[p * SD + col], y = S[q * SD + col];
          float2 nx = cscale(x, c), ny = cscale(y, c);
          cms(nx, se, y);
          cmac(ny, sec, x);
          S[p * SD + col] = nx;
          S[q * SD + col] = ny;
        }
      __syncthreads();
      // columns: S <- S J, U <- U J
      if (mine)
        for (int row = warp; row < m; row += nwarp) {
          {
            const float2 x = S[row * SD + p], y = S[row * SD + q];
            float2 nx = cscale(x, c), ny = cscale(y, c);
            cms(nx, sec, y);
            cmac(ny, se, x);
            S[row * SD + p] = nx;
            S[row * SD + q] = ny;
          }
          {
            const float2 x = U[row * SD + p], y = U[row * SD + q];
            float2 nx = cscale(x, c), ny = cscale(y, c);
            cms(nx, sec, y);
            cmac(ny, se, x);
            U[row * SD + p] = nx;
            U[row * SD + q] = ny;
          }
        }
      __syncthreads();
    }
  }

  // Each rotation is applied in FP32, so over the sweeps the columns of U
  // drift from unit norm (~1e-6 for 60 rows); E_kk = U_L Sigma_L below
  // scales with them, so every column is renormalised (thread c on column c).
  for (int c = tid; c < m; c += nth) {
    float nb = 0.f;
    for (int a = 0; a < m; ++a) nb += cabs2(U[a * SD + c]);
    const float sc = nb > 0.f ? 1.f / sqrtf(nb) : 1.f;
    for (int a = 0; a < m; ++a) U[a * SD + c] = cscale(U[a * SD + c], sc);
  }
  __syncthreads();

  // 3. order of the eigenvalues (descending); the top L columns of U
  if (tid < m) {
    const float la = S[tid * SD + tid].x;
    int rk = 0;
    for (int b = 0; b < m; ++b) {
      const float lb = S[b * SD + b].x;
      rk += (lb > la) || (lb == la && b < tid);
    }
    pq[rk] = tid;
  }
  __syncthreads();

  // The kept columns and the next one (Lw of them), in rank order,
  // orthonormalised against each other by warp 0 (modified Gram-Schmidt,
  // lanes over the rows): the close-pair rotation below would amplify their
  // mutual defect by lambda / gap.
  const int Lw = L < m ? L + 1 : m;
  if (warp == 0) {
    for (int r = 0; r < Lw; ++r) {
      const int cr = pq[r];
      for (int r2 = 0; r2 < r; ++r2) {
        const int c2 = pq[r2];
        float2 pr = cz();
        for (int a = lane; a < m; a += 32) cmacc(pr, U[a * SD + cr], U[a * SD + c2]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          pr.x += __shfl_xor_sync(FULL, pr.x, o);
          pr.y += __shfl_xor_sync(FULL, pr.y, o);
        }
        for (int a = lane; a < m; a += 32) cms(U[a * SD + cr], pr, U[a * SD + c2]);
        __syncwarp();
      }
      float nb = 0.f;
      for (int a = lane; a < m; a += 32) nb += cabs2(U[a * SD + cr]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(FULL, nb, o);
      const float sc = nb > 0.f ? 1.f / sqrtf(nb) : 1.f;
      for (int a = lane; a < m; a += 32) U[a * SD + cr] = cscale(U[a * SD + cr], sc);
      __syncwarp();
    }
  }
  __syncthreads();

  // 4. W rows r < Lw: W[r][c] = sum_b conj(U[b][idx_r]) H~[b][c] (reuses Hc)
  float2* W = Hc;
  for (int idx = tid; idx < Lw * n; idx += nth) {
    const int r = idx / n, c = idx - r * n;
    const int col = pq[r];
    float2 v = cz();
    for (int b = 0; b < m; ++b) cmacc(v, H[(size_t)b * n + c], U[b * SD + col]);
    W[r * n + c] = v;
  }
  __syncthreads();
  // Close pairs among the kept vectors and the first discarded one
  // (eigenvalues of rank r and r + 1 within kPolishWindow lambda_1): the
  // rows of W are rotated once more from their 2 x 2 Gram accumulated in
  // double-float, as in the register precoder, by warp 0 (lanes over the
  // columns of W and the rows of U).
  // With at most 16 rows, pairs closer than kPrecoderCloseGap lambda_1, the
  // first discarded eigenvalue included, list the unit (with its vectors of
  // ranks 0 .. min(L + 1, m) - 1, after this step) for the double-float
  // refinement.
  if (warp == 0) {
    const float lmax = S[pq[0] * SD + pq[0]].x;
    int close_mask = 0;                     // bit r: the pair (r, r + 1) is close
    if (A.list_close && m <= 16)
      for (int r = 0; r < L && r + 1 < m; ++r) {
        const float lr = S[pq[r] * SD + pq[r]].x, ls = S[pq[r + 1] * SD + pq[r + 1]].x;
        if (lr - ls < kPrecoderCloseGap * lmax && ls >= kPrecoderWeak * lmax) close_mask |= 1 << r;
      }
    for (int r = 0; r + 1 < Lw; ++r) {
      const int cp = pq[r], cq = pq[r + 1];
      if (!(S[cp * SD + cp].x - S[cq * SD + cq].x < kPolishWindow * lmax)) continue;
      float alh = 0.f, all = 0.f, beh = 0.f, bel = 0.f;
      float2 gah = cz(), gal = cz();
      for (int c = lane; c < n; c += 32) {
        const float2 x = W[r * n + c], y = W[(r + 1) * n + c];
        df_add_prod(alh, all, x.x, x.x);
        df_add_prod(alh, all, x.y, x.y);
        df_add_prod(beh, bel, y.x, y.x);
        df_add_prod(beh, bel, y.y, y.y);
        df_cmacc(gah, gal, x, y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        df_add(alh, all, __shfl_xor_sync(FULL, alh, o), __shfl_xor_sync(FULL, all, o));
        df_add(beh, bel, __shfl_xor_sync(FULL, beh, o), __shfl_xor_sync(FULL, bel, o));
        df_add(gah.x, gal.x, __shfl_xor_sync(FULL, gah.x, o), __shfl_xor_sync(FULL, gal.x, o));
        df_add(gah.y, gal.y, __shfl_xor_sync(FULL, gah.y, o), __shfl_xor_sync(FULL, gal.y, o));
      }
      const float dba = __fadd_rn(__fsub_rn(beh, alh), __fsub_rn(bel, all));
      const float gx = gah.x + gal.x, gy = gah.y + gal.y;
      const float ab = sqrtf(fmaf(gx, gx, gy * gy));
      if (ab > 0.f && ab > 1e-12f * sqrtf(alh) * sqrtf(beh)) {
        const float tau = dba / (2.f * ab);
        const float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
        const float cr = 1.f / sqrtf(fmaf(t, t, 1.f));
        const float sr = t * cr;
        const float2 e = make_float2(gx / ab, gy / ab);
        const float2 se = cscale(e, sr), sec = cscale(cconj(e), sr);
        for (int c = lane; c < n; c += 32) {           // W <- J* W (rows r, r + 1)
          const float2 x = W[r * n + c], y = W[(r + 1) * n + c];
          float2 nx = cscale(x, cr), ny = cscale(y, cr);
          cms(nx, se, y);
          cmac(ny, sec, x);
          W[r * n + c] = nx;
          W[(r + 1) * n + c] = ny;
        }
        for (int a = lane; a < m; a += 32) {           // U <- U J (columns p, q)
          const float2 x = U[a * SD + cp], y = U[a * SD + cq];
          float2 nx = cscale(x, cr), ny = cscale(y, cr);
          cms(nx, sec, y);
          cmac(ny, se, x);
          U[a * SD + cp] = nx;
          U[a * SD + cq] = ny;
        }
      }
      __syncwarp();
    }
    int pos = -1;
    if (close_mask != 0 && lane == 0) pos = atomicAdd(A.rcount, 1);
    pos = __shfl_sync(FULL, pos, 0);
    if (pos >= 0 && pos < A.J * K) {
      const int R = min(L + 1, m);
      for (int i2 = lane; i2 < R * m; i2 += 32) {
        const int r = i2 / m, a = i2 - r * m;
        A.Uclose[((size_t)pos * R + r) * m + a] = U[a * SD + pq[r]];
      }
      if (lane == 0) {
        A.rlist[pos] = k * K + kap;
        A.close_mask[pos] = close_mask;
      }
    }
  }
  __syncthreads();
  float s2[LT];
  bool deficient = false;
#pragma unroll
  for (int r = 0; r < LT; ++r) {
    float part = 0.f;
    if (r < L)
      for (int c = tid; c < n; c += nth) part += cabs2(W[r * n + c]);
    s2[r] = block_sum(part, red);
    deficient |= (r < L) && !(s2[r] > 0.f);
  }
  // 5. V~[:, r] = conj(W row r) / sigma_r, E_kk = U_L Sigma_L, flags
  float2* Vout = A.V + ((size_t)k * K + kap) * n * L;
  for (int idx = tid; idx < n * L; idx += nth) {
    const int c = idx / L, r = idx - c * L;
    float inv = 0.f;
#pragma unroll
    for (int rr = 0; rr < LT; ++rr)
      if (rr == r) inv = s2[rr] > 0.f ? rsqrtf(s2[rr]) : 0.f;
    Vout[idx] = cscale(cconj(W[r * n + c]), inv);
  }
  float2* Eout = A.Eserv + ((size_t)k * K + kap) * m * L;
  for (int idx = tid; idx < m * L; idx += nth) {
    const int a = idx / L, r = idx - a * L;
    float sg = 0.f;
#pragma unroll
    for (int rr = 0; rr < LT; ++rr)
      if (rr == r) sg = s2[rr] > 0.f ? sqrtf(s2[rr]) : 0.f;
    Eout[idx] = cscale(U[a * SD + pq[r]], sg);
  }
  if (tid == 0)
    A.pflag[(size_t)k * K + kap] = (deficient ? TS_FLAG_RANK_DEFICIENT : 0) |
                                   (converged ? 0 : TS_FLAG_EIG_UNCONVERGED);
}

// In-place Cholesky (lower) of the m x m Hermitian matrix in R (row stride
// SD) by the CTA; false if a pivot was not positive (replaced by 1).
__device__ bool chol_block(float2* R, int m, int SD, int* bad) {
  const int tid = threadIdx.x, nth = blockDim.x;
  if (tid == 0) *bad = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (tid == 0) {
      float d = R[j * SD + j].x;
      if (!(d > 0.f)) { *bad = 1; d = 1.f; }
      R[j * SD + j] = make_float2(sqrtf(d), 0.f);
    }
    __syncthreads();
    const float inv = 1.f / R[j * SD + j].x;
    for (int i = j + 1 + tid; i < m; i += nth) R[i * SD + j] = cscale(R[i * SD + j], inv);
    __syncthreads();
    const int w = m - j - 1;
    for (int t = tid; t < w * w; t += nth) {
      const int i = j + 1 + t / w, kk = j + 1 + t % w;
      if (kk <= i) cms(R[i * SD + kk], R[i * SD + j], cconj(R[kk * SD + j]));
    }
    __syncthreads();
  }
  return *bad == 0;
}

// Lower-triangular solves with the FP32 factor in R (row stride SD), thread
// r on column r of the m x L right-hand side in X (row stride L), in place:
// X <- L^{-1} X, then (conjT) X <- L^{-*} X.
__device__ void solve_lower(const float2* R, int SD, int m, float2* X, int L, int r) {
  for (int a = 0; a < m; ++a) {
    float2 v = X[a * L + r];
    for (int b = 0; b < a; ++b) cms(v, R[a * SD + b], X[b * L + r]);
    X[a * L + r] = cscale(v, 1.f / R[a * SD + a].x);
  }
}
__device__ void solve_lower_conjT(const float2* R, int SD, int m, float2* X, int L, int r) {
  for (int a = m - 1; a >= 0; --a) {
    float2 v = X[a * L + r];
    for (int b = a + 1; b < m; ++b) cmsc(v, X[b * L + r], R[b * SD + a]);   // v -= conj(L[b][a]) x_b
    X[a * L + r] = cscale(v, 1.f / R[a * SD + a].x);
  }
}

__device__ __forceinline__ void dmac_l(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

// Finalisation of one unit with m up to 64 rows (eq. 25-28).  With many
// rows the interference covariance R = sum_{k != i} E_ik E_ik* + sigma^2 I
// has a wide spectrum (a low-rank interference on sigma^2 I), and its FP32
// rounding alone moves the SINR by u ||R|| / sigma^2 ~ 1e-5, so every unit
// is evaluated the accurate way:
//   1. R in double-float from the stored FP32 effective channels (each
//      product exact, the sums compensated), shared memory Rh + Rl;
//   2. Cholesky of the FP32 part Rh (chol_block), Y = R^{-1} E_ii with that
//      factor, refined three times with residuals E_ii - R Y in FP64;
//   3. F = I + E_ii* Y (L x L) and its Cholesky factor in FP64,
//      x_r = [F^{-1}]_rr, SINR_r = (1 - x_r) / x_r (the identity form of
//      eq. 5, exact in FP64 for the refined Y).
// TS_FLAG_REFINED is set on every unit of this path.
struct LargeFinPlan {
  int SD, off_Rh, off_Rl, off_Lf, off_E, off_Es, off_X, off_Yd, off_F, off_misc, total;  // float2 units
};
__host__ __device__ inline LargeFinPlan large_fin_plan(int m, int L, int LT) {
  LargeFinPlan pl;
  pl.SD = m + 1;
  int o = 0;
  pl.off_Rh = o; o += m * pl.SD;
  pl.off_Rl = o; o += m * pl.SD;
  pl.off_Lf = o; o += m * pl.SD;
  pl.off_E = o; o += m * L;
  pl.off_Es = o; o += m * L;                 // one interferer's E, then the residual
  pl.off_X = o; o += m * L;
  o = (o + 1) & ~1;
  pl.off_Yd = o; o += 2 * m * L;             // double2
  pl.off_F = o; o += 2 * LT * LT;            // double2
  pl.off_misc = o; o += 2 * LT + 4;          // x_r (double), flag
  pl.total = o;
  return pl;
}

template <int MG, int LT, bool SVD>
__global__ void __launch_bounds__(kLargeThreads) k_sinr_finalize_large(const SinrArgs A,
                                                                       const LargeFinPlan pl) {
  extern __shared__ __align__(16) float2 sm[];
  const int m = A.m, L = A.L, K = A.K, J = A.J;
  const int kap = blockIdx.x, i = blockIdx.y;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int SD = pl.SD;
  float2* Rh = sm + pl.off_Rh;
  float2* Rl = sm + pl.off_Rl;
  float2* Lf = sm + pl.off_Lf;
  float2* E = sm + pl.off_E;
  float2* Es = sm + pl.off_Es;
  float2* X = sm + pl.off_X;
  double2* Yd = reinterpret_cast<double2*>(sm + pl.off_Yd);
  double2* F = reinterpret_cast<double2*>(sm + pl.off_F);
  double* xs = reinterpret_cast<double*>(sm + pl.off_misc);
  int* bad = reinterpret_cast<int*>(xs + LT);

  for (int idx = tid; idx < m * L; idx += nth) E[idx] = A.Eserv[((size_t)i * K + kap) * m * L + idx];
  // 1. R = sigma^2 I + sum_s E_s E_s*, lower triangle, double-float
  const float sg = A.sigma2[i];
  for (int idx = tid; idx < m * m; idx += nth) {
    const int a = idx / m, b = idx - a * m;
    Rh[a * SD + b] = make_float2(a == b ? sg : 0.f, 0.f);
    Rl[a * SD + b] = cz();
  }
  for (int s = 0; s < J - 1; ++s) {
    __syncthreads();                             // previous interferer consumed
    for (int idx = tid; idx < m * L; idx += nth)
      Es[idx] = A.Eint[(((size_t)i * (J - 1) + s) * K + kap) * m * L + idx];
    __syncthreads();
    for (int idx = tid; idx < m * m; idx += nth) {
      const int a = idx / m, b = idx - a * m;
      if (b > a) continue;
      float2 h = Rh[a * SD + b], lo = Rl[a * SD + b];
      for (int l = 0; l < L; ++l) df_cmacc(h, lo, Es[a * L + l], Es[b * L + l]);
      Rh[a * SD + b] = h;
      Rl[a * SD + b] = lo;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < m * m; idx += nth) {
    const int a = idx / m, b = idx - a * m;
    if (b <= a) Lf[a * SD + b] = Rh[a * SD + b];
  }
  __syncthreads();
  // 2. factor, solve, refine
  bool ok = chol_block(Lf, m, SD, bad);
  for (int idx = tid; idx < m * L; idx += nth) X[idx] = E[idx];
  __syncthreads();
  if (tid < L) {
    solve_lower(Lf, SD, m, X, L, tid);
    solve_lower_conjT(Lf, SD, m, X, L, tid);
  }
  __syncthreads();
  for (int idx = tid; idx < m * L; idx += nth) Yd[idx] = make_double2(X[idx].x, X[idx].y);
  for (int it = 0; it < 3; ++it) {
    __syncthreads();
    // residual E - R Y in FP64 (R Hermitian: entries above the diagonal
    // are the conjugates of the stored lower triangle)
    for (int idx = tid; idx < m * L; idx += nth) {
      const int a = idx / L, r = idx - a * L;
      double2 acc = make_double2(E[idx].x, E[idx].y);
      for (int b = 0; b < m; ++b) {
        const bool lower = b <= a;
        const int at = lower ? a * SD + b : b * SD + a;
        double2 rv = make_double2((double)Rh[at].x + (double)Rl[at].x, (double)Rh[at].y + (double)Rl[at].y);
        if (!lower) rv.y = -rv.y;
        dmac_l(acc, make_double2(-rv.x, -rv.y), Yd[b * L + r]);
      }
      X[idx] = make_float2((float)acc.x, (float)acc.y);
    }
    __syncthreads();
    if (tid < L) {
      solve_lower(Lf, SD, m, X, L, tid);
      solve_lower_conjT(Lf, SD, m, X, L, tid);
    }
    __syncthreads();
    for (int idx = tid; idx < m * L; idx += nth) {
      Yd[idx].x += X[idx].x;
      Yd[idx].y += X[idx].y;
    }
  }
  __syncthreads();
  // 3. F = I + E* Y (FP64), its factor, x_r
  for (int idx = tid; idx < L * L; idx += nth) {
    const int r = idx / L, s = idx - r * L;
    double2 v = make_double2(r == s ? 1.0 : 0.0, 0.0);
    for (int a = 0; a < m; ++a) dmac_l(v, make_double2(E[a * L + r].x, -E[a * L + r].y), Yd[a * L + s]);
    F[r * LT + s] = v;
  }
  __syncthreads();
  if (tid == 0) {
    int fbad = 0;
    for (int j = 0; j < L; ++j) {
      double d = F[j * LT + j].x;
      for (int t = 0; t < j; ++t) d -= F[j * LT + t].x * F[j * LT + t].x + F[j * LT + t].y * F[j * LT + t].y;
      if (!(d > 0.0)) { fbad = 1; d = 1.0; }
      const double ljj = sqrt(d);
      F[j * LT + j] = make_double2(ljj, 0.0);
      for (int r = j + 1; r < L; ++r) {
        double2 v = F[r * LT + j];
        for (int t = 0; t < j; ++t) {
          const double2 x = F[r * LT + t], y = F[j * LT + t];
          v.x -= x.x * y.x + x.y * y.y;
          v.y -= x.y * y.x - x.x * y.y;
        }
        F[r * LT + j] = make_double2(v.x / ljj, v.y / ljj);
      }
    }
    if (fbad) *bad = 1;
  }
  __syncthreads();
  ok = ok && *bad == 0;
  if (tid < L) {
    // x_r = |L_F^{-1} e_r|^2 by forward substitution from row r
    double2 y[LT];
    double x = 0.0;
#pragma unroll
    for (int s = 0; s < LT; ++s) {
      y[s] = make_double2(0.0, 0.0);
      if (s < tid || s >= L) continue;
      double2 v = make_double2(s == tid ? 1.0 : 0.0, 0.0);
#pragma unroll
      for (int t = 0; t < LT; ++t)
        if (t >= tid && t < s) {
          const double2 l = F[s * LT + t];
          v.x -= l.x * y[t].x - l.y * y[t].y;
          v.y -= l.x * y[t].y + l.y * y[t].x;
        }
      const double lss = F[s * LT + s].x;
      y[s] = make_double2(v.x / lss, v.y / lss);
      x += y[s].x * y[s].x + y[s].y * y[s].y;
    }
    xs[tid] = x;
  }
  __syncthreads();

  uint8_t pf = 0;
  if (SVD)
    for (int kk = 0; kk < J; ++kk) pf |= A.pflag[(size_t)kk * K + kap];
  const bool valid = ok && !(pf & TS_FLAG_TIMEOUT);
  bool finite = true;
  for (int r = 0; r < L; ++r) {
    const float sv = valid ? (float)((1.0 - xs[r]) / xs[r]) : __int_as_float(0x7fc00000);
    finite = finite && isfinite(sv);
    if (tid == 0) A.sinr[((size_t)i * K + kap) * L + r] = sv;
  }
  if (A.flags != nullptr && tid == 0) {
    uint8_t f = ok ? TS_FLAG_REFINED : TS_FLAG_NOT_PD;
    if (valid && !finite) f |= TS_FLAG_NONFINITE;
    A.flags[(size_t)i * K + kap] = f | pf;
  }
}

template <int MG, int LT>
cudaError_t large_precoder(const SinrArgs& A, cudaStream_t s) {
  const LargePrecPlan pl = large_prec_plan(A.m, A.n, A.L);
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget || A.Hserv == nullptr) return cudaErrorInvalidValue;
  auto kern = k_svd_precoder_large<MG, LT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(A.K, A.J), kLargeThreads, smem, s>>>(A, pl);
  return cudaGetLastError();
}

template <int MG, int LT>
cudaError_t large_finalize(const SinrArgs& A, bool svd, cudaStream_t s) {
  const LargeFinPlan pl = large_fin_plan(A.m, A.L, LT);
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget) return cudaErrorInvalidValue;
  auto kern = svd ? k_sinr_finalize_large<MG, LT, true> : k_sinr_finalize_large<MG, LT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(A.K, A.J), kLargeThreads, smem, s>>>(A, pl);
  return cudaGetLastError();
}

}  // namespace

// The dispatch templates of sinr_impl.cuh, specialised for 32 and 64 rows.
#define TS_LARGE_INSTANCES(MG, LT)                                                         \
  template <>                                                                              \
  cudaError_t run_precoder<MG, LT>(const SinrArgs& A, cudaStream_t s) {                    \
    return large_precoder<MG, LT>(A, s);                                                   \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t run_serving<MG, LT>(const SinrArgs& A, cudaStream_t s) {                     \
    return launch_link_wide<MG, LT, true>(A, s);                                           \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t run_rebuild<MG, LT>(const SinrArgs&, cudaStream_t) {                         \
    return cudaErrorInvalidValue;                                                          \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t run_links<MG, LT>(const SinrArgs& A, bool svd, cudaStream_t s) {             \
    return svd ? launch_link_wide<MG, LT, false>(A, s) : cudaErrorInvalidValue;            \
  }                                                                                        \
  template <>                                                                              \
  cudaError_t run_finalize<MG, LT>(const SinrArgs& A, bool svd, cudaStream_t s) {          \
    return large_finalize<MG, LT>(A, svd, s);                                              \
  }

}  // namespace detail

cudaError_t launch_precoder_staged(const SinrArgs& a, cudaStream_t s) {
  using namespace detail;
  if (a.m > kMaxRankM || a.L > 8) return cudaErrorInvalidValue;
  return a.L <= 2 ? large_precoder<16, 2>(a, s)
                  : a.L <= 4 ? large_precoder<16, 4>(a, s) : large_precoder<16, 8>(a, s);
}

namespace detail {

TS_LARGE_INSTANCES(32, 2)
TS_LARGE_INSTANCES(32, 4)
TS_LARGE_INSTANCES(32, 8)
TS_LARGE_INSTANCES(64, 2)
TS_LARGE_INSTANCES(64, 4)
TS_LARGE_INSTANCES(64, 8)
#undef TS_LARGE_INSTANCES

}  // namespace detail
}  // namespace ts
