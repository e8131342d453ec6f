// Wide-core link kernel of the SVD path (included by sinr_impl.cuh, whose
// helpers it uses: path_coef, the cp.async wrappers, kThreads, kSmemBudget).
#pragma once

namespace ts {
namespace detail {

// Wide-core variant of the blocked link pass, for ranks beyond what the
// narrow kernels stage (p > 32 or P p > 8192): the paper's compressed sizes
// (p ~ 100-200 of P ~ 400 paths) and the dense-channel comparator at large P.
// Each lane holds X subcarriers and 4 / X rows of a unit: X = 2 as in
// k_sinr_link_blk; X = 4 (one row) for 64-row units, whose 64 lanes then
// read each core row from shared memory once per q for four subcarriers.
// NT threads per CTA: 256 for 64-row units (16 subcarriers per CTA, so that
// each core slab brought in serves 16), else 128.  The projection w = c* C
// streams C_ik and the path coefficients through shared memory in
// double-buffered chunks of PC paths and keeps w [T][p] in shared memory; the core then streams in stages of (column
// chunk, kWideQC slabs G[q]), double-buffered, and the H~ accumulators of a
// column chunk persist across its slabs.  Dense-channel comparator (C = I,
// p = P): w = c* is evaluated per stage into the stage buffer instead.
// SERVE: the serving link (k = i), whose rows H~_ii(kappa) go to Hserv for
// the precoder kernel, with the column chunks split over grid z (columns are
// independent there); otherwise the interfering links' partial covariances,
// as in k_sinr_link_blk.
constexpr int kWideQC = 16;

struct WidePlan {
  int T, QR, SG, SV, WS, PC, wide, cps;
  int off_ws, off_stage, stage, off_Gs, off_Vs, off_Wc, proj, off_Cc, off_cc, total;
};

// QR: the columns of w = c* C held at once (p, or a multiple of 32 below p:
// the link pass then runs in p / QR passes over the core, each accumulating
// E += H~[q-range] V~, which is linear in the core's mode-3 slabs).
__host__ __device__ inline WidePlan wide_plan(int MG, int LT, int p, bool identity, bool serve,
                                              int PC, int QR, int NT = kThreads, int X = 2) {
  constexpr int NC = 4;
  WidePlan pl;
  pl.T = 2 * NT / (MG / 2);
  pl.QR = QR;
  pl.SG = NC + 2;
  pl.SV = NC * LT + 2;
  pl.WS = kWideQC + 1;
  pl.PC = PC;
  pl.wide = 0;
  pl.cps = 1 << 30;
  int o = 0;
  pl.off_ws = o;
  if (!identity) o += pl.T * (QR + 1);
  o = (o + 1) & ~1;
  pl.off_stage = o;
  int so = 0;
  pl.off_Gs = so; so += kWideQC * MG * pl.SG;
  pl.off_Vs = so; if (!serve) so += pl.T * pl.SV;
  pl.off_Wc = so; if (identity) so += pl.T * pl.WS;
  so = (so + 1) & ~1;
  pl.stage = so;
  // projection buffers (C chunk [PC][QR], coefficient chunk [T][PC + 1]),
  // sharing the region of the stage buffers (used one after the other)
  pl.off_Cc = 0;
  pl.off_cc = (PC * QR + 1) & ~1;
  pl.proj = identity ? 0 : ((pl.off_cc + pl.T * (PC + 1) + 1) & ~1);
  const int es = (NT * (4 / X) / MG) * (X * MG * LT + 2);
  int region = 2 * so > es ? 2 * so : es;
  if (2 * pl.proj > region) region = 2 * pl.proj;
  o += region;
  pl.total = o;
  return pl;
}

template <int MG, int LT, bool SERVE, int NT, int X>
__global__ void __launch_bounds__(NT, NT > kThreads ? 2 : 0) k_sinr_link_wide(const SinrArgs A,
                                                                              const WidePlan pl) {
  constexpr int NC = 4;
  constexpr int R = 4 / X;                  // rows per lane
  constexpr int GL = MG / R;                // lanes per subcarrier group
  constexpr int T = X * NT / GL;
  constexpr int QS = NT / T;                // threads per subcarrier in the projection
  constexpr int QA = 32 / QS;               // projection outputs per thread and 32-column block
  constexpr int QC = kWideQC;
  extern __shared__ __align__(16) float2 sm[];
  const int tid = threadIdx.x;
  const int gp = tid / GL, j = tid % GL;
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * T;
  const int J = A.J, m = A.m, n = A.n, p = A.p, L = A.L, K = A.K, P = A.P;
  const int k = SERVE ? i : (z < i ? z : z + 1);
  const int ch = i * J + k;
  const int QR = pl.QR;
  const int nchunk = (n + NC - 1) / NC;
  const int cbeg = SERVE ? z * pl.cps : 0;
  const int cend = SERVE ? min(nchunk, cbeg + pl.cps) : nchunk;
  const bool ident = A.identity_C;
  float2* ws = sm + pl.off_ws;
  float2* stage0 = sm + pl.off_stage;
  const bool wide = pl.wide != 0;
  if (!SERVE && A.rcount != nullptr && tid == 0 && blockIdx.x == 0 && i == 0 && z == 0) *A.rcount = 0;
  if (cend <= cbeg) return;                 // an empty column slice (uniform over the CTA)

  // c_q(kappa) of this link (dense tile or path form), from global memory
  auto coef_at = [&](int kap, int q) -> float2 {
    return A.coef_mode == 0 ? A.coef[((size_t)ch * A.Kc + A.kap_off + kap) * P + q]
                            : path_coef(__ldg(A.coef + (size_t)ch * P + q),
                                        __ldg(A.turns + (size_t)ch * P + q), A.kap_off + kap);
  };

  // the current pass: columns [qlo, qlo + qn) of w, nq slabs per column chunk
  int qlo = 0, qn = 0, nq = 1;
  auto issue_stage = [&](int st) {
    float2* buf = stage0 + (st & 1) * pl.stage;
    const int cidx = cbeg + st / nq, qi = st % nq;
    const int c0 = cidx * NC, q0 = qlo + qi * QC;
    const int qc = min(QC, qlo + qn - q0);
    const float2* Gch = A.G + (size_t)ch * p * m * n;
    if (wide) {
      constexpr int GU = MG * NC / 2;                 // 16-byte units per slab
      const int cc = 2 * (tid % (NC / 2)), aa = (tid / (NC / 2)) % MG;
      const bool rowok = aa < m && c0 + cc < n;
      for (int ql = tid / GU; ql < qc; ql += NT / GU)
        cp_async16(buf + pl.off_Gs + (ql * MG + aa) * pl.SG + cc,
                   rowok ? Gch + ((size_t)(q0 + ql) * m + aa) * n + c0 + cc : A.G, rowok);
      if (!SERVE && qi == nq - 1) {
        constexpr int VU = NC * LT / 2;
        const int l = 2 * (tid % (LT / 2)), vc = (tid / (LT / 2)) % NC;
        const bool colok = c0 + vc < n && l < L;
        for (int t = tid / VU; t < T; t += NT / VU) {
          const bool ok = colok && kap0 + t < K;
          cp_async16(buf + pl.off_Vs + t * pl.SV + vc * LT + l,
                     ok ? A.V + (((size_t)k * K + kap0 + t) * n + c0 + vc) * L + l : A.V, ok);
        }
      }
    } else {
      for (int idx = tid; idx < qc * MG * NC; idx += NT) {
        const int cc = idx % NC, aa = (idx / NC) % MG, ql = idx / (NC * MG);
        const int c = c0 + cc;
        const bool ok = aa < m && c < n;
        cp_async8(buf + pl.off_Gs + (ql * MG + aa) * pl.SG + cc,
                  ok ? Gch + ((size_t)(q0 + ql) * m + aa) * n + c : A.G, ok);
      }
      if (!SERVE && qi == nq - 1) {
        for (int idx = tid; idx < T * NC * LT; idx += NT) {
          const int l = idx % LT, cc = (idx / LT) % NC, t = idx / (LT * NC);
          const int kk2 = kap0 + t, c = c0 + cc;
          const bool ok = kk2 < K && c < n && l < L;
          cp_async8(buf + pl.off_Vs + t * pl.SV + cc * LT + l,
                    ok ? A.V + (((size_t)k * K + kk2) * n + c) * L + l : A.V, ok);
        }
      }
    }
    if (ident) {
      // dense channel: w_q = conj(c_q(kappa)) for the slab
      for (int idx = tid; idx < T * qc; idx += NT) {
        const int t = idx / qc, ql = idx - t * qc;
        buf[pl.off_Wc + t * pl.WS + ql] = kap0 + t < K ? cconj(coef_at(kap0 + t, q0 + ql)) : cz();
      }
    }
  };

  float2 E[X][R][LT];   // [subcarrier X gp + x][row j + r GL][stream]
#pragma unroll
  for (int x = 0; x < X; ++x)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int l = 0; l < LT; ++l) E[x][r][l] = cz();
  float2 h[X][R][NC];

  for (qlo = 0; qlo < p; qlo += QR) {
    qn = min(QR, p - qlo);
    nq = (qn + QC - 1) / QC;
    const int nstage = (cend - cbeg) * nq;
    if (SERVE && A.Wserv != nullptr) {
      // the serving links' projections come from k_wide_proj (one pass)
      const float2* src = A.Wserv + ((size_t)i * K + kap0) * p;
      for (int idx = tid; idx < T * p; idx += NT) {
        const int t = idx / p, q = idx - t * p;
        ws[t * (QR + 1) + q] = kap0 + t < K ? src[idx] : cz();
      }
    } else if (!ident) {
      // projection w[t][q] = sum_P C[P][q] conj(c_P(kappa_t)) (eq. 15) for
      // the pass's columns, in chunks of PC paths: C rows by asynchronous
      // copies, coefficients evaluated into shared memory, one chunk ahead
      // of the accumulation.  Thread (t, qs) owns columns qb + qs QA + u of
      // each 32-column block.
      const int PC = pl.PC;
      const int npc = (P + PC - 1) / PC;
      const float2* Cch = A.C + (size_t)ch * P * p + qlo;
      const bool c16 = (p % 2 == 0) && (((uintptr_t)A.C & 15u) == 0);
      auto issue_proj = [&](int ci) {
        float2* buf = stage0 + (ci & 1) * pl.proj;
        const int P0 = ci * PC, pc = min(PC, P - P0);
        const float2* src = Cch + (size_t)P0 * p;
        if (c16) {
          for (int idx = 2 * tid; idx < pc * qn; idx += 2 * NT) {
            const int row = idx / qn, col = idx - row * qn;
            cp_async16(buf + pl.off_Cc + row * QR + col, src + (size_t)row * p + col, true);
          }
        } else {
          for (int idx = tid; idx < pc * qn; idx += NT) {
            const int row = idx / qn, col = idx - row * qn;
            cp_async8(buf + pl.off_Cc + row * QR + col, src + (size_t)row * p + col, true);
          }
        }
        for (int idx = tid; idx < T * PC; idx += NT) {
          const int t = idx / PC, pp = idx - t * PC;
          buf[pl.off_cc + t * (PC + 1) + pp] =
              (pp < pc && kap0 + t < K) ? coef_at(kap0 + t, P0 + pp) : cz();
        }
      };
      const int t = tid / QS, qs = tid % QS;
      issue_proj(0);
      cp_async_commit();
      for (int ci = 0; ci < npc; ++ci) {
        if (ci + 1 < npc) issue_proj(ci + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const float2* buf = stage0 + (ci & 1) * pl.proj;
        const int pc = min(PC, P - ci * PC);
        const float2* crow = buf + pl.off_cc + t * (PC + 1);
        for (int qb = 0; qb < qn; qb += 32) {
          const int q0 = qb + qs * QA;
          if (q0 >= qn) continue;
          float2 acc[QA];
#pragma unroll
          for (int u = 0; u < QA; ++u) acc[u] = cz();
          const float2* Cb = buf + pl.off_Cc + q0;
          for (int pp = 0; pp < pc; ++pp) {
            const float2 c = crow[pp];
            const float2* Cr = Cb + pp * QR;
#pragma unroll
            for (int u = 0; u < QA; ++u)
              if (q0 + u < qn) cmacc(acc[u], Cr[u], c);
          }
          float2* wout = ws + t * (QR + 1) + q0;
#pragma unroll
          for (int u = 0; u < QA; ++u)
            if (q0 + u < qn) wout[u] = ci == 0 ? acc[u] : cadd(wout[u], acc[u]);
        }
        __syncthreads();     // this buffer is refilled two chunks later
      }
      cp_async_wait<0>();
    }

    issue_stage(0);
    cp_async_commit();
    if (nstage > 1) issue_stage(1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    for (int st = 0; st < nstage; ++st) {
      if (st > 0) {
        if (st + 1 < nstage) issue_stage(st + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
      }
      const float2* buf = stage0 + (st & 1) * pl.stage;
      const int cidx = cbeg + st / nq, qi = st % nq;
      const int q0 = qlo + qi * QC, qc = min(QC, qlo + qn - q0);
      if (qi == 0) {
#pragma unroll
        for (int x = 0; x < X; ++x)
#pragma unroll
          for (int r = 0; r < R; ++r)
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) h[x][r][cc] = cz();
      }
      const int wst = ident ? pl.WS : QR + 1;
      const float2* w0 = ident ? buf + pl.off_Wc + (X * gp) * pl.WS
                               : ws + (X * gp) * (QR + 1) + (q0 - qlo);
      const float2* g0 = buf + pl.off_Gs + j * pl.SG;
#pragma unroll 4
      for (int q = 0; q < qc; ++q) {
        float2 wv[X];
#pragma unroll
        for (int x = 0; x < X; ++x) wv[x] = w0[x * wst + q];
        const float2* gq = g0 + q * MG * pl.SG;
#pragma unroll
        for (int c2 = 0; c2 < NC / 2; ++c2) {
          float4 u[R];
#pragma unroll
          for (int r = 0; r < R; ++r) u[r] = reinterpret_cast<const float4*>(gq + r * GL * pl.SG)[c2];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float2 u0 = make_float2(u[r].x, u[r].y), u1 = make_float2(u[r].z, u[r].w);
#pragma unroll
            for (int x = 0; x < X; ++x) {
              cmac(h[x][r][2 * c2], wv[x], u0);
              cmac(h[x][r][2 * c2 + 1], wv[x], u1);
            }
          }
        }
      }
      if (qi == nq - 1) {
        const int c0 = cidx * NC;
        if (SERVE) {
#pragma unroll
          for (int x = 0; x < X; ++x) {
            const int kap = kap0 + X * gp + x;
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int a = j + r * GL;
              if (kap >= K || a >= m) continue;
              float2* Hrow = A.Hserv + (((size_t)i * K + kap) * m + a) * n;
#pragma unroll
              for (int cc = 0; cc < NC; ++cc)
                if (c0 + cc < n) Hrow[c0 + cc] = h[x][r][cc];
            }
          }
        } else {
          const float2* va = buf + pl.off_Vs + (X * gp) * pl.SV;
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
#pragma unroll
            for (int l2 = 0; l2 < LT / 2; ++l2) {
              float4 v[X];
#pragma unroll
              for (int x = 0; x < X; ++x) v[x] = reinterpret_cast<const float4*>(va + x * pl.SV + cc * LT)[l2];
#pragma unroll
              for (int r = 0; r < R; ++r)
#pragma unroll
                for (int x = 0; x < X; ++x) {
                  cmac(E[x][r][2 * l2], h[x][r][cc], make_float2(v[x].x, v[x].y));
                  cmac(E[x][r][2 * l2 + 1], h[x][r][cc], make_float2(v[x].z, v[x].w));
                }
            }
          }
        }
      }
      __syncthreads();   // this buffer is refilled two stages later
    }
    cp_async_wait<0>();
  }
  if (SERVE) return;

  // rows of the interfering effective channel E_ik (eq. 24) of this lane's
  // subcarriers; the finalisation forms the covariance of eq. (25)
#pragma unroll
  for (int x = 0; x < X; ++x) {
    const int kap = kap0 + X * gp + x;
    if (kap >= K) continue;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int a = j + r * GL;
      if (a >= m) continue;
      float2* Eout = A.Eint + ((((size_t)i * (J - 1) + z) * K + kap) * m + a) * L;
#pragma unroll
      for (int l = 0; l < LT; ++l)
        if (l < L) Eout[l] = E[x][r][l];
    }
  }
}

// Projections of the serving links for the wide-core serving pass, whose
// column slices would otherwise each recompute them: CTA (tile, BS i,
// 32-column block) accumulates w[t][q] = sum_P C_ii[P][q] conj(c_P(kappa_t))
// (eq. 15) in registers over double-buffered chunks of C rows and path
// coefficients, then writes Wserv[i][kappa][q].
constexpr int kProjT = 64;           // subcarriers per CTA
template <int T>
__global__ void __launch_bounds__(kThreads) k_wide_proj(const SinrArgs A, const WidePlan pl) {
  constexpr int QS = kThreads / T, QA = 32 / QS;
  extern __shared__ __align__(16) float2 sm[];
  const int tid = threadIdx.x;
  const int i = blockIdx.y;
  const int kap0 = blockIdx.x * T;
  const int qb = blockIdx.z * 32;
  const int J = A.J, p = A.p, K = A.K, P = A.P;
  const int ch = i * J + i;
  const int PC = pl.PC;
  const int npc = (P + PC - 1) / PC;
  const float2* Cch = A.C + (size_t)ch * P * p;
  const bool c16 = (p % 2 == 0) && (((uintptr_t)A.C & 15u) == 0);
  auto coef_at = [&](int kap, int q) -> float2 {
    return A.coef_mode == 0 ? A.coef[((size_t)ch * A.Kc + A.kap_off + kap) * P + q]
                            : path_coef(__ldg(A.coef + (size_t)ch * P + q),
                                        __ldg(A.turns + (size_t)ch * P + q), A.kap_off + kap);
  };
  auto issue = [&](int ci) {
    float2* buf = sm + (ci & 1) * pl.proj;
    const int P0 = ci * PC, pc = min(PC, P - P0);
    const float2* src = Cch + (size_t)P0 * p;
    if (c16) {
      for (int idx = 2 * tid; idx < pc * p; idx += 2 * kThreads)
        cp_async16(buf + pl.off_Cc + idx, src + idx, true);
    } else {
      for (int idx = tid; idx < pc * p; idx += kThreads) cp_async8(buf + pl.off_Cc + idx, src + idx, true);
    }
    for (int idx = tid; idx < T * PC; idx += kThreads) {
      const int t = idx / PC, pp = idx - t * PC;
      buf[pl.off_cc + t * (PC + 1) + pp] = (pp < pc && kap0 + t < K) ? coef_at(kap0 + t, P0 + pp) : cz();
    }
  };
  const int t = tid / QS, qs = tid % QS;
  const int q0 = qb + qs * QA;
  float2 acc[QA];
#pragma unroll
  for (int u = 0; u < QA; ++u) acc[u] = cz();
  issue(0);
  cp_async_commit();
  for (int ci = 0; ci < npc; ++ci) {
    if (ci + 1 < npc) issue(ci + 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float2* buf = sm + (ci & 1) * pl.proj;
    const int pc = min(PC, P - ci * PC);
    const float2* crow = buf + pl.off_cc + t * (PC + 1);
    const float2* Cb = buf + pl.off_Cc + q0;
    if (q0 < p) {
      for (int pp = 0; pp < pc; ++pp) {
        const float2 c = crow[pp];
        const float2* Cr = Cb + pp * p;
#pragma unroll
        for (int u = 0; u < QA; ++u)
          if (q0 + u < p) cmacc(acc[u], Cr[u], c);
      }
    }
    __syncthreads();     // this buffer is refilled two chunks later
  }
  cp_async_wait<0>();
  if (kap0 + t < K) {
    float2* out = A.Wserv + ((size_t)i * K + kap0 + t) * p;
#pragma unroll
    for (int u = 0; u < QA; ++u)
      if (q0 + u < p) out[q0 + u] = acc[u];
  }
}

template <int MG, int LT, bool SERVE>
cudaError_t launch_link_wide(const SinrArgs& A, cudaStream_t s) {
  if (!SERVE && A.J < 2) return cudaSuccess;
  // 64-row units: 256 threads (at most 128 registers, two CTAs per SM), so
  // that each core slab brought into shared memory serves 16 subcarriers
  // instead of 8, with one row and four subcarriers per lane (26.7 -> 19.4
  // ms for the 420 links of (60, 230, 150) units; 32-row units already hold
  // 16 subcarriers per 128-thread CTA)
  constexpr int NT = (!SERVE && MG >= 64) ? 2 * kThreads : kThreads;
  constexpr int X = MG >= 64 ? 4 : 2;
  // shared memory decides how many CTAs share an SM (128 threads: 3 within
  // 75 KB, 2 within 113 KB; 256 threads, at most 128 registers: 2 within
  // 113 KB): take the
  // plan with the most CTAs per SM, then the fewest passes over the core
  // (columns of w held at once: p, or 128, 64, 32 for the interfering
  // links), then the largest projection chunk (16 .. 2 paths)
  const bool passes = !SERVE && !A.identity_C;
  WidePlan pl = wide_plan(MG, LT, A.p, A.identity_C, SERVE, 2, A.p, NT, X);
  int best_ctas = -1, best_passes = 1 << 30, best_pc = 0;
  for (int qr : {A.p, 128, 64, 32}) {
    if (qr != A.p && (!passes || qr >= A.p)) continue;
    const int npass = (A.p + qr - 1) / qr;
    for (int pc = 16; pc >= 2; pc /= 2) {
      const WidePlan t = wide_plan(MG, LT, A.p, A.identity_C, SERVE, pc, qr, NT, X);
      const size_t bytes = (size_t)t.total * sizeof(float2);
      if (bytes > kSmemBudget) continue;
      const int ctas = bytes <= 75 * 1024 && NT == kThreads ? 3 : bytes <= 113 * 1024 ? 2 : 1;
      if (ctas > best_ctas || (ctas == best_ctas && (npass < best_passes ||
                                                     (npass == best_passes && pc > best_pc)))) {
        best_ctas = ctas;
        best_passes = npass;
        best_pc = pc;
        pl = t;
      }
    }
  }
  const size_t smem = (size_t)pl.total * sizeof(float2);
  if (smem > kSmemBudget) return cudaErrorInvalidValue;
  pl.wide = (A.n % 2 == 0) && (A.L % 2 == 0) && (((uintptr_t)A.G & 15u) == 0) &&
            (((uintptr_t)A.V & 15u) == 0 || SERVE);
  const int tiles = (A.K + pl.T - 1) / pl.T;
  int nz = SERVE ? 1 : A.J - 1;
  if (SERVE && A.Wserv != nullptr) {
    // the projections once per (tile, serving link, 32 columns)
    int PCp = 16;
    WidePlan pp = wide_plan(8, 2, A.p, false, true, PCp, A.p);
    while (PCp > 2 && (size_t)2 * pp.proj * sizeof(float2) > kSmemBudget) {
      PCp /= 2;
      pp = wide_plan(8, 2, A.p, false, true, PCp, A.p);
    }
    const size_t psm = (size_t)2 * pp.proj * sizeof(float2);
    if (psm > kSmemBudget) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_wide_proj<kProjT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)psm);
    if (e != cudaSuccess) return e;
    dim3 pgrid((A.K + kProjT - 1) / kProjT, A.J, (A.p + 31) / 32);
    k_wide_proj<kProjT><<<pgrid, kThreads, psm, s>>>(A, pp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (SERVE) {
    // the serving links alone are J CTAs per tile: split their column
    // chunks so that about two CTAs per SM run
    const int nchunk = (A.n + 3) / 4;
    int slices = (2 * 152 + A.J * tiles - 1) / (A.J * tiles);
    if (slices > nchunk) slices = nchunk;
    if (slices < 1) slices = 1;
    pl.cps = (nchunk + slices - 1) / slices;
    nz = (nchunk + pl.cps - 1) / pl.cps;
  }
  dim3 grid(tiles, A.J, nz);
  auto kern = k_sinr_link_wide<MG, LT, SERVE, NT, X>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, NT, smem, s>>>(A, pl);
  return cudaGetLastError();
}

}  // namespace detail
}  // namespace ts
