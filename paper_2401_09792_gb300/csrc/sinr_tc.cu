// Interfering-link pass of the SVD-precoded SINR with the core contraction
// (eq. 15) on the tensor cores (tcgen05), in the reduced-precision modes:
//   TF32:    H~ = w (x) G with w and G rounded to TF32, FP32 accumulation;
//   BF16X2:  w = w_hi + w_lo, G = G_hi + G_lo in BF16 and
//            H~ = w_hi G_hi + w_lo G_hi + w_hi G_lo, FP32 accumulation.
// Everything else (projection w = c* C, effective channel E = H~ V~,
// covariance rows E E*) stays FP32 on the FMA pipe.
//
// The complex contraction over the p core slabs is one real GEMM per tile:
// rows = the T = 128 subcarriers of the tile (TMEM lanes), columns = (row a,
// column c, re/im) of H~, reduction over K = [Re w | Im w] (x3 segments for
// BF16X2) against the core rewritten once per call by k_core_prep as
//   re column: [Re G ; -Im G],   im column: [Im G ; Re G]
// (and [hi | hi | lo] segments for BF16X2).  Operands are K-major without
// swizzle in shared memory: 8-row x 16-byte core matrices, K-adjacent ones
// 128 bytes apart (LBO), row groups 128 * K_bytes / 16 bytes apart (SBO).
//
// Operands are prepared once per call: k_core_prep rewrites every link's
// core, k_tc_proj computes the projections w = c* C (FP32) of every
// interfering link and subcarrier tile and writes them rounded or split.
// Per CTA (tile, UE i, interfering BS k): the projection operand arrives by
// one bulk copy; the core is consumed in column blocks of CB columns of H~
// (CB = 4 for m <= 4, else 2; N = 2 MG CB accumulator columns), each block's
// operand fetched by one bulk copy (cp.async.bulk + mbarrier transaction
// count) into a three-slot ring two blocks ahead, and multiplied by one
// thread into one of two TMEM buffers one block ahead of the epilogue; the
// precoder rows of the block are staged by cp.async two blocks ahead.  The
// epilogue thread (row group g, subcarrier t) reads its RPT rows of the H~
// block from TMEM (tcgen05.ld) and accumulates E rows; at the end the E rows
// are exchanged through shared memory and the partial covariance rows
// written as in the FP32 kernel.  Every wait is bounded; on a timeout the
// tile's precoder flags get TS_FLAG_TIMEOUT and the kernel releases its TMEM
// and returns.
#include <cuda_bf16.h>

#include "sinr_impl.cuh"

namespace ts {
namespace detail {
namespace {

constexpr int kTile = 128;     // subcarriers per CTA = MMA M = TMEM lanes
constexpr int kBStages = 3;    // core-operand ring (loads run two blocks ahead)
constexpr long kSpinLimit = 1L << 24;

struct TcPlan {
  int ES;          // operand element bytes (4 TF32, 2 BF16)
  int Kpad;        // reduction length in elements, padded to 32 bytes
  int Ntile;       // accumulator columns per block = 2 MG CB
  int nblk;        // column blocks = ceil(n / CB)
  int SV;          // precoder stage row stride (float2), per subcarrier
  int off_A, off_B, off_V, off_bar, smem;   // byte offsets
  size_t prep_bytes_per_link;               // k_core_prep output per link
  size_t a_bytes_per_tile;                  // k_tc_proj output per (link, tile)
};

__host__ __device__ constexpr int tc_rpt(int MG) { return MG < 4 ? MG : 4; }
// H~ columns per accumulator block (N = 2 MG CB accumulator columns)
__host__ __device__ constexpr int tc_cb(int MG) { return MG >= 8 ? 2 : 4; }

inline TcPlan tc_plan(int MG, int LT, int n, int p, int prec) {
  TcPlan t;
  t.ES = prec == TS_PREC_TF32 ? 4 : 2;
  const int kused = prec == TS_PREC_TF32 ? 2 * p : 6 * p;
  const int kq = 32 / t.ES;                      // elements per 32 bytes
  t.Kpad = (kused + kq - 1) / kq * kq;
  const int CB = tc_cb(MG);
  t.Ntile = 2 * MG * CB;
  t.nblk = (n + CB - 1) / CB;
  t.SV = CB * LT + 2;
  int o = 0;
  t.off_A = o; o += kTile * t.Kpad * t.ES;
  t.off_B = o; o += kBStages * t.Ntile * t.Kpad * t.ES;
  t.off_V = o; o += 2 * kTile * t.SV * 8;
  // E exchange at the end reuses the front of the buffer
  const int ex = kTile * MG * (LT * 8) + kTile * 16;
  if (ex > o) o = ex;
  o = (o + 15) & ~15;
  t.off_bar = o; o += 64;
  t.smem = o;
  t.prep_bytes_per_link = (size_t)t.nblk * t.Ntile * t.Kpad * t.ES;
  t.a_bytes_per_tile = (size_t)kTile * t.Kpad * t.ES;
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// canonical K-major no-swizzle layout: byte offset of (row r, k-byte kb)
__host__ __device__ __forceinline__ uint32_t kmajor_off(int r, int kb, int kbytes) {
  return (uint32_t)((r >> 3) * (128 * (kbytes >> 4)) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;               // LBO: K-adjacent core matrices
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;    // SBO: row-group stride
  d |= (uint64_t)1 << 46;                        // descriptor version
  return d;                                      // base offset 0, no swizzle
}

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// bounded wait on an mbarrier phase; false on timeout
__device__ __forceinline__ bool mbar_wait_limit(uint32_t bar, uint32_t parity, long limit) {
  for (long it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_limit(bar, parity, kSpinLimit);
}

// Self-test of the bounded wait the tensor-core kernel relies on: one
// thread waits on phase 0 of an mbarrier of count 1 that nothing arrives at
// (arrive == 0) or that it arrives at first (arrive != 0), for at most
// `limit` tries; out[0] = 1 if the wait gave up, 0 if the phase completed.
__global__ void k_wait_selftest(long limit, int arrive, int* out) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_u32(&bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  if (arrive) {
    uint64_t tok;                                   // the arrival token (unused)
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(tok) : "r"(b) : "memory");
    asm volatile("" ::"l"(tok));
  }
  out[0] = mbar_wait_limit(b, 0, limit) ? 0 : 1;
}

// ------------------------------------------------------------ core operand
// B operand of link ch, column block b, in the canonical layout: row
// j = ((g CB + c) RPT + a_in) 2 + ri of the block (row a = g RPT + a_in,
// column c0 + c of H~), k over [Re w | Im w] (x3 segments for BF16X2):
//   re row: [Re G ; -Im G],   im row: [Im G ; Re G]
// (BF16X2: segments [hi | hi | lo]).  One thread writes one 16-byte chunk;
// eight consecutive threads fill one 128-byte core matrix; padding is zero.
template <int PREC>
__global__ void __launch_bounds__(256) k_core_prep(const float2* __restrict__ G, int m, int n, int p,
                                                   int MG, int Ntile, int Kpad, int nblk, int nblocks,
                                                   unsigned char* __restrict__ out) {
  // y = ch * nblk + b: one operand block; threads over its chunks
  constexpr int ES = PREC == TS_PREC_TF32 ? 4 : 2;
  constexpr int EPC = 16 / ES;
  const int kbytes = Kpad * ES, nkc = kbytes / 16;
  const int RPT = tc_rpt(MG), CB = tc_cb(MG);
  const int p2 = 2 * p, kused = PREC == TS_PREC_TF32 ? p2 : 3 * p2;
  const int nchunk = Ntile * nkc;
  for (int y = blockIdx.y; y < nblocks; y += gridDim.y)
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nchunk; idx += gridDim.x * blockDim.x) {
    const int ch = y / nblk, b = y - ch * nblk;
    unsigned char* blk = out + (size_t)y * Ntile * kbytes;
    const int r = idx & 7, rest = idx >> 3;
    const int rg = rest / nkc, kc = rest - rg * nkc;
    const int j = rg * 8 + r;
    const int ri = j & 1, a_in = (j >> 1) % RPT, cg = (j >> 1) / RPT;
    const int c = b * CB + cg % CB, a = (cg / CB) * RPT + a_in;
    const bool live = a < m && c < n;
    const float2* gcol = G + ((size_t)ch * p * m + a) * n + c;     // + q m n
    float2 gv[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      int kk = kc * EPC + e;
      kk = kk >= 2 * p2 ? kk - 2 * p2 : kk >= p2 ? kk - p2 : kk;
      const int q = kk < p ? kk : kk - p;
      gv[e] = live && kc * EPC + e < kused ? __ldg(gcol + (size_t)q * m * n) : cz();
    }
    float x[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      const int k = kc * EPC + e;
      const int kk = k >= 2 * p2 ? k - 2 * p2 : k >= p2 ? k - p2 : k;
      // re row: [Re G ; -Im G], im row: [Im G ; Re G]
      float v = ri == 0 ? (kk < p ? gv[e].x : -gv[e].y) : (kk < p ? gv[e].y : gv[e].x);
      if (PREC == TS_PREC_BF16X2 && k >= 2 * p2) v -= __bfloat162float(__float2bfloat16_rn(v));
      x[e] = v;
    }
    uint32_t words[4];
    if (PREC == TS_PREC_TF32) {
#pragma unroll
      for (int e = 0; e < 4; ++e) words[e] = __float_as_uint(to_tf32(x[e % EPC]));
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w)
        words[w] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[(2 * w) % EPC])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[(2 * w + 1) % EPC])) << 16);
    }
    *reinterpret_cast<uint4*>(blk + kmajor_off(j, kc * 16, kbytes)) =
        make_uint4(words[0], words[1], words[2], words[3]);
  }
}

// ------------------------------------------------------ projection operand
// A operand of (interfering link (i, k), subcarrier tile): row t =
// subcarrier kap0 + t, k over [Re w | Im w] with w = C_ik^T conj(c_ik(kappa))
// (eq. 15) in FP32, then rounded to TF32 or split [hi | lo | hi] in BF16, in
// the canonical K-major layout.  The coefficients of a chunk of 32 paths are
// evaluated once per (subcarrier, path) into shared memory; thread (t, h)
// accumulates w_q for q in [8 h, 8 h + 8).  The rows are then written as
// 16-byte chunks (eight consecutive threads fill one 128-byte core matrix);
// rows beyond K are zero.
constexpr int kProjPC = 32;

constexpr int kProjQ = 8;      // projections w_q per thread

template <int PREC>
__global__ void __launch_bounds__(4 * kTile) k_tc_proj(const SinrArgs A, int Kpad, unsigned char* __restrict__ out) {
  constexpr int ES = PREC == TS_PREC_TF32 ? 4 : 2;
  constexpr int EPC = 16 / ES;                  // elements per 16-byte chunk
  extern __shared__ __align__(16) unsigned char smp[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int t = tid % kTile, h = tid / kTile;
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * kTile;
  const int J = A.J, p = A.p, P = A.P, K = A.K;
  const int k = z < i ? z : z + 1;
  const int ch = i * J + k;
  const int kbytes = Kpad * ES, nkc = kbytes / 16;
  const int WS = 2 * p + 1;
  float* wrow = reinterpret_cast<float*>(smp);                        // [kTile][2p + 1]
  float2* cs = reinterpret_cast<float2*>(smp + ((kTile * WS * 4 + 15) & ~15));   // [kTile][PC + 1]
  float2* sC = cs + kTile * (kProjPC + 1);                            // [PC][p] chunk of C_ik
  const float2* Cch = A.C + (size_t)ch * P * p;
  float2 acc[kProjQ];
#pragma unroll
  for (int u = 0; u < kProjQ; ++u) acc[u] = cz();
  for (int P0 = 0; P0 < P; P0 += kProjPC) {
    const int pc = min(kProjPC, P - P0);
    __syncthreads();
    for (int idx = tid; idx < pc * p; idx += nth) sC[idx] = Cch[(size_t)P0 * p + idx];
    for (int idx = tid; idx < kTile * kProjPC; idx += nth) {
      const int tt = idx / kProjPC, pp = idx % kProjPC;
      const int kap = kap0 + tt;
      float2 c = cz();
      if (pp < pc && kap < K)
        c = A.coef_mode == 0 ? A.coef[((size_t)ch * K + kap) * P + P0 + pp]
                             : path_coef(A.coef[(size_t)ch * P + P0 + pp], A.turns[(size_t)ch * P + P0 + pp], kap);
      cs[tt * (kProjPC + 1) + pp] = c;
    }
    __syncthreads();
    const float2* crow_t = cs + t * (kProjPC + 1);
    for (int pp = 0; pp < pc; ++pp) {
      const float2 c = crow_t[pp];
      const float2* Crow = sC + pp * p + kProjQ * h;
#pragma unroll
      for (int u = 0; u < kProjQ; ++u)
        if (kProjQ * h + u < p) cmacc(acc[u], Crow[u], c);
    }
  }
  float* wr = wrow + t * WS;
#pragma unroll
  for (int u = 0; u < kProjQ; ++u) {
    const int q = kProjQ * h + u;
    if (q < p) {
      wr[q] = acc[u].x;
      wr[p + q] = acc[u].y;
    }
  }
  __syncthreads();
  const int kused = PREC == TS_PREC_TF32 ? 2 * p : 6 * p;
  unsigned char* dst = out + (((size_t)i * (J - 1) + z) * gridDim.x + blockIdx.x) * (size_t)kTile * kbytes;
  const int p2 = 2 * p;
  for (int idx = tid; idx < kTile * nkc; idx += nth) {
    const int r = idx & 7, rest = idx >> 3;
    const int rg = rest / nkc, kc = rest - rg * nkc;
    const int row = rg * 8 + r;
    const float* src = wrow + row * WS;
    uint32_t words[4];
    if (PREC == TS_PREC_TF32) {
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int kk = kc * EPC + e;
        words[e] = __float_as_uint(kk < kused ? to_tf32(src[kk]) : 0.f);
      }
    } else {
      __nv_bfloat16 hv[8];
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int kk = kc * EPC + e;
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (kk < kused) {
          const int seg = kk >= 2 * p2 ? 2 : kk >= p2 ? 1 : 0;
          const float x = src[kk - seg * p2];
          const __nv_bfloat16 hi = __float2bfloat16_rn(x);
          v = seg == 1 ? __float2bfloat16_rn(x - __bfloat162float(hi)) : hi;
        }
        hv[e] = v;
      }
#pragma unroll
      for (int w = 0; w < 4; ++w)
        words[w] = (uint32_t)__bfloat16_as_ushort(hv[2 * w]) | ((uint32_t)__bfloat16_as_ushort(hv[2 * w + 1]) << 16);
    }
    *reinterpret_cast<uint4*>(dst + kmajor_off(row, kc * 16, kbytes)) =
        make_uint4(words[0], words[1], words[2], words[3]);
  }
}

// ----------------------------------------------------------- link kernel
template <int MG, int LT, int PREC>
__global__ void __launch_bounds__(128 * (MG / tc_rpt(MG)))
    k_sinr_link_tc(const SinrArgs A, const unsigned char* __restrict__ prep,
                   const unsigned char* __restrict__ aop, TcPlan tp) {
  constexpr int RPT = tc_rpt(MG);
  constexpr int RG = MG / RPT;
  constexpr int NT = 128 * RG;
  constexpr int ES = PREC == TS_PREC_TF32 ? 4 : 2;
  constexpr int KMMA = 32 / ES;                 // K elements per MMA instruction
  constexpr int kCB = tc_cb(MG);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = warp / 4, t = (warp % 4) * 32 + lane;    // row group, subcarrier of the tile
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * kTile;
  const int J = A.J, m = A.m, n = A.n, L = A.L, K = A.K;
  const int k = z < i ? z : z + 1;
  const int ch = i * J + k;
  const int kbytes = tp.Kpad * ES;
  const int nblk = tp.nblk;
  unsigned char* sA = smem + tp.off_A;
  unsigned char* sB = smem + tp.off_B;
  float2* sV = reinterpret_cast<float2*>(smem + tp.off_V);
  // mbarriers: [0, kBStages) core-operand loads, two MMA completions, the
  // projection operand
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tp.off_bar);
  const uint32_t bar_b0 = smem_u32(&bars[0]), bar_m0 = smem_u32(&bars[kBStages]);
  const uint32_t bar_a = smem_u32(&bars[kBStages + 2]);
  const size_t blk_bytes = (size_t)tp.Ntile * kbytes;
  const unsigned char* prep_ch = prep + (size_t)ch * nblk * blk_bytes;
  const bool wideV = (L % 2 == 0) && ((reinterpret_cast<uintptr_t>(A.V) & 15u) == 0);

  if (tid == 0) {
    abort_flag = 0;
    // the refinement list of the finalize kernel that follows starts empty
    if (A.rcount != nullptr && blockIdx.x == 0 && i == 0 && z == 0) *A.rcount = 0;
    for (int s = 0; s < kBStages + 3; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(2 * tp.Ntile < 32 ? 32 : 2 * tp.Ntile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();

  // core operand of block b: one bulk copy (tid 0) into ring slot b % 3
  auto issue_B = [&](int b) {
    if (b >= nblk || tid != 0) return;
    const int s = b % kBStages;
    const uint32_t bar = bar_b0 + 8 * s;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                 "r"((uint32_t)blk_bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sB + s * blk_bytes)),
        "l"(prep_ch + (size_t)b * blk_bytes), "r"((uint32_t)blk_bytes), "r"(bar)
        : "memory");
  };
  // precoder rows V~_k(kappa)[c0 .. c0+CB)[0 .. L) of the tile for block b
  // (cp.async by every thread, stage b % 2), one commit group per call
  auto issue_V = [&](int b) {
    if (b < nblk) {
      const int c0 = b * kCB;
      float2* dst = sV + (b & 1) * kTile * tp.SV;
      if (wideV) {
        constexpr int U = kCB * LT / 2;            // 16-byte units per subcarrier
        for (int idx = tid; idx < kTile * U; idx += NT) {
          const int tt = idx / U, u = idx - tt * U;
          const int cc = u / (LT / 2), l = 2 * (u % (LT / 2));
          const bool ok = kap0 + tt < K && c0 + cc < n && l < L;
          cp_async16(dst + tt * tp.SV + cc * LT + l,
                     ok ? A.V + (((size_t)k * K + kap0 + tt) * n + c0 + cc) * L + l : A.V, ok);
        }
      } else {
        for (int idx = tid; idx < kTile * kCB * LT; idx += NT) {
          const int tt = idx / (kCB * LT), u = idx - tt * (kCB * LT);
          const int cc = u / LT, l = u % LT;
          const bool ok = kap0 + tt < K && c0 + cc < n && l < L;
          cp_async8(dst + tt * tp.SV + cc * LT + l,
                    ok ? A.V + (((size_t)k * K + kap0 + tt) * n + c0 + cc) * L + l : A.V, ok);
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  // projection operand of the tile (one bulk copy), core operand of blocks
  // 0..2, precoder rows of blocks 0, 1
  const uint32_t a_bytes = (uint32_t)(kTile * kbytes);
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_a), "r"(a_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sA)),
        "l"(aop + (((size_t)i * (J - 1) + z) * gridDim.x + blockIdx.x) * (size_t)a_bytes), "r"(a_bytes),
        "r"(bar_a)
        : "memory");
  }
  issue_B(0);
  issue_B(1);
  issue_B(2);
  issue_V(0);
  issue_V(1);

  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  const uint32_t idesc = (1u << 4) | ((PREC == TS_PREC_TF32 ? 2u : 1u) << 7) |
                         ((PREC == TS_PREC_TF32 ? 2u : 1u) << 10) | ((uint32_t)(tp.Ntile >> 3) << 17) |
                         ((uint32_t)(kTile >> 4) << 24);
  const uint32_t sbo = 128u * (uint32_t)(kbytes >> 4);
  auto issue_mma = [&](int b) -> bool {
    // tid 0 only: wait for the block's operand, then K/KMMA instructions
    const int s = b & 1, sb = b % kBStages;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (b == 0 && !mbar_wait(bar_a, 0)) return false;
    if (!mbar_wait(bar_b0 + 8 * sb, (uint32_t)((b / kBStages) & 1))) return false;
    const uint32_t d = tmem + (uint32_t)(s * tp.Ntile);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + sb * blk_bytes);
    for (int ks = 0; ks < tp.Kpad / KMMA; ++ks) {
      const uint64_t ad = smem_desc(a0 + ks * 256, sbo);
      const uint64_t bd = smem_desc(b0 + ks * 256, sbo);
      const uint32_t accum = ks > 0;
      if (PREC == TS_PREC_TF32)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
      else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     bar_m0 + 8 * s)
                 : "memory");
    return true;
  };
  if (tid == 0 && !issue_mma(0)) abort_flag = 1;

  float2 E[RPT][LT];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int l = 0; l < LT; ++l) E[r][l] = cz();

  bool aborted = false;
  for (int b = 0; b < nblk; ++b) {
    const int s = b & 1;
    // MMA(b + 1) into the other TMEM buffer, whose last reader (block b - 1)
    // finished before the barrier that ended the previous iteration
    if (tid == 0 && b + 1 < nblk && !abort_flag && !issue_mma(b + 1)) abort_flag = 1;
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();                                                // rows of block b staged
    if (abort_flag) { aborted = true; break; }
    if (!mbar_wait(bar_m0 + 8 * s, (uint32_t)((b >> 1) & 1))) abort_flag = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // this thread's H~ block: RPT rows x CB columns, re/im pairs
    constexpr int NCOL = 2 * RPT * kCB;
    uint32_t h[NCOL];
    const uint32_t taddr = tmem + ((uint32_t)((warp % 4) * 32) << 16) +
                           (uint32_t)(s * tp.Ntile + g * NCOL);
    if constexpr (NCOL == 32) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]),
            "=r"(h[7]), "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]),
            "=r"(h[14]), "=r"(h[15]), "=r"(h[16]), "=r"(h[17]), "=r"(h[18]), "=r"(h[19]), "=r"(h[20]),
            "=r"(h[21]), "=r"(h[22]), "=r"(h[23]), "=r"(h[24]), "=r"(h[25]), "=r"(h[26]), "=r"(h[27]),
            "=r"(h[28]), "=r"(h[29]), "=r"(h[30]), "=r"(h[31])
          : "r"(taddr));
    } else if constexpr (NCOL == 16) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]),
            "=r"(h[7]), "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]),
            "=r"(h[14]), "=r"(h[15])
          : "r"(taddr));
    } else {
      static_assert(NCOL == 8, "tcgen05.ld shape");
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                   : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]),
                     "=r"(h[7])
                   : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const float2* vrow = sV + s * kTile * tp.SV + t * tp.SV;
#pragma unroll
    for (int cc = 0; cc < kCB; ++cc) {
#pragma unroll
      for (int l2 = 0; l2 < LT / 2; ++l2) {
        const float4 v = reinterpret_cast<const float4*>(vrow + cc * LT)[l2];
        const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const float2 hv = make_float2(__uint_as_float(h[(cc * RPT + r) * 2]),
                                        __uint_as_float(h[(cc * RPT + r) * 2 + 1]));
          cmac(E[r][2 * l2], hv, v0);
          cmac(E[r][2 * l2 + 1], hv, v1);
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    issue_B(b + 3);     // slot of block b: MMA(b) has completed
    issue_V(b + 2);     // stage of block b: its epilogue is done
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag) aborted = true;

  if (!aborted) {
    // partial covariance rows (E E*)[a][b], b < m (eq. 25), through an
    // exchange of the E rows of the tile in shared memory
    float2* X = reinterpret_cast<float2*>(smem);
    const int XS = MG * LT + 2;
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int l = 0; l < LT; ++l) X[t * XS + (g * RPT + r) * LT + l] = E[r][l];
    __syncthreads();
    const int kap = kap0 + t;
    if (kap < K) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int a = g * RPT + r;
        if (a >= m) continue;
        float2* Rout = A.Rpart + ((((size_t)i * (J - 1) + z) * K + kap) * m + a) * m;
        for (int bb = 0; bb < m; ++bb) {
          float2 acc = cz();
          const float2* eb = X + t * XS + bb * LT;
#pragma unroll
          for (int l = 0; l < LT; ++l) cmacc(acc, E[r][l], eb[l]);
          Rout[bb] = acc;
        }
      }
    }
  } else {
    // an operand or an MMA never arrived: flag the tile's units and stop;
    // pending bulk copies and MMAs get another bounded wait before the
    // accumulator memory is released
    if (tid == 0) {
      for (int s = 0; s < kBStages; ++s) mbar_wait(bar_b0 + 8 * s, 0);
      for (int s = 0; s < 2; ++s) mbar_wait(bar_m0 + 8 * s, 0);
      mbar_wait(bar_a, 0);
    }
    if (g == 0 && kap0 + t < K) A.pflag[(size_t)i * K + kap0 + t] |= TS_FLAG_TIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * tp.Ntile < 32 ? 32 : 2 * tp.Ntile));
}

// both operands: the core of every link and the projections of the
// interfering links' tiles (each written in full, padding included)
template <int PREC>
cudaError_t launch_prep(const SinrArgs& A, int MG, int LT, unsigned char* prep, cudaStream_t s) {
  const TcPlan tp = tc_plan(MG, LT, A.n, A.p, PREC);
  const size_t bbytes = tp.prep_bytes_per_link * (size_t)A.J * A.J;
  const int nchunk = tp.Ntile * (tp.Kpad * tp.ES / 16);
  const int nblocks = A.J * A.J * tp.nblk;
  dim3 pgrid((nchunk + 255) / 256, nblocks < 65535 ? nblocks : 65535);
  k_core_prep<PREC><<<pgrid, 256, 0, s>>>(A.G, A.m, A.n, A.p, MG, tp.Ntile, tp.Kpad, tp.nblk, nblocks,
                                          prep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || A.J < 2) return e;
  const int smem = ((kTile * (2 * A.p + 1) * 4 + 15) & ~15) + kTile * (kProjPC + 1) * 8 +
                   kProjPC * A.p * 8;
  e = cudaFuncSetAttribute(k_tc_proj<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + kTile - 1) / kTile, A.J, A.J - 1);
  k_tc_proj<PREC><<<grid, kTile * ((A.p + kProjQ - 1) / kProjQ), smem, s>>>(A, tp.Kpad, prep + bbytes);
  return cudaGetLastError();
}

template <int MG, int LT, int PREC>
cudaError_t launch_tc(const SinrArgs& A, const unsigned char* prep, cudaStream_t s) {
  if (A.J < 2) return cudaSuccess;
  const TcPlan tp = tc_plan(MG, LT, A.n, A.p, PREC);
  auto kern = k_sinr_link_tc<MG, LT, PREC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tp.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + kTile - 1) / kTile, A.J, A.J - 1);
  const unsigned char* aop = prep + tp.prep_bytes_per_link * (size_t)A.J * A.J;
  kern<<<grid, 128 * (MG / tc_rpt(MG)), tp.smem, s>>>(A, prep, aop, tp);
  return cudaGetLastError();
}

template <int MG, int LT>
cudaError_t launch_tc_prec(const SinrArgs& A, int prec, const unsigned char* prep, cudaStream_t s) {
  return prec == TS_PREC_TF32 ? launch_tc<MG, LT, TS_PREC_TF32>(A, prep, s)
                              : launch_tc<MG, LT, TS_PREC_BF16X2>(A, prep, s);
}

inline int tc_mg(int m) { return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16; }
// stream tiles as in the FP32 kernels: 16-lane groups start at 4
inline int tc_lt(int m, int L) { return L <= 2 && m <= 8 ? 2 : L <= 4 ? 4 : 8; }

}  // namespace
}  // namespace detail

bool tc_supported(int m, int L, int p) {
  const int MG = detail::tc_mg(m), LT = detail::tc_lt(m, L);
  if (m > 16 || L > 8 || LT > MG || p > 32) return false;
  const detail::TcPlan tp = detail::tc_plan(MG, LT, 512, p, TS_PREC_BF16X2);
  return tp.smem <= 227 * 1024;
}

size_t tc_prep_bytes(int J, int m, int L, int n, int p, int K, int prec) {
  const detail::TcPlan tp = detail::tc_plan(detail::tc_mg(m), detail::tc_lt(m, L), n, p, prec);
  const size_t tiles = (size_t)(K + detail::kTile - 1) / detail::kTile;
  return tp.prep_bytes_per_link * (size_t)J * J + tp.a_bytes_per_tile * tiles * J * (J - 1);
}

cudaError_t launch_core_prep(const SinrArgs& a, int prec, void* prep, cudaStream_t s) {
  using namespace detail;
  unsigned char* pp = static_cast<unsigned char*>(prep);
  return prec == TS_PREC_TF32 ? launch_prep<TS_PREC_TF32>(a, tc_mg(a.m), tc_lt(a.m, a.L), pp, s)
                              : launch_prep<TS_PREC_BF16X2>(a, tc_mg(a.m), tc_lt(a.m, a.L), pp, s);
}

cudaError_t launch_sinr_links_tc(const SinrArgs& a, int prec, const void* prep, cudaStream_t s) {
  using namespace detail;
  const unsigned char* pp = static_cast<const unsigned char*>(prep);
  switch (tc_mg(a.m) * 100 + tc_lt(a.m, a.L)) {
    case 202: return launch_tc_prec<2, 2>(a, prec, pp, s);
    case 402: return launch_tc_prec<4, 2>(a, prec, pp, s);
    case 404: return launch_tc_prec<4, 4>(a, prec, pp, s);
    case 802: return launch_tc_prec<8, 2>(a, prec, pp, s);
    case 804: return launch_tc_prec<8, 4>(a, prec, pp, s);
    case 808: return launch_tc_prec<8, 8>(a, prec, pp, s);
    case 1604: return launch_tc_prec<16, 4>(a, prec, pp, s);
    case 1608: return launch_tc_prec<16, 8>(a, prec, pp, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ts

extern "C" int ts_selftest_bounded_wait(long long limit, int arrive, int* out, void* stream) {
  if (out == nullptr) return TS_ERR_NULL;
  if (((uintptr_t)out & 3u) != 0) return TS_ERR_ALIGN;
  if (limit < 1 || limit > (1LL << 24)) return TS_ERR_DIMS;
  ts::detail::k_wait_selftest<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>((long)limit, arrive, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TS_OK : ts::record_cuda_error(e);
}
