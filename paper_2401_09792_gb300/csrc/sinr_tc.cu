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
// Per CTA (tile, UE i, interfering BS k): the projection writes the A
// operand; the core is consumed in column blocks of CB = 4 columns of H~
// (N = 8 MG accumulator columns per block), each block's operand fetched by
// one bulk copy (cp.async.bulk + mbarrier transaction count) and multiplied
// by one thread into one of two TMEM buffers, one block ahead of the
// epilogue; the precoder rows of the block are staged by cp.async.  The
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
constexpr int kCB = 4;         // H~ columns per accumulator block
constexpr long kSpinLimit = 1L << 24;

struct TcPlan {
  int ES;          // operand element bytes (4 TF32, 2 BF16)
  int Kpad;        // reduction length in elements, padded to 32 bytes
  int Ntile;       // accumulator columns per block = 2 MG CB
  int nblk;        // column blocks = ceil(n / CB)
  int SV;          // precoder stage row stride (float2), per subcarrier
  int off_A, off_B, off_V, off_bar, smem;   // byte offsets
  size_t prep_bytes_per_link;               // k_core_prep output per link
};

__host__ __device__ constexpr int tc_rpt(int MG) { return MG < 4 ? MG : 4; }

inline TcPlan tc_plan(int MG, int LT, int n, int p, int prec) {
  TcPlan t;
  t.ES = prec == TS_PREC_TF32 ? 4 : 2;
  const int kused = prec == TS_PREC_TF32 ? 2 * p : 6 * p;
  const int kq = 32 / t.ES;                      // elements per 32 bytes
  t.Kpad = (kused + kq - 1) / kq * kq;
  t.Ntile = 2 * MG * kCB;
  t.nblk = (n + kCB - 1) / kCB;
  t.SV = kCB * LT + 2;
  int o = 0;
  t.off_A = o; o += kTile * t.Kpad * t.ES;
  t.off_B = o; o += 2 * t.Ntile * t.Kpad * t.ES;
  t.off_V = o; o += 2 * kTile * t.SV * 8;
  // E exchange at the end reuses the front of the buffer
  const int ex = kTile * MG * (LT * 8) + kTile * 16;
  if (ex > o) o = ex;
  o = (o + 15) & ~15;
  t.off_bar = o; o += 64;
  t.smem = o;
  t.prep_bytes_per_link = (size_t)t.nblk * t.Ntile * t.Kpad * t.ES;
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

template <int PREC>
__device__ __forceinline__ void store_split(unsigned char* base, int r, int k, int kused_seg,
                                            int kbytes, float x, bool a_side) {
  // TF32: one element at k.  BF16X2: segments [hi | lo | hi] (A side) or
  // [hi | hi | lo] (B side), each kused_seg wide.
  if (PREC == TS_PREC_TF32) {
    *reinterpret_cast<float*>(base + kmajor_off(r, k * 4, kbytes)) = to_tf32(x);
  } else {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    const __nv_bfloat16 s1 = a_side ? lo : hi, s2 = a_side ? hi : lo;
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_off(r, k * 2, kbytes)) = hi;
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_off(r, (k + kused_seg) * 2, kbytes)) = s1;
    *reinterpret_cast<__nv_bfloat16*>(base + kmajor_off(r, (k + 2 * kused_seg) * 2, kbytes)) = s2;
  }
}

// bounded wait on an mbarrier phase; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

// ------------------------------------------------------------ core operand
// B operand of link ch, column block b, in the canonical layout: row
// j = ((g CB + c) RPT + a_in) 2 + ri of the block (row a = g RPT + a_in,
// column c0 + c of H~), k over [Re w | Im w] (x3 segments for BF16X2).
template <int PREC>
__global__ void k_core_prep(const float2* __restrict__ G, int nch, int m, int n, int p, int MG,
                            int Ntile, int Kpad, int nblk, unsigned char* __restrict__ out) {
  const int ES = PREC == TS_PREC_TF32 ? 4 : 2;
  const int kbytes = Kpad * ES;
  const int RPT = tc_rpt(MG);
  const size_t per_block = (size_t)Ntile * kbytes;
  const size_t total = (size_t)nch * nblk * Ntile * (2 * p);   // (row, k < 2p) pairs
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx % (2 * p));
    size_t rest = idx / (2 * p);
    const int j = (int)(rest % Ntile);
    rest /= Ntile;
    const int b = (int)(rest % nblk);
    const int ch = (int)(rest / nblk);
    const int ri = j & 1, a_in = (j >> 1) % RPT, cg = (j >> 1) / RPT;
    const int c = b * kCB + cg % kCB, g = cg / kCB;
    const int a = g * RPT + a_in;
    float x = 0.f;
    if (a < m && c < n) {
      const int q = k < p ? k : k - p;
      const float2 gv = G[(((size_t)ch * p + q) * m + a) * n + c];
      // re column: [Re G ; -Im G], im column: [Im G ; Re G]
      x = ri == 0 ? (k < p ? gv.x : -gv.y) : (k < p ? gv.y : gv.x);
    }
    unsigned char* blk = out + ((size_t)ch * nblk + b) * per_block;
    store_split<PREC>(blk, j, k, 2 * p, kbytes, x, false);
  }
  // padding of K beyond the used segments is zeroed by the host (memset)
}

// ----------------------------------------------------------- link kernel
template <int MG, int LT, int PREC>
__global__ void __launch_bounds__(128 * (MG / tc_rpt(MG)))
    k_sinr_link_tc(const SinrArgs A, const unsigned char* __restrict__ prep, TcPlan tp) {
  constexpr int RPT = tc_rpt(MG);
  constexpr int RG = MG / RPT;
  constexpr int NT = 128 * RG;
  constexpr int ES = PREC == TS_PREC_TF32 ? 4 : 2;
  constexpr int KMMA = 32 / ES;                 // K elements per MMA instruction
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int g = warp / 4, t = (warp % 4) * 32 + lane;    // row group, subcarrier of the tile
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * kTile;
  const int J = A.J, m = A.m, n = A.n, p = A.p, L = A.L, K = A.K, P = A.P;
  const int k = z < i ? z : z + 1;
  const int ch = i * J + k;
  const int kbytes = tp.Kpad * ES;
  const int nblk = tp.nblk;
  unsigned char* sA = smem + tp.off_A;
  unsigned char* sB = smem + tp.off_B;
  float2* sV = reinterpret_cast<float2*>(smem + tp.off_V);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tp.off_bar);   // [0,1] B loads, [2,3] MMA
  const uint32_t bar_b0 = smem_u32(&bars[0]), bar_m0 = smem_u32(&bars[2]);
  const size_t blk_bytes = (size_t)tp.Ntile * kbytes;
  const unsigned char* prep_ch = prep + (size_t)ch * nblk * blk_bytes;
  const bool wideV = (L % 2 == 0) && ((reinterpret_cast<uintptr_t>(A.V) & 15u) == 0);

  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < 4; ++s)
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

  // block loads: the B operand by one bulk copy (tid 0), the precoder rows
  // V~_k(kappa)[c0 .. c0+CB)[0 .. L) of the tile by cp.async
  auto issue_block = [&](int b) {
    const int s = b & 1;
    if (b < nblk) {
      if (tid == 0) {
        const uint32_t bar = bar_b0 + 8 * s;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((uint32_t)blk_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sB + s * blk_bytes)),
            "l"(prep_ch + (size_t)b * blk_bytes), "r"((uint32_t)blk_bytes), "r"(bar)
            : "memory");
      }
      const int c0 = b * kCB;
      float2* dst = sV + s * kTile * tp.SV;
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
  issue_block(0);
  issue_block(1);

  // projection w = C^T conj(c(kappa)) (eq. 15) in FP32 -> A operand; thread
  // (g, t) takes q = g, g + RG, ...
  {
    const int kap = kap0 + t;
    const float2* Cch = A.C + (size_t)ch * P * p;
    constexpr int QA = (32 + RG - 1) / RG;
    float2 acc[QA];
#pragma unroll
    for (int u = 0; u < QA; ++u) acc[u] = cz();
    if (kap < K) {
      for (int pp = 0; pp < P; ++pp) {
        const float2 c = A.coef_mode == 0
                             ? A.coef[((size_t)ch * K + kap) * P + pp]
                             : path_coef(A.coef[(size_t)ch * P + pp], A.turns[(size_t)ch * P + pp], kap);
        const float2* crow = Cch + (size_t)pp * p;
#pragma unroll
        for (int u = 0; u < QA; ++u) {
          const int q = g + u * RG;
          if (q < p) cmacc(acc[u], __ldg(crow + q), c);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < QA; ++u) {
      const int q = g + u * RG;
      if (q < p) {
        store_split<PREC>(sA, t, q, 2 * p, kbytes, acc[u].x, true);
        store_split<PREC>(sA, t, p + q, 2 * p, kbytes, acc[u].y, true);
      }
    }
    // zero the K padding of this row
    const int kused = PREC == TS_PREC_TF32 ? 2 * p : 6 * p;
    for (int kk = kused + g; kk < tp.Kpad; kk += RG) {
      if (ES == 4) *reinterpret_cast<float*>(sA + kmajor_off(t, kk * 4, kbytes)) = 0.f;
      else *reinterpret_cast<__nv_bfloat16*>(sA + kmajor_off(t, kk * 2, kbytes)) = __float2bfloat16_rn(0.f);
    }
  }
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
    const int s = b & 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!mbar_wait(bar_b0 + 8 * s, (uint32_t)((b >> 1) & 1))) return false;
    const uint32_t d = tmem + (uint32_t)(s * tp.Ntile);
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB + s * blk_bytes);
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
    if (tid == 0 && b + 1 < nblk && !abort_flag && !issue_mma(b + 1)) abort_flag = 1;
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
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
    } else {
      static_assert(NCOL == 16, "tcgen05.ld shape");
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]),
            "=r"(h[7]), "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]),
            "=r"(h[14]), "=r"(h[15])
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
    issue_block(b + 2);
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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
      for (int s = 0; s < 2; ++s) {
        mbar_wait(bar_b0 + 8 * s, 0);
        mbar_wait(bar_m0 + 8 * s, 0);
      }
    }
    if (g == 0 && kap0 + t < K) A.pflag[(size_t)i * K + kap0 + t] |= TS_FLAG_TIMEOUT;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * tp.Ntile < 32 ? 32 : 2 * tp.Ntile));
}

template <int PREC>
cudaError_t launch_prep(const SinrArgs& A, int MG, int LT, unsigned char* prep, cudaStream_t s) {
  const TcPlan tp = tc_plan(MG, LT, A.n, A.p, PREC);
  cudaError_t e = cudaMemsetAsync(prep, 0, tp.prep_bytes_per_link * (size_t)A.J * A.J, s);
  if (e != cudaSuccess) return e;
  const size_t total = (size_t)A.J * A.J * tp.nblk * tp.Ntile * 2 * A.p;
  const int threads = 256;
  const size_t want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
  k_core_prep<PREC><<<blocks, threads, 0, s>>>(A.G, A.J * A.J, A.m, A.n, A.p, MG, tp.Ntile, tp.Kpad,
                                               tp.nblk, prep);
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
  kern<<<grid, 128 * (MG / tc_rpt(MG)), tp.smem, s>>>(A, prep, tp);
  return cudaGetLastError();
}

template <int MG, int LT>
cudaError_t launch_tc_prec(const SinrArgs& A, int prec, const unsigned char* prep, cudaStream_t s) {
  return prec == TS_PREC_TF32 ? launch_tc<MG, LT, TS_PREC_TF32>(A, prep, s)
                              : launch_tc<MG, LT, TS_PREC_BF16X2>(A, prep, s);
}

inline int tc_mg(int m) { return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16; }
inline int tc_lt(int L) { return L <= 2 ? 2 : L <= 4 ? 4 : 8; }

}  // namespace
}  // namespace detail

bool tc_supported(int m, int L, int p) {
  const int MG = detail::tc_mg(m), LT = detail::tc_lt(L);
  if (m > 16 || L > 8 || LT > MG || p > 32) return false;
  const detail::TcPlan tp = detail::tc_plan(MG, LT, 512, p, TS_PREC_BF16X2);
  return tp.smem <= 227 * 1024;
}

size_t tc_prep_bytes(int J, int m, int L, int n, int p, int prec) {
  return detail::tc_plan(detail::tc_mg(m), detail::tc_lt(L), n, p, prec).prep_bytes_per_link *
         (size_t)J * J;
}

cudaError_t launch_core_prep(const SinrArgs& a, int prec, void* prep, cudaStream_t s) {
  using namespace detail;
  unsigned char* pp = static_cast<unsigned char*>(prep);
  return prec == TS_PREC_TF32 ? launch_prep<TS_PREC_TF32>(a, tc_mg(a.m), tc_lt(a.L), pp, s)
                              : launch_prep<TS_PREC_BF16X2>(a, tc_mg(a.m), tc_lt(a.L), pp, s);
}

cudaError_t launch_sinr_links_tc(const SinrArgs& a, int prec, const void* prep, cudaStream_t s) {
  using namespace detail;
  const unsigned char* pp = static_cast<const unsigned char*>(prep);
  switch (tc_mg(a.m) * 100 + tc_lt(a.L)) {
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
