// Interfering-link pass of the SVD-precoded SINR with the core contraction
// of eq. (15) on the tensor cores (tcgen05, TMEM accumulators), in three
// arithmetic modes:
//   TF32:    w = c* C and G rounded to TF32, one product chain;
//   TF32X3:  w = w_hi + w_lo and G = G_hi + G_lo in TF32 (11 + 11 significant
//            bits), products w_hi G_hi + w_hi G_lo + w_lo G_hi, FP32
//            accumulation in TMEM: close to FP32 accuracy;
//   BF16X2:  the same three products with BF16 parts (8 + 8 bits).
// The projection w = c* C and the effective channel E = H~ V~ (eq. 24) are
// FP32 (FMA pipe); the finalisation forms the covariance from E.
//
// The complex contraction over the p core slabs is one real GEMM per
// (subcarrier tile, interfering link): rows = the 128 subcarriers of the
// tile (TMEM lanes), columns = (column c, row a, re/im) of H~, reduction
// over k = [Re w | Im w] against the core rewritten once per call by
// k_core_prep as  re column: [Re G ; -Im G],  im column: [Im G ; Re G].
// Operands are K-major without swizzle in shared memory (8-row x 16-byte
// core matrices; K-adjacent ones 128 bytes apart, row groups K_bytes * 8
// apart), hi and lo parts as two K segments of each operand.
//
// k_sinr_link_tc: one CTA per (tile, UE i, interfering BS k), warp
// specialised.  Warp 0, one thread: bulk copies (cp.async.bulk, mbarrier
// transaction counts) of the projection operand (staged in the second core
// slot, then copied once into TMEM with tcgen05.cp) and of the core operand
// in blocks of CB columns of H~ (N = 128 accumulator columns) into a
// two-slot ring, and the MMAs of each block (A from TMEM, B from shared
// memory) into one of two TMEM buffers.  Warp 1, one thread: the precoder
// rows of each block for the tile's subcarriers, laid out contiguously once
// per call by k_v_tiles, one bulk copy per block into a ring of one to four
// slots.  Warps 2 .. 1 + 4 RG (RG row groups of RPT rows): thread
// (lane quadrant, group g) owns subcarrier t of the tile and rows
// g RPT .. g RPT + RPT - 1; per block it reads its H~ rows from TMEM
// (tcgen05.ld, one column at a time) and accumulates E += H~ V~, then frees
// the TMEM buffer and the precoder slot.  No CTA-wide barrier in the loop:
// the roles meet only at mbarriers.  Every
// wait is bounded; on a timeout the tile's precoder flags get
// TS_FLAG_TIMEOUT, outstanding copies and MMAs get another bounded wait,
// and the TMEM is released.
//
// The same kernel with SERVE (TF32X3, before the precoders) forms the
// serving links' H~_ii: one CTA per (tile, UE i), the serving link's
// projections as the A operand, no precoder rows; the epilogue stores the
// accumulator columns as rows of H~_ii for the precoder to read.
#include <cuda_bf16.h>

#include "sinr_impl.cuh"

namespace ts {
namespace detail {
namespace {

constexpr int kTile = 128;     // subcarriers per CTA = MMA M = TMEM lanes
constexpr int kNtile = 128;    // accumulator columns per block (MMA N)
constexpr int kBStages = 2;    // core-operand ring
// A tcgen05.mma of kind::tf32 with M = 128 and K = 8 takes about as long
// for N = 64 as for N = 128 (a fixed issue cost of ~110 cycles on GB300,
// measured), so N = 128 halves the MMA time per column; the core ring then
// holds two 64 KB blocks, and the projection operand (the same size, as
// kTile = kNtile) is staged in the second until it is copied into TMEM.
static_assert(kTile == kNtile, "the projection operand is staged in a core slot");
static_assert(kBStages == 2, "mbarrier layout and projection staging assume two core slots");
constexpr int kVStages = 4;    // precoder-row ring (at most; down to one when shared memory is short)
constexpr long kSpinLimit = 1L << 24;

__host__ __device__ constexpr int tc_rpt(int MG) { return MG < 8 ? MG : 8; }
__host__ __device__ constexpr int tc_rg(int MG) { return MG / tc_rpt(MG); }
// H~ columns per block: N = 2 MG CB = kNtile
__host__ __device__ constexpr int tc_cb(int MG) { return kNtile / (2 * MG); }
__host__ __device__ constexpr int tc_es(int prec) { return prec == TS_PREC_BF16X2 ? 2 : 4; }
__host__ __device__ constexpr int tc_nseg(int prec) { return prec == TS_PREC_TF32 ? 1 : 2; }

struct TcPlan {
  int ES;          // operand element bytes (4 TF32, 2 BF16)
  int nseg;        // K segments per operand (hi; hi, lo)
  int kseg;        // elements per K segment: 2p padded to 32 bytes
  int kbytes;      // bytes per operand row
  int nblk;        // column blocks = ceil(n / CB)
  int VS;          // row stride of one subcarrier's precoder rows of a block
                   // (float2): CB L, or CB L + 2 (see v_piece)
  int vstages;     // slots of the precoder-row ring (1 .. kVStages)
  int nthreads;    // 32 (2 + 4 RG): MMA warp, precoder-row warp, epilogue warps
  int off_A, off_B, off_V, off_bar, smem;   // byte offsets
  size_t prep_bytes_per_link;               // k_core_prep output per link
  size_t a_bytes_per_tile;                  // k_tc_proj output per (link, tile)
  size_t v_bytes_per_tile;                  // k_v_tiles output per (BS, tile)
};

inline TcPlan tc_plan(int MG, int L, int n, int p, int prec) {
  TcPlan t;
  t.ES = tc_es(prec);
  t.nseg = tc_nseg(prec);
  const int kq = 32 / t.ES;                      // elements per 32 bytes
  t.kseg = (2 * p + kq - 1) / kq * kq;
  t.kbytes = t.nseg * t.kseg * t.ES;
  const int CB = tc_cb(MG);
  t.nblk = (n + CB - 1) / CB;
  t.VS = CB * L;
  if ((t.VS / 2) % 8 != 0 && (t.VS / 2) % 2 == 0) t.VS += 2;
  t.nthreads = 32 * (2 + 4 * tc_rg(MG));
  int o = 0;
  t.off_B = o; o += kBStages * kNtile * t.kbytes;
  t.off_A = t.off_B + (kBStages - 1) * kNtile * t.kbytes;     // staged in the last core slot
  // as many precoder-row slots as fit beside the operands (227 KB per CTA,
  // 1 KB of it static)
  t.vstages = kVStages;
  while (t.vstages > 1 && o + t.vstages * kTile * t.VS * 8 + 24 * 8 + 16 > 226 * 1024) --t.vstages;
  t.off_V = o; o += t.vstages * kTile * t.VS * 8;
  o = (o + 15) & ~15;
  t.off_bar = o; o += 24 * 8;
  t.smem = o;
  t.prep_bytes_per_link = (size_t)t.nblk * kNtile * t.kbytes;
  t.a_bytes_per_tile = (size_t)kTile * t.kbytes;
  t.v_bytes_per_tile = (size_t)t.nblk * kTile * t.VS * 8;
  return t;
}

// Position of 16-byte piece j of subcarrier t's precoder row (R pieces of
// data) in the tile layout and in shared memory.  The epilogue threads of a
// quarter warp (eight consecutive subcarriers) read the same j at once: rows
// of a multiple of 8 pieces permute their pieces by t mod 8 (XOR), other
// rows have an odd stride in pieces (VS padded), so the eight reads fall in
// distinct shared-memory banks (a plain 128-byte stride made them an 8-way
// conflict).
__host__ __device__ __forceinline__ int v_piece(int j, int t, int R) {
  return (R & 7) == 0 ? (j ^ (t & 7)) : j;
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
// j = ((cl RG + g) RPT + a_in) 2 + ri of the block (column c0 + cl and row
// a = g RPT + a_in of H~, re/im), k over [Re w | Im w] per K segment:
//   re row: [Re G ; -Im G],   im row: [Im G ; Re G]
// segment 0 the rounded value (hi), segment 1 the rounded remainder (lo).
// One CTA per (link, block): the block's core slab G[q][a][c0 .. c0+CB) is
// staged in shared memory with coalesced loads (MG CB = 64 complex per q),
// then every thread writes 16-byte chunks of the block; padding is zero.
template <int PREC>
__global__ void __launch_bounds__(256) k_core_prep(const float2* __restrict__ G, int m, int n, int p,
                                                   int MG, int kseg, int kbytes, int nblk, int nblocks,
                                                   unsigned char* __restrict__ out) {
  constexpr int ES = tc_es(PREC);
  constexpr int EPC = 16 / ES;                    // elements per 16-byte chunk
  __shared__ float2 Gs[32 * (kNtile / 2)];        // [q][a][cl], p <= 32, MG CB = kNtile / 2
  const int nkc = kbytes / 16;
  const int RPT = tc_rpt(MG), RG = tc_rg(MG), CB = tc_cb(MG);
  const int nchunk = kNtile * nkc;
  for (int y = blockIdx.x; y < nblocks; y += gridDim.x) {
    const int ch = y / nblk, b = y - ch * nblk;
    __syncthreads();                               // the previous block's slab consumed
    for (int idx = threadIdx.x; idx < p * MG * CB; idx += blockDim.x) {
      const int cl = idx % CB, a = (idx / CB) % MG, q = idx / (CB * MG);
      const int c = b * CB + cl;
      Gs[idx] = (a < m && c < n) ? __ldg(G + (((size_t)ch * p + q) * m + a) * n + c) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    unsigned char* blk = out + (size_t)y * kNtile * kbytes;
    for (int idx = threadIdx.x; idx < nchunk; idx += blockDim.x) {
      const int r = idx & 7, rest = idx >> 3;
      const int rg = rest / nkc, kc = rest - rg * nkc;
      const int j = rg * 8 + r;
      const int ri = j & 1, a_in = (j >> 1) % RPT, cg = (j >> 1) / RPT;
      const int cl = cg / RG, a = (cg % RG) * RPT + a_in;
      float x[EPC];
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int k = kc * EPC + e;                // element within the row
        const int seg = k / kseg, kk = k - seg * kseg;
        float v = 0.f;
        if (kk < 2 * p) {
          const int q = kk < p ? kk : kk - p;
          const float2 gv = Gs[(q * MG + a) * CB + cl];   // zero for padding rows and columns
          // re row: [Re G ; -Im G], im row: [Im G ; Re G]
          v = ri == 0 ? (kk < p ? gv.x : -gv.y) : (kk < p ? gv.y : gv.x);
          if (PREC == TS_PREC_BF16X2) {
            const float hi = __bfloat162float(__float2bfloat16_rn(v));
            v = seg == 0 ? hi : v - hi;
          } else {
            const float hi = to_tf32(v);
            v = seg == 0 ? hi : to_tf32(v - hi);
          }
        }
        x[e] = v;
      }
      uint32_t words[4];
      if (ES == 4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) words[e] = __float_as_uint(x[e % EPC]);
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
}

// ------------------------------------------------------ projection operand
// A operand of (interfering link (i, k), subcarrier tile), or with serv of
// the serving link (i, i) (grid z = 1, its own output region): row t =
// subcarrier kap0 + t, k over [Re w | Im w] with w = C_ik^T conj(c_ik(kappa))
// (eq. 15) in FP32, then per K segment rounded (hi) or the rounded
// remainder (lo), in the canonical K-major layout.  The coefficients of a
// chunk of 32 paths are evaluated once per (subcarrier, path) into shared
// memory; thread (t, h) accumulates w_q for q in [8 h, 8 h + 8).  The rows
// are then written as 16-byte chunks; rows beyond K are zero.
constexpr int kProjPC = 32;
constexpr int kProjQ = 8;      // projections w_q per thread

template <int PREC>
__global__ void __launch_bounds__(4 * kTile) k_tc_proj(const SinrArgs A, int kseg, int kbytes, int serv,
                                                       unsigned char* __restrict__ out) {
  constexpr int ES = tc_es(PREC);
  constexpr int EPC = 16 / ES;
  extern __shared__ __align__(16) unsigned char smp[];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int t = tid % kTile, h = tid / kTile;
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * kTile;
  const int J = A.J, p = A.p, P = A.P, K = A.K;
  const int k = serv ? i : (z < i ? z : z + 1);
  const int ch = i * J + k;
  const int nkc = kbytes / 16;
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
        c = A.coef_mode == 0 ? A.coef[((size_t)ch * A.Kc + A.kap_off + kap) * P + P0 + pp]
                             : path_coef(A.coef[(size_t)ch * P + P0 + pp], A.turns[(size_t)ch * P + P0 + pp],
                                         A.kap_off + kap);
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
  unsigned char* dst =
      out + ((serv ? (size_t)i : (size_t)i * (J - 1) + z) * gridDim.x + blockIdx.x) * (size_t)kTile * kbytes;
  for (int idx = tid; idx < kTile * nkc; idx += nth) {
    const int r = idx & 7, rest = idx >> 3;
    const int rg = rest / nkc, kc = rest - rg * nkc;
    const int row = rg * 8 + r;
    const float* src = wrow + row * WS;
    float x[EPC];
#pragma unroll
    for (int e = 0; e < EPC; ++e) {
      const int kel = kc * EPC + e;
      const int seg = kel / kseg, kk = kel - seg * kseg;
      float v = 0.f;
      if (kk < 2 * p) {
        const float w = src[kk];
        if (PREC == TS_PREC_BF16X2) {
          const float hi = __bfloat162float(__float2bfloat16_rn(w));
          v = seg == 0 ? hi : w - hi;
        } else {
          const float hi = to_tf32(w);
          v = seg == 0 ? hi : to_tf32(w - hi);
        }
      }
      x[e] = v;
    }
    uint32_t words[4];
    if (ES == 4) {
#pragma unroll
      for (int e = 0; e < 4; ++e) words[e] = __float_as_uint(x[e % EPC]);
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w)
        words[w] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[(2 * w) % EPC])) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[(2 * w + 1) % EPC])) << 16);
    }
    *reinterpret_cast<uint4*>(dst + kmajor_off(row, kc * 16, kbytes)) =
        make_uint4(words[0], words[1], words[2], words[3]);
  }
}

// ------------------------------------------------------- precoder tiles
// The precoder rows V~_k(kappa)[c][l] of a (tile, column block) for the
// link kernel, as one contiguous chunk: Vt[k][tile][b][t][VS] (t the
// subcarrier of the tile; a row holds [CB][L] as 16-byte pieces placed by
// v_piece), zero beyond K and n and in the row padding, so that one bulk
// copy moves a block's rows for all 128 subcarriers.
__global__ void k_v_tiles(const float2* __restrict__ V, int J, int K, int n, int L, int CB, int VS,
                          int nblk, int ntile, float2* __restrict__ Vt) {
  // 16-byte pieces: L is even, so a piece holds two streams of one column
  const int half = VS / 2;                        // pieces per (tile, block, subcarrier) row
  const int data = CB * L / 2;                    // of which hold precoder entries
  const size_t total = (size_t)J * ntile * nblk * kTile * half;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    size_t r = idx / half;
    const int t = (int)(r % kTile);
    const int piece = v_piece((int)(idx % half), t, data);    // an involution
    r /= kTile;
    const int b = (int)(r % nblk);
    r /= nblk;
    const int tile = (int)(r % ntile);
    const int k = (int)(r / ntile);
    const int e = 2 * piece, c = e / L;
    const int kap = tile * kTile + t, col = b * CB + c;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (piece < data && kap < K && col < n)
      v = __ldg(reinterpret_cast<const float4*>(V + (((size_t)k * K + kap) * n + b * CB) * L + e));
    reinterpret_cast<float4*>(Vt)[idx] = v;
  }
}

// ----------------------------------------------------------- link kernel
constexpr int kBars = 21;      // mbarriers of the link kernel (see below)

// One accumulator column group of a row group: the 2 RPT FP32 words (re, im
// of RPT rows of H~) of this thread's TMEM lane, starting at column taddr.
// Warp-collective; the caller waits (tcgen05.wait::ld) before reading h.
template <int RPT>
__device__ __forceinline__ void tmem_ld_rows(uint32_t taddr, uint32_t (&h)[2 * RPT]) {
  if constexpr (RPT == 8) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]), "=r"(h[7]),
          "=r"(h[8]), "=r"(h[9]), "=r"(h[10]), "=r"(h[11]), "=r"(h[12]), "=r"(h[13]), "=r"(h[14]), "=r"(h[15])
        : "r"(taddr));
  } else if constexpr (RPT == 4) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3]), "=r"(h[4]), "=r"(h[5]), "=r"(h[6]),
                   "=r"(h[7])
                 : "r"(taddr));
  } else {
    static_assert(RPT == 2, "tcgen05.ld shape");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(h[0]), "=r"(h[1]), "=r"(h[2]), "=r"(h[3])
                 : "r"(taddr));
  }
}

template <int MG, int LT, int PREC, bool SERVE>
__global__ void __launch_bounds__(32 * (2 + 4 * tc_rg(MG)), 1)
    k_sinr_link_tc(const SinrArgs A, const unsigned char* __restrict__ prep,
                   const unsigned char* __restrict__ aop, const float2* __restrict__ vtiles, TcPlan tp) {
  constexpr int RPT = tc_rpt(MG), RG = tc_rg(MG), CB = tc_cb(MG);
  constexpr int ES = tc_es(PREC);
  constexpr int KMMA = 32 / ES;                 // K elements per MMA instruction
  constexpr int NEPI = 4 * RG;                  // epilogue warps
  constexpr int NCHAIN = PREC == TS_PREC_TF32 ? 1 : 3;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid % 32;
  const int i = blockIdx.y, z = blockIdx.z;
  const int kap0 = blockIdx.x * kTile;
  const int J = A.J, m = A.m, n = A.n, L = A.L, K = A.K;
  const int k = SERVE ? i : (z < i ? z : z + 1);
  const int ch = i * J + k;
  const int kbytes = tp.kbytes, nblk = tp.nblk;
  unsigned char* sA = smem + tp.off_A;
  unsigned char* sB = smem + tp.off_B;
  float2* sV = reinterpret_cast<float2*>(smem + tp.off_V);
  // mbarriers: 0, 1 core block loaded, 3, 4 its MMAs done (slot free),
  // 6, 7 TMEM buffer written, 8, 9 TMEM buffer read (one arrival per
  // epilogue warp), 10 projection operand loaded, 11 final drain,
  // 12..15 precoder rows of a block loaded, 16..19 read (one arrival per
  // epilogue warp), 20 projection operand copied into TMEM (its staging
  // slot free for core blocks)
  const uint32_t bar0 = smem_u32(smem + tp.off_bar);
  const size_t blk_bytes = (size_t)kNtile * kbytes;
  const unsigned char* prep_ch = prep + (size_t)ch * nblk * blk_bytes;
  volatile int* abort_v = &abort_flag;

  if (tid == 0) {
    abort_flag = 0;
    // the refinement list of the finalize kernel that follows starts empty
    if (!SERVE && A.rcount != nullptr && blockIdx.x == 0 && i == 0 && z == 0) *A.rcount = 0;
    for (int s = 0; s < kBars; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0 + 8u * s),
                   "r"((s == 8 || s == 9 || (s >= 16 && s < 20)) ? (uint32_t)NEPI : 1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)), "r"(4 * kNtile));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- projection operand and MMAs (one thread)
      const uint32_t a_bytes = (uint32_t)(kTile * kbytes);
      const uint32_t afull = bar0 + 8u * 10;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(afull), "r"(a_bytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_u32(sA)),
          "l"(aop + ((SERVE ? (size_t)i : (size_t)i * (J - 1) + z) * gridDim.x + blockIdx.x) * (size_t)a_bytes),
          "r"(a_bytes),
          "r"(afull)
          : "memory");
      const uint32_t idesc = (1u << 4) | ((PREC == TS_PREC_BF16X2 ? 1u : 2u) << 7) |
                             ((PREC == TS_PREC_BF16X2 ? 1u : 2u) << 10) | ((uint32_t)(kNtile >> 3) << 17) |
                             ((uint32_t)(kTile >> 4) << 24);
      const uint32_t sbo = 128u * (uint32_t)(kbytes >> 4);
      const uint32_t segoff = (uint32_t)(tp.kseg * ES * 8);      // K segment start, bytes
      const int nk = tp.kseg / KMMA;                              // MMAs per chain
      const uint32_t segcols = (uint32_t)(tp.kseg * ES / 4);      // K segment start, TMEM columns
      // the projection operand once into TMEM columns 2 kNtile .. (one
      // tcgen05.cp per 32 bytes of K: 8 columns of 128 lanes), so that the
      // MMAs read only the core blocks from shared memory; its staging slot
      // takes core blocks once the copies have read it (barrier 20)
      const uint32_t at0 = tmem + 2u * kNtile;
      bool ok = mbar_wait(afull, 0);
      if (ok) {
        for (int j = 0; j < kbytes / 32; ++j)
          asm volatile("tcgen05.cp.cta_group::1.128x256b [%0], %1;" ::"r"(at0 + 8u * j),
                       "l"(smem_desc(smem_u32(sA) + 256u * j, sbo))
                       : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar0 + 8u * 20) : "memory");
      }
      for (int b = 0; ok && b < nblk; ++b) {
        const int s = b % kBStages, t = b & 1;
        if (!mbar_wait(bar0 + 8u * s, (uint32_t)((b / kBStages) & 1))) { ok = false; break; }
        if (b >= 2 && !mbar_wait(bar0 + 8u * (8 + t), (uint32_t)(((b - 2) >> 1) & 1))) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(t * kNtile);
        const uint32_t b0 = smem_u32(sB + s * blk_bytes);
#pragma unroll
        for (int c = 0; c < NCHAIN; ++c) {
          // chains (hi, hi), (hi, lo), (lo, hi) of (A segment, B segment)
          const uint32_t at = at0 + (c == 2 ? segcols : 0u);
          // descriptor of the chain's first K step; a K step (256 bytes)
          // adds 16 to its 14-bit start-address field (no carry: shared
          // addresses stay below 2^18)
          const uint64_t bdc = smem_desc(b0 + (c == 1 ? segoff : 0u), sbo);
          for (int ks = 0; ks < nk; ++ks) {
            const uint64_t bd = bdc + 16ull * ks;
            const uint32_t accum = (c > 0 || ks > 0) ? 1u : 0u;
            if (PREC == TS_PREC_BF16X2)
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                           "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                           "r"(at + 8u * ks), "l"(bd), "r"(idesc), "r"(accum));
            else
              asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                           "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
                           "r"(at + 8u * ks), "l"(bd), "r"(idesc), "r"(accum));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar0 + 8u * (6 + t)) : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         bar0 + 8u * (3 + s)) : "memory");
      }
      if (!ok) *abort_v = 1;
      // drain: every MMA and copy into TMEM issued so far has completed
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       bar0 + 8u * 11) : "memory");
      if (!mbar_wait(bar0 + 8u * 11, 0)) *abort_v = 1;
      if (!ok) mbar_wait(afull, 0);
    }
  } else if (warp == 1) {
    // ---------------- core blocks and precoder rows, in block order: core
    // block b once the MMAs of block b - kBStages have read its slot (the
    // last slot first once the projection operand is in TMEM), the
    // precoder rows of block b (k_v_tiles laid them out contiguously) once
    // the epilogue has read its slot of the ring
    if (lane == 0) {
      const uint32_t chunk = (uint32_t)(kTile * tp.VS * 8);
      const float2* vt = SERVE ? nullptr : vtiles + ((size_t)k * gridDim.x + blockIdx.x) * tp.v_bytes_per_tile / 8;
      bool ok = true;
      int nB = 0, nV = 0;                          // blocks whose copies were issued
      for (int b = 0; b < nblk; ++b) {
        const int s = b % kBStages;
        if (b == kBStages - 1 && !mbar_wait(bar0 + 8u * 20, 0)) { ok = false; break; }
        if (b >= kBStages && !mbar_wait(bar0 + 8u * (3 + s), (uint32_t)(((b / kBStages) - 1) & 1))) {
          ok = false;
          break;
        }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar0 + 8u * s),
                     "r"((uint32_t)blk_bytes) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_u32(sB + s * blk_bytes)),
            "l"(prep_ch + (size_t)b * blk_bytes), "r"((uint32_t)blk_bytes), "r"(bar0 + 8u * s)
            : "memory");
        nB = b + 1;
        if constexpr (!SERVE) {
          const int slot = b % tp.vstages;
          if (b >= tp.vstages && !mbar_wait(bar0 + 8u * (16 + slot), (uint32_t)(((b / tp.vstages) - 1) & 1))) {
            ok = false;
            break;
          }
          const uint32_t vfull = bar0 + 8u * (12 + slot);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(vfull), "r"(chunk)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(sV + (size_t)slot * kTile * tp.VS)),
              "l"(vt + (size_t)b * kTile * tp.VS), "r"(chunk), "r"(vfull)
              : "memory");
          nV = b + 1;
        }
      }
      if (!ok) *abort_v = 1;
      // drain: the last copy of every slot has landed (each slot has at
      // most one phase outstanding: a copy is issued only after the
      // previous one into its slot was consumed)
      for (int sl = 0; sl < kBStages; ++sl)
        if (sl < nB) mbar_wait(bar0 + 8u * sl, (uint32_t)(((nB - 1 - sl) / kBStages) & 1));
      for (int sl = 0; sl < kVStages; ++sl)
        if (sl < tp.vstages && sl < nV)
          mbar_wait(bar0 + 8u * (12 + sl), (uint32_t)(((nV - 1 - sl) / tp.vstages) & 1));
    }
  } else if constexpr (SERVE) {
    // ---------------- serving links: the rows of H~_ii (subcarrier t_in, rows
    // of group g) from TMEM to Hserv, four adjacent columns (one 32-byte
    // sector) per store where rows are 32-byte aligned (n a multiple of 4)
    static_assert(tc_cb(MG) % 4 == 0, "column blocks of whole sectors");
    const int ew = warp - 2, quad = warp & 3, g = ew >> 2;
    const int t_in = quad * 32 + lane;
    const int kap = kap0 + t_in;
    const bool vec = (n & 3) == 0;
    bool good = true;
    for (int b = 0; b < nblk; ++b) {
      const int t = b & 1;
      if (!mbar_wait(bar0 + 8u * (6 + t), (uint32_t)((b >> 1) & 1))) { good = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int ncb = min(CB, n - b * CB);
      const uint32_t tcol = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(t * kNtile + g * 2 * RPT);
#pragma unroll
      for (int c4 = 0; c4 < CB; c4 += 4) {
        if (c4 >= ncb) break;
        uint32_t h[4][2 * RPT];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c4 + q < ncb) tmem_ld_rows<RPT>(tcol + (uint32_t)((c4 + q) * RG * 2 * RPT), h[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (kap < K) {
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const int a = g * RPT + r;
            if (a >= m) continue;
            float2* dst = A.Hserv + (((size_t)i * A.serv_stride * K + kap) * m + a) * n + b * CB + c4;
            if (vec && c4 + 4 <= ncb) {
              asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(dst),
                           "r"(h[0][2 * r]), "r"(h[0][2 * r + 1]), "r"(h[1][2 * r]), "r"(h[1][2 * r + 1]),
                           "r"(h[2][2 * r]), "r"(h[2][2 * r + 1]), "r"(h[3][2 * r]), "r"(h[3][2 * r + 1])
                           : "memory");
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (c4 + q < ncb)
                  dst[q] = make_float2(__uint_as_float(h[q][2 * r]), __uint_as_float(h[q][2 * r + 1]));
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 8u * (8 + t)) : "memory");
    }
    if (!good) *abort_v = 1;
  } else {
    // ---------------- epilogue: E += H~ V~ for (subcarrier t_in, rows of group g)
    const int ew = warp - 2, quad = warp & 3, g = ew >> 2;
    const int t_in = quad * 32 + lane;           // TMEM lane = subcarrier of the tile
    const int kap = kap0 + t_in;
    float2 E[RPT][LT];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int l = 0; l < LT; ++l) E[r][l] = cz();
    bool good = true;
    for (int b = 0; b < nblk; ++b) {
      const int t = b & 1, slot = b % tp.vstages;
      if (!mbar_wait(bar0 + 8u * (12 + slot), (uint32_t)((b / tp.vstages) & 1))) { good = false; break; }
      if (!mbar_wait(bar0 + 8u * (6 + t), (uint32_t)((b >> 1) & 1))) { good = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float2* vb = sV + ((size_t)slot * kTile + t_in) * tp.VS;
      const int ncb = min(CB, n - b * CB);       // columns of this block (uniform)
      const uint32_t tcol = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(t * kNtile + g * 2 * RPT);
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        if (cc >= ncb) break;
        uint32_t hc[2 * RPT];
        tmem_ld_rows<RPT>(tcol + (uint32_t)(cc * RG * 2 * RPT), hc);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int l2 = 0; l2 < LT / 2; ++l2) {
          if (2 * l2 >= L) break;
          const float4 v = reinterpret_cast<const float4*>(vb)[v_piece(cc * (L / 2) + l2, t_in, CB * L / 2)];
          const float2 v0 = make_float2(v.x, v.y), v1 = make_float2(v.z, v.w);
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            const float2 hv = make_float2(__uint_as_float(hc[2 * r]), __uint_as_float(hc[2 * r + 1]));
            cmac(E[r][2 * l2], hv, v0);
            cmac(E[r][2 * l2 + 1], hv, v1);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 8u * (8 + t)) : "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar0 + 8u * (16 + slot)) : "memory");
      }
    }
    if (!good) *abort_v = 1;
    // rows of the interfering effective channel E_ik (eq. 24); the
    // finalisation forms the covariance of eq. (25)
    // (four streams, one 32-byte sector, per store when L is a multiple of
    // 4, so that every row starts on a sector)
    if (good && kap < K) {
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        const int a = g * RPT + r;
        if (a >= m) continue;
        float2* Eout = A.Eint + ((((size_t)i * (J - 1) + z) * K + kap) * m + a) * L;
        if ((L & 3) == 0) {
#pragma unroll
          for (int l4 = 0; l4 < LT / 4; ++l4)
            if (4 * l4 < L)
              asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(Eout + 4 * l4),
                           "f"(E[r][4 * l4].x), "f"(E[r][4 * l4].y), "f"(E[r][4 * l4 + 1].x),
                           "f"(E[r][4 * l4 + 1].y), "f"(E[r][4 * l4 + 2].x), "f"(E[r][4 * l4 + 2].y),
                           "f"(E[r][4 * l4 + 3].x), "f"(E[r][4 * l4 + 3].y)
                           : "memory");
        } else {
#pragma unroll
          for (int l = 0; l < LT; ++l)
            if (l < L) Eout[l] = E[r][l];
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_v) {
    // an operand or an MMA never arrived: the tile's units are flagged (and
    // get NaN from the finalisation); for the serving links the tile's rows
    // of H~_ii become NaN, which the precoder that reads them reports as
    // unconverged (TS_FLAG_EIG_UNCONVERGED, NaN SINRs)
    if constexpr (SERVE) {
      const size_t rows = (size_t)min(kTile, K - kap0) * m * n;
      float2* dst = A.Hserv + ((size_t)i * A.serv_stride * K + kap0) * m * n;
      for (size_t e = tid; e < rows; e += blockDim.x) dst[e] = make_float2(__int_as_float(0x7fc00000), 0.f);
    } else {
      for (int t = tid; t < kTile; t += blockDim.x)
        if (kap0 + t < K) A.pflag[(size_t)i * K + kap0 + t] |= TS_FLAG_TIMEOUT;
    }
  }
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(4 * kNtile));
}

// Layout of the operand buffer: the core operand of every link, the
// projections of the interfering links' tiles, the precoder-row tiles, and
// (TF32X3 only) the projections of the serving links' tiles.
struct TcLayout {
  size_t aop, vt, serv, total;
};

inline TcLayout tc_layout(const TcPlan& tp, int J, int K, int prec) {
  const size_t ntile = (size_t)(K + kTile - 1) / kTile;
  TcLayout l;
  l.aop = tp.prep_bytes_per_link * (size_t)J * J;
  l.vt = l.aop + tp.a_bytes_per_tile * ntile * J * (J - 1);
  l.serv = l.vt + tp.v_bytes_per_tile * ntile * J;
  l.total = l.serv + (prec == TS_PREC_TF32X3 ? tp.a_bytes_per_tile * ntile * J : 0);
  return l;
}

// the operands that do not depend on the precoders: the core of every link
// and the projections of the interfering links' tiles, with `serving` also
// those of the serving links' tiles (each written in full, padding included)
template <int PREC>
cudaError_t launch_operands(const SinrArgs& A, int MG, bool serving, unsigned char* prep, cudaStream_t s) {
  const TcPlan tp = tc_plan(MG, A.L, A.n, A.p, PREC);
  const TcLayout lay = tc_layout(tp, A.J, A.K, PREC);
  const int nblocks = A.J * A.J * tp.nblk;
  const int pgrid = nblocks < 152 * 64 ? nblocks : 152 * 64;
  k_core_prep<PREC><<<pgrid, 256, 0, s>>>(A.G, A.m, A.n, A.p, MG, tp.kseg, tp.kbytes, tp.nblk, nblocks,
                                          prep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || (A.J < 2 && !serving)) return e;
  const int smem = ((kTile * (2 * A.p + 1) * 4 + 15) & ~15) + kTile * (kProjPC + 1) * 8 +
                   kProjPC * A.p * 8;
  e = cudaFuncSetAttribute(k_tc_proj<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int ntile = (A.K + kTile - 1) / kTile;
  const int nthr = kTile * ((A.p + kProjQ - 1) / kProjQ);
  if (A.J >= 2) {
    k_tc_proj<PREC><<<dim3(ntile, A.J, A.J - 1), nthr, smem, s>>>(A, tp.kseg, tp.kbytes, 0, prep + lay.aop);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (serving) {
    k_tc_proj<PREC><<<dim3(ntile, A.J, 1), nthr, smem, s>>>(A, tp.kseg, tp.kbytes, 1, prep + lay.serv);
    e = cudaGetLastError();
  }
  return e;
}

// the precoder rows, tiled per (tile, column block)
template <int PREC>
cudaError_t launch_vtiles(const SinrArgs& A, int MG, unsigned char* prep, cudaStream_t s) {
  if (A.J < 2) return cudaSuccess;
  const TcPlan tp = tc_plan(MG, A.L, A.n, A.p, PREC);
  const TcLayout lay = tc_layout(tp, A.J, A.K, PREC);
  const int ntile = (A.K + kTile - 1) / kTile;
  const size_t vtotal = (size_t)A.J * ntile * tp.nblk * kTile * (tp.VS / 2);   // 16-byte pieces
  const int vblocks = (int)((vtotal + 255) / 256 < 152 * 16 ? (vtotal + 255) / 256 : 152 * 16);
  k_v_tiles<<<vblocks, 256, 0, s>>>(A.V, A.J, A.K, A.n, A.L, tc_cb(MG), tp.VS, tp.nblk, ntile,
                                    reinterpret_cast<float2*>(prep + lay.vt));
  return cudaGetLastError();
}

template <int MG, int LT, int PREC>
cudaError_t launch_tc(const SinrArgs& A, const unsigned char* prep, cudaStream_t s) {
  if (A.J < 2) return cudaSuccess;
  const TcPlan tp = tc_plan(MG, A.L, A.n, A.p, PREC);
  const TcLayout lay = tc_layout(tp, A.J, A.K, PREC);
  auto kern = k_sinr_link_tc<MG, LT, PREC, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tp.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + kTile - 1) / kTile, A.J, A.J - 1);
  kern<<<grid, tp.nthreads, tp.smem, s>>>(A, prep, prep + lay.aop, reinterpret_cast<const float2*>(prep + lay.vt),
                                          tp);
  return cudaGetLastError();
}

// the serving links' H~_ii (TF32X3) into Hserv: the link kernel without the
// precoder-row ring
template <int MG>
cudaError_t launch_serve_tc(const SinrArgs& A, const unsigned char* prep, cudaStream_t s) {
  TcPlan tp = tc_plan(MG, A.L, A.n, A.p, TS_PREC_TF32X3);
  const TcLayout lay = tc_layout(tp, A.J, A.K, TS_PREC_TF32X3);
  tp.off_bar = (tp.off_V + 15) & ~15;
  tp.smem = tp.off_bar + 24 * 8;
  auto kern = k_sinr_link_tc<MG, 2, TS_PREC_TF32X3, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tp.smem);
  if (e != cudaSuccess) return e;
  dim3 grid((A.K + kTile - 1) / kTile, A.J, 1);
  kern<<<grid, tp.nthreads, tp.smem, s>>>(A, prep, prep + lay.serv, nullptr, tp);
  return cudaGetLastError();
}

template <int MG, int LT>
cudaError_t launch_tc_prec(const SinrArgs& A, int prec, const unsigned char* prep, cudaStream_t s) {
  if (prec == TS_PREC_TF32) return launch_tc<MG, LT, TS_PREC_TF32>(A, prep, s);
  if (prec == TS_PREC_TF32X3) return launch_tc<MG, LT, TS_PREC_TF32X3>(A, prep, s);
  return launch_tc<MG, LT, TS_PREC_BF16X2>(A, prep, s);
}

inline int tc_mg(int m) { return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : 16; }
// stream tiles as in the FP32 kernels: 16-lane groups start at 4
inline int tc_lt(int m, int L) { return L <= 2 && m <= 8 ? 2 : L <= 4 ? 4 : 8; }

}  // namespace
}  // namespace detail

bool tc_supported(int m, int L, int p) {
  const int MG = detail::tc_mg(m), LT = detail::tc_lt(m, L);
  // even L: the precoder rows of a block are copied as 16-byte multiples
  if (m > 16 || L > 8 || (L & 1) || LT > MG || p > 32) return false;
  const detail::TcPlan tp = detail::tc_plan(MG, L, 512, p, TS_PREC_TF32X3);
  return tp.smem + 1024 <= 227 * 1024;   // + the static shared memory of the kernel
}

size_t tc_prep_bytes(int J, int m, int L, int n, int p, int K, int prec) {
  const detail::TcPlan tp = detail::tc_plan(detail::tc_mg(m), L, n, p, prec);
  return detail::tc_layout(tp, J, K, prec).total;
}

cudaError_t launch_tc_operands(const SinrArgs& a, int prec, bool serving, void* prep, cudaStream_t s) {
  using namespace detail;
  unsigned char* pp = static_cast<unsigned char*>(prep);
  const int MG = tc_mg(a.m);
  if (prec == TS_PREC_TF32) return launch_operands<TS_PREC_TF32>(a, MG, false, pp, s);
  if (prec == TS_PREC_TF32X3) return launch_operands<TS_PREC_TF32X3>(a, MG, serving, pp, s);
  return launch_operands<TS_PREC_BF16X2>(a, MG, false, pp, s);
}

cudaError_t launch_tc_vtiles(const SinrArgs& a, int prec, void* prep, cudaStream_t s) {
  using namespace detail;
  unsigned char* pp = static_cast<unsigned char*>(prep);
  const int MG = tc_mg(a.m);
  if (prec == TS_PREC_TF32) return launch_vtiles<TS_PREC_TF32>(a, MG, pp, s);
  if (prec == TS_PREC_TF32X3) return launch_vtiles<TS_PREC_TF32X3>(a, MG, pp, s);
  return launch_vtiles<TS_PREC_BF16X2>(a, MG, pp, s);
}

cudaError_t launch_core_prep(const SinrArgs& a, int prec, void* prep, cudaStream_t s) {
  cudaError_t e = launch_tc_operands(a, prec, false, prep, s);
  return e == cudaSuccess ? launch_tc_vtiles(a, prec, prep, s) : e;
}

cudaError_t launch_serving_tc(const SinrArgs& a, const void* prep, cudaStream_t s) {
  using namespace detail;
  const unsigned char* pp = static_cast<const unsigned char*>(prep);
  switch (tc_mg(a.m)) {
    case 2: return launch_serve_tc<2>(a, pp, s);
    case 4: return launch_serve_tc<4>(a, pp, s);
    case 8: return launch_serve_tc<8>(a, pp, s);
    default: return launch_serve_tc<16>(a, pp, s);
  }
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
