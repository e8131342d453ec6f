// Dispatch of the SINR kernels and the small helper kernels (coefficients,
// precoder projection, wideband-precoder fold).  The SINR kernel templates
// live in sinr_impl.cuh and are instantiated in sinr_mg*.cu.
#include "sinr_impl.cuh"

namespace ts {
namespace detail {
extern template cudaError_t run_precoder<2, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<2, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<2, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<2, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<2, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<4, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<4, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<4, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<4, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<4, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<4, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<4, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<4, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<4, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<4, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<8, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<8, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<8, 2>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<8, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<8, 2>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<8, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<8, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<8, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<8, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<8, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<8, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<8, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<8, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<8, 8>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<8, 8>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<16, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<16, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<16, 4>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<16, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<16, 4>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<16, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<16, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<16, 8>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<16, 8>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<16, 8>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_precoder<16, 16>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_serving<16, 16>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_rebuild<16, 16>(const SinrArgs&, cudaStream_t);
extern template cudaError_t run_links<16, 16>(const SinrArgs&, bool, cudaStream_t);
extern template cudaError_t run_finalize<16, 16>(const SinrArgs&, bool, cudaStream_t);

// Units with more than 16 rows (sinr_large.cu): specialisations of the
// dispatch templates for 32 and 64 rows.
#define TS_LARGE_DECL(MG, LT)                                                        \
  template <> cudaError_t run_precoder<MG, LT>(const SinrArgs&, cudaStream_t);       \
  template <> cudaError_t run_serving<MG, LT>(const SinrArgs&, cudaStream_t);        \
  template <> cudaError_t run_rebuild<MG, LT>(const SinrArgs&, cudaStream_t);        \
  template <> cudaError_t run_links<MG, LT>(const SinrArgs&, bool, cudaStream_t);    \
  template <> cudaError_t run_finalize<MG, LT>(const SinrArgs&, bool, cudaStream_t);
TS_LARGE_DECL(32, 2)
TS_LARGE_DECL(32, 4)
TS_LARGE_DECL(32, 8)
TS_LARGE_DECL(64, 2)
TS_LARGE_DECL(64, 4)
TS_LARGE_DECL(64, 8)
#undef TS_LARGE_DECL

namespace {
// ------------------------------------------------------------ small kernels
__device__ __forceinline__ unsigned long long turn_fixed(float tau, float df) {
  // df * tau cycles per subcarrier, reduced mod 1 and scaled to 2^-64 turns
  double t = (double)df * (double)tau;
  t -= floor(t);
  const double x = t * 18446744073709551616.0;  // 2^64
  return (x >= 18446744073709551616.0) ? 0ull : (unsigned long long)x;
}

__global__ void k_turns(const float* tau, float df, int count, unsigned long long* turns) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) turns[idx] = turn_fixed(tau[idx], df);
}

__global__ void k_coefficients(const float2* alpha, const float* tau, float df, int nch, int K,
                               int P, float2* c) {
  const size_t total = (size_t)nch * K * P;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int pp = (int)(idx % P);
    const size_t rest = idx / P;
    const int kap = (int)(rest % K);
    const size_t ch = rest / K;
    c[idx] = path_coef(alpha[ch * P + pp], turn_fixed(tau[ch * P + pp], df), kap);
  }
}

__global__ void k_project_precoder(const float2* B, const float2* Pfull, int J, int N, int n,
                                   int L, float2* Pt) {
  // Pt[k][b][l] = sum_N B[k][N][b] * Pfull[k][N][l]
  const int total = J * n * L;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int l = idx % L, b = (idx / L) % n, k = idx / (L * n);
    float2 acc = cz();
    for (int r = 0; r < N; ++r)
      cmac(acc, B[((size_t)k * N + r) * n + b], Pfull[((size_t)k * N + r) * L + l]);
    Pt[idx] = acc;
  }
}

__global__ void k_mmse_fold(const float2* G, const float2* Pt, int J, int m, int n, int p, int L,
                            float2* F) {
  // F[ch][q][a][l] = sum_b G[ch][q][a][b] Pt[k][b][l], ch = i*J + k
  const size_t total = (size_t)J * J * p * m * L;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int l = (int)(idx % L);
    const size_t qa = idx / L;  // (ch*p + q)*m + a
    const size_t ch = qa / ((size_t)p * m);
    const int k = (int)(ch % J);
    const float2* grow = G + qa * n;
    const float2* pk = Pt + (size_t)k * n * L;
    float2 acc = cz();
    for (int b = 0; b < n; ++b) cmac(acc, grow[b], pk[(size_t)b * L + l]);
    F[idx] = acc;
  }
}

int group_size(int m) { return m <= 2 ? 2 : m <= 4 ? 4 : m <= 8 ? 8 : m <= 16 ? 16 : m <= 32 ? 32 : 64; }
int ltile(int L) { return L <= 2 ? 2 : L <= 4 ? 4 : L <= 8 ? 8 : 16; }
}  // namespace
}  // namespace detail

using detail::group_size;
using detail::ltile;
using detail::run_precoder;
using detail::run_links;
using detail::run_rebuild;
using detail::run_serving;
using detail::run_finalize;

#define TS_DISPATCH(FN, ...)                                                        \
  do {                                                                              \
    const int MG_ = group_size(a.m), LT_ = ltile(a.L);                              \
    if (MG_ == 2) return FN<2, 2>(__VA_ARGS__);                                     \
    if (MG_ == 4) return LT_ <= 2 ? FN<4, 2>(__VA_ARGS__) : FN<4, 4>(__VA_ARGS__);  \
    if (MG_ == 8)                                                                   \
      return LT_ <= 2 ? FN<8, 2>(__VA_ARGS__)                                       \
                      : LT_ <= 4 ? FN<8, 4>(__VA_ARGS__) : FN<8, 8>(__VA_ARGS__);   \
    if (MG_ == 16)                                                                  \
      return LT_ <= 4 ? FN<16, 4>(__VA_ARGS__)                                      \
                      : LT_ <= 8 ? FN<16, 8>(__VA_ARGS__) : FN<16, 16>(__VA_ARGS__);\
    if (MG_ == 32)                                                                  \
      return LT_ <= 2 ? FN<32, 2>(__VA_ARGS__)                                      \
                      : LT_ <= 4 ? FN<32, 4>(__VA_ARGS__) : FN<32, 8>(__VA_ARGS__); \
    return LT_ <= 2 ? FN<64, 2>(__VA_ARGS__)                                        \
                    : LT_ <= 4 ? FN<64, 4>(__VA_ARGS__) : FN<64, 8>(__VA_ARGS__);   \
  } while (0)

cudaError_t launch_svd_precoder(const SinrArgs& a, cudaStream_t s) { TS_DISPATCH(run_precoder, a, s); }


cudaError_t launch_sinr_rebuild(const SinrArgs& a, cudaStream_t s) { TS_DISPATCH(run_rebuild, a, s); }
cudaError_t launch_sinr_serving(const SinrArgs& a, cudaStream_t s) { TS_DISPATCH(run_serving, a, s); }

cudaError_t launch_sinr_links(const SinrArgs& a, bool svd, cudaStream_t s) {
  TS_DISPATCH(run_links, a, svd, s);
}

cudaError_t launch_sinr_finalize(const SinrArgs& a, bool svd, cudaStream_t s) {
  TS_DISPATCH(run_finalize, a, svd, s);
}

cudaError_t launch_turns(const float* tau, float df, int count, unsigned long long* turns,
                         cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  detail::k_turns<<<(count + 255) / 256, 256, 0, s>>>(tau, df, count, turns);
  return cudaGetLastError();
}

cudaError_t launch_coefficients(const float2* alpha, const float* tau, float df, int nch, int K,
                                int P, float2* c, cudaStream_t s) {
  const size_t total = (size_t)nch * K * P;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
  detail::k_coefficients<<<blocks, 256, 0, s>>>(alpha, tau, df, nch, K, P, c);
  return cudaGetLastError();
}

cudaError_t launch_project_precoder(const float2* B, const float2* Pfull, int J, int N, int n,
                                    int L, float2* Pt, cudaStream_t s) {
  const int total = J * n * L;
  if (total == 0) return cudaSuccess;
  detail::k_project_precoder<<<(total + 255) / 256, 256, 0, s>>>(B, Pfull, J, N, n, L, Pt);
  return cudaGetLastError();
}

cudaError_t launch_mmse_fold(const float2* G, const float2* Pt, int J, int m, int n, int p, int L,
                             float2* F, cudaStream_t s) {
  const size_t total = (size_t)J * J * p * m * L;
  if (total == 0) return cudaSuccess;
  const int blocks = (int)((total + 255) / 256 < 152 * 16 ? (total + 255) / 256 : 152 * 16);
  detail::k_mmse_fold<<<blocks, 256, 0, s>>>(G, Pt, J, m, n, p, L, F);
  return cudaGetLastError();
}

}  // namespace ts
