// C ABI of the tuckersinr library: argument checks, workspace carving and
// kernel dispatch.  No allocation, no synchronisation, no exceptions.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "kernels.h"
#include "tuckersinr.h"

#include <math.h>

namespace {

thread_local int g_last_cuda = 0;
// optional caller-owned events recorded around the dominant kernel of the
// next SINR calls on this host thread (ts_set_timing_events)
thread_local cudaEvent_t g_ev_start = nullptr;
thread_local cudaEvent_t g_ev_stop = nullptr;
// optional caller-owned event recorded once the precoders of an SVD call
// are in the workspace (ts_set_phase_event)
thread_local cudaEvent_t g_ev_phase = nullptr;
// SINR sensitivity to R (see k_sinr_finalize) above which a unit is
// re-evaluated from a double-float R with FP64 residuals
// (ts_set_refinement); infinity turns refinement off
thread_local float g_refine_sens = 8.f;
thread_local int g_fit_iters = 40;
// rows per unit of the SVD path (more than kMaxRankM: shared-memory kernels)
constexpr int kMaxRankMLarge = 64;
// launch-shape choices of the batch planner (0: default heuristics)
thread_local ts::Tuning g_tuning = {0, 0};
thread_local bool g_timing_suspended = false;
// subcarrier range of the SINR calls in progress on this host thread (the
// range entry points): local subcarrier 0 is g_kap_off, the dense
// coefficients have g_Kc subcarriers (0: the call's own K)
thread_local int g_kap_off = 0;
thread_local int g_Kc = 0;
struct RangeScope {
  RangeScope(int off, int Kc) { g_kap_off = off; g_Kc = Kc; }
  ~RangeScope() { g_kap_off = 0; g_Kc = 0; }
};

// Side streams on which the UE groups of a several-UE call run concurrently
// (created on first use per device, kept for the life of the process).
constexpr int kSideStreams = 4;
std::mutex g_side_mu;
std::vector<std::vector<cudaStream_t>> g_side;

cudaError_t side_streams(cudaStream_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_side_mu);
  if ((int)g_side.size() <= dev) g_side.resize(dev + 1);
  std::vector<cudaStream_t>& v = g_side[dev];
  while ((int)v.size() < kSideStreams) {
    cudaStream_t st = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    v.push_back(st);
  }
  for (int j = 0; j < kSideStreams; ++j) out[j] = v[j];
  return cudaSuccess;
}

// Finalisation, then the FP64-residual refinement of the units it listed.
// The list counter is zeroed by the link kernel that precedes the finalize
// kernel (one thread of its first CTA); only an SVD call with a single cell
// has no link kernel and zeroes it here.
cudaError_t finalize_refined(const ts::SinrArgs& a, bool svd, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (svd && a.J < 2) e = cudaMemsetAsync(a.rcount, 0, sizeof(int), s);
  if (e == cudaSuccess) e = ts::launch_sinr_finalize(a, svd, s);
  if (e == cudaSuccess && a.refine_sens < INFINITY && a.m <= ts::kMaxRankM)
    e = ts::launch_sinr_refine(a, svd, s);
  return e;
}

// The per-link kernel (the dominant one) bracketed by the timing events,
// then the finalisation.
cudaError_t links_then_finalize(const ts::SinrArgs& a, bool svd, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const bool timed = g_ev_start != nullptr && g_ev_stop != nullptr && !g_timing_suspended;
  if (timed) e = cudaEventRecord(g_ev_start, s);
  if (e == cudaSuccess) e = ts::launch_sinr_links(a, svd, s);
  if (e == cudaSuccess && timed) e = cudaEventRecord(g_ev_stop, s);
  if (e == cudaSuccess) e = finalize_refined(a, svd, s);
  return e;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TS_OK;
  g_last_cuda = (int)e;
  return TS_ERR_CUDA;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// NULL counts as aligned (optional pointers are checked separately)
bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

// Sizes the SINR kernels accept.
int check_dims(const ts_dims* d, bool identity = false) {
  if (d == nullptr) return TS_ERR_NULL;
  if (d->J < 1 || d->M < 1 || d->N < 1 || d->P < 1 || d->K < 1) return TS_ERR_DIMS;
  if (d->m < 1 || d->n < 1 || d->p < 1 || d->L < 1) return TS_ERR_DIMS;
  if (d->m > d->M || d->n > d->N || d->p > d->P) return TS_ERR_DIMS;
  if (d->m > kMaxRankMLarge) return TS_ERR_DIMS;
  if (d->L > d->m || d->L > d->n) return TS_ERR_DIMS;
  // units with more than 16 rows: shared-memory kernels, up to 8 streams
  if (d->m > ts::kMaxRankM && d->L > 8) return TS_ERR_DIMS;
  // staging limits of the kernels: the projections w [subcarrier tile][p]
  // live in shared memory (the dense-channel comparator, C = I, keeps no
  // projections: p = P <= 1024); serving channels of more than 512 columns
  // go through the shared-memory precoder (m <= 16, L <= 8)
  if (d->P > 1024 || (!identity && d->p > ts::kMaxRankPWide) || d->n > 1024) return TS_ERR_DIMS;
  if (d->n > ts::kMaxNRegisterPrecoder && d->m <= ts::kMaxRankM && d->L > 8) return TS_ERR_DIMS;
  if ((int64_t)d->J * d->J > 65535 || d->J > 65535) return TS_ERR_DIMS;
  return TS_OK;
}

// The wideband-precoder path and the adjoints stage C_ik (P x p) and a core
// column chunk whole: p <= 32 and P p <= 8192; the adjoints also need the
// register precoder's full SVD (n <= 512).  The SVD path streams larger
// cores through the wide-core kernel.
int check_narrow(const ts_dims* d) {
  const int st = check_dims(d);
  if (st != TS_OK) return st;
  return ts::wide_core(d->P, d->p) || d->m > ts::kMaxRankM || d->n > ts::kMaxNRegisterPrecoder
             ? TS_ERR_DIMS : TS_OK;
}

// The SVD precoder forms the serving links' channels itself (small cores,
// register-resident units); otherwise a serving pass writes them first.
bool fuses_serve(const ts_dims* d) {
  return d->m <= ts::kMaxRankM && ts::precoder_fuses_serve(d->m, d->n, d->p);
}

// Workspace layout (byte offsets from the base, each 256-byte aligned).
struct Workspace {
  size_t turns = 0, V = 0, Hserv = 0, Wserv = 0, Ueig = 0, lam = 0, conv = 0, Uclose = 0,
         cmask = 0, Eserv = 0, Eint = 0, pflag = 0, F = 0, rlist = 0, rcount = 0, total = 0;
};

Workspace carve(const ts_dims* d, int op) {
  Workspace w;
  size_t o = 0;
  const size_t nch = (size_t)d->J * d->J;
  w.turns = o;
  o = align_up(o + nch * d->P * sizeof(unsigned long long), 256);
  w.Eserv = o;
  o = align_up(o + (size_t)d->J * d->K * d->m * d->L * sizeof(float2), 256);
  w.Eint = o;
  o = align_up(o + (size_t)d->J * (d->J - 1) * d->K * d->m * d->L * sizeof(float2), 256);
  if (op == TS_OP_SINR_SVD) {
    w.V = o;
    o = align_up(o + (size_t)d->J * d->K * d->n * d->L * sizeof(float2), 256);
    if (!fuses_serve(d)) {
      w.Hserv = o;
      o = align_up(o + (size_t)d->J * d->K * d->m * d->n * sizeof(float2), 256);
      if (d->m <= ts::kMaxRankM && d->n <= ts::kMaxNRegisterPrecoder) {
        // the two-phase precoder's eigenvectors, eigenvalues and convergence
        w.Ueig = o;
        o = align_up(o + (size_t)d->J * d->K * ts::kMaxRankM * ts::kMaxRankM * sizeof(float2), 256);
        w.lam = o;
        o = align_up(o + (size_t)d->J * d->K * ts::kMaxRankM * sizeof(float), 256);
        w.conv = o;
        o = align_up(o + (size_t)d->J * d->K, 256);
      }
      if (ts::wide_core(d->P, d->p)) {
        w.Wserv = o;
        o = align_up(o + (size_t)d->J * d->K * d->p * sizeof(float2), 256);
      }
    }
    w.pflag = o;
    o = align_up(o + (size_t)d->J * d->K, 256);
    if (d->m <= 16) {
      // vectors of the units listed for the close-pair refinement
      const int R = d->L + 1 < d->m ? d->L + 1 : d->m;
      w.Uclose = o;
      o = align_up(o + (size_t)d->J * d->K * R * d->m * sizeof(float2), 256);
      w.cmask = o;
      o = align_up(o + (size_t)d->J * d->K * sizeof(int), 256);
    }
  } else {
    w.F = o;
    o = align_up(o + nch * d->p * d->m * d->L * sizeof(float2), 256);
  }
  w.rlist = o;
  o = align_up(o + (size_t)d->J * d->K * sizeof(int), 256);
  w.rcount = o;
  o = align_up(o + sizeof(int), 256);
  w.total = o;
  return w;
}

// Reduced-precision workspace: the ts_sinr_svd workspace, then the core
// rewritten as a tensor-core operand.
size_t prec_workspace_bytes(const ts_dims* d, int prec) {
  return carve(d, TS_OP_SINR_SVD).total + ts::tc_prep_bytes(d->J, d->m, d->L, d->n, d->p, d->K, prec);
}

// Adjoint workspace (byte offsets, each 256-byte aligned).
struct AdjWorkspace {
  size_t turns = 0, Hall = 0, V = 0, Eserv = 0, pflag = 0, U = 0, S = 0, Vm = 0, W = 0, E = 0,
         gE = 0, gH = 0, gV = 0, gw = 0, part = 0, total = 0;
};

AdjWorkspace carve_adjoint(const ts_dims* d, bool svd) {
  AdjWorkspace w;
  size_t o = 0;
  const size_t nch = (size_t)d->J * d->J, K = d->K, m = d->m, n = d->n, L = d->L, p = d->p;
  auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
  w.turns = take(nch * d->P * sizeof(unsigned long long));
  w.Hall = take(nch * K * m * n * sizeof(float2));
  if (svd) {
    w.V = take((size_t)d->J * K * n * L * sizeof(float2));
    w.Eserv = take((size_t)d->J * K * m * L * sizeof(float2));
    w.pflag = take((size_t)d->J * K);
    w.U = take((size_t)d->J * K * m * m * sizeof(float2));
    w.S = take((size_t)d->J * K * m * sizeof(float));
    w.Vm = take((size_t)d->J * K * n * m * sizeof(float2));
  }
  w.W = take(nch * K * p * sizeof(float2));
  w.E = take(nch * K * m * L * sizeof(float2));
  w.gE = take(nch * K * m * L * sizeof(float2));
  w.gH = take(nch * K * m * n * sizeof(float2));
  w.gV = take((size_t)d->J * K * n * L * sizeof(float2));
  w.gw = take(nch * K * p * sizeof(float2));
  w.part = take(ts::adjoint_part_elems(d->J, d->m, d->n, d->p, d->P, d->K) * sizeof(float2));
  w.total = o;
  return w;
}

ts::FitDims fit_dims(const ts_dims* d, int model = TS_MODEL_GROUPWISE) {
  return ts::FitDims{d->J, d->M, d->N, d->P, d->m, d->n, d->p, model, g_fit_iters};
}

// Sizes the fit accepts: ranks up to 256 (the eigensolver blocks stay within
// 512 columns).
int fit_checks(const ts_dims* d) {
  if (d == nullptr) return TS_ERR_NULL;
  if (d->J < 1 || d->M < 1 || d->N < 1 || d->P < 1) return TS_ERR_DIMS;
  if (d->m < 1 || d->n < 1 || d->p < 1 || d->m > d->M || d->n > d->N || d->p > d->P) return TS_ERR_DIMS;
  if (d->m > 256 || d->n > 256 || d->p > 256) return TS_ERR_DIMS;
  if (d->M > 4096 || d->N > 4096 || d->P > 4096 || d->J > 256) return TS_ERR_DIMS;
  return TS_OK;
}

// Sizes the reconstruction accepts: any ranks up to the dimensions (a plain
// mode-product chain; no eigensolver block limit).
int reconstruct_checks(const ts_dims* d) {
  if (d == nullptr) return TS_ERR_NULL;
  if (d->J < 1 || d->M < 1 || d->N < 1 || d->P < 1) return TS_ERR_DIMS;
  if (d->m < 1 || d->n < 1 || d->p < 1 || d->m > d->M || d->n > d->N || d->p > d->P) return TS_ERR_DIMS;
  if (d->M > 4096 || d->N > 4096 || d->P > 4096 || d->J > 256) return TS_ERR_DIMS;
  return TS_OK;
}

int check_coef(const ts_coef* c) {
  if (c == nullptr) return TS_ERR_NULL;
  if (c->mode == TS_COEF_DENSE) {
    if (c->c == nullptr) return TS_ERR_NULL;
    if (!aligned8(c->c)) return TS_ERR_ALIGN;
  } else if (c->mode == TS_COEF_PATHS) {
    if (c->alpha == nullptr || c->tau_s == nullptr) return TS_ERR_NULL;
    if (!aligned8(c->alpha) || ((uintptr_t)c->tau_s & 3u)) return TS_ERR_ALIGN;
  } else {
    return TS_ERR_MODE;
  }
  return TS_OK;
}

ts_dims dense_dims(const ts_dims* d);

ts::SinrArgs base_args(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                       const float* sigma2, float* sinr, uint8_t* flags, char* ws,
                       const Workspace& w) {
  ts::SinrArgs a{};
  a.J = d->J; a.m = d->m; a.n = d->n; a.p = d->p; a.P = d->P; a.K = d->K; a.L = d->L;
  a.coef_mode = coef->mode;
  a.G = reinterpret_cast<const float2*>(G);
  a.C = reinterpret_cast<const float2*>(C);
  a.coef = reinterpret_cast<const float2*>(coef->mode == TS_COEF_DENSE ? coef->c : coef->alpha);
  a.kap_off = g_kap_off;
  a.Kc = g_Kc > 0 ? g_Kc : d->K;
  a.turns = reinterpret_cast<const unsigned long long*>(ws + w.turns);
  a.Eserv = reinterpret_cast<float2*>(ws + w.Eserv);
  a.Eint = reinterpret_cast<float2*>(ws + w.Eint);
  a.sigma2 = sigma2;
  a.sinr = sinr;
  a.flags = flags;
  a.rlist = reinterpret_cast<int*>(ws + w.rlist);
  a.rcount = reinterpret_cast<int*>(ws + w.rcount);
  a.refine_sens = g_refine_sens;
  a.link_variant = g_tuning.link_variant;
  a.precoder_split = g_tuning.precoder_split;
  return a;
}

}  // namespace

namespace ts {
int record_cuda_error(cudaError_t e) { return cuda_status(e); }
void set_tuning(Tuning t) { g_tuning = t; }
void suspend_timing(bool suspended) { g_timing_suspended = suspended; }
}  // namespace ts

extern "C" {

const char* ts_status_string(int status) {
  switch (status) {
    case TS_OK: return "ok";
    case TS_ERR_DIMS: return "sizes out of range or inconsistent";
    case TS_ERR_NULL: return "a required pointer is NULL";
    case TS_ERR_ALIGN: return "a pointer is not suitably aligned";
    case TS_ERR_WORKSPACE: return "workspace too small";
    case TS_ERR_CUDA: return "CUDA launch failed";
    case TS_ERR_MODE: return "unknown coefficient mode or operation";
    default: return "unknown status";
  }
}

int ts_last_cuda_error(void) { return g_last_cuda; }

int ts_abi_version(void) { return 1; }

void ts_set_timing_events(void* start, void* stop) {
  g_ev_start = static_cast<cudaEvent_t>(start);
  g_ev_stop = static_cast<cudaEvent_t>(stop);
}

void ts_set_phase_event(void* event) { g_ev_phase = static_cast<cudaEvent_t>(event); }

void ts_set_fit_iterations(int iterations) { g_fit_iters = iterations > 0 ? iterations : 40; }

void ts_set_refinement(float threshold) {
  g_refine_sens = threshold < 0.f ? INFINITY : threshold;
}

size_t ts_workspace_bytes(const ts_dims* d, int op) {
  if (d == nullptr) return 0;
  if (op == TS_OP_SINR_SVD_MULTIUSER || op == TS_OP_DENSE_SVD_MULTIUSER) {
    const ts_dims e = op == TS_OP_DENSE_SVD_MULTIUSER ? dense_dims(d) : *d;
    if (check_dims(&e, op == TS_OP_DENSE_SVD_MULTIUSER) != TS_OK) return 0;
    return 2 * carve(&e, TS_OP_SINR_SVD).total;
  }
  if (op == TS_OP_DENSE_SVD || op == TS_OP_DENSE_MMSE) {
    const ts_dims e = dense_dims(d);
    if ((op == TS_OP_DENSE_SVD ? check_dims(&e, true) : check_narrow(&e)) != TS_OK) return 0;
    return carve(&e, op == TS_OP_DENSE_SVD ? TS_OP_SINR_SVD : TS_OP_SINR_MMSE).total;
  }
  if (check_dims(d) != TS_OK) return 0;
  if (op == TS_OP_TUCKER_FIT) return fit_checks(d) == TS_OK ? ts::fit_workspace_bytes(fit_dims(d)) : 0;
  if (op == TS_OP_TUCKER_FIT_SHARED || op == TS_OP_TUCKER_FIT_INDIVIDUAL)
    return fit_checks(d) == TS_OK
               ? ts::fit_workspace_bytes(fit_dims(d, op == TS_OP_TUCKER_FIT_SHARED ? TS_MODEL_SHARED
                                                                                 : TS_MODEL_INDIVIDUAL))
               : 0;
  if (op == TS_OP_RECONSTRUCT)
    return reconstruct_checks(d) == TS_OK ? ts::reconstruct_workspace_bytes(fit_dims(d)) : 0;
  if (op == TS_OP_SINR_SVD_ADJOINT || op == TS_OP_SINR_MMSE_ADJOINT)
    return check_narrow(d) == TS_OK ? carve_adjoint(d, op == TS_OP_SINR_SVD_ADJOINT).total : 0;
  if (op == TS_OP_SINR_MMSE && check_narrow(d) != TS_OK) return 0;
  if (op == TS_OP_SINR_SVD_TF32 || op == TS_OP_SINR_SVD_BF16X2 || op == TS_OP_SINR_SVD_TF32X3)
    return ts::tc_supported(d->m, d->L, d->p) && check_narrow(d) == TS_OK
               ? prec_workspace_bytes(d, op == TS_OP_SINR_SVD_TF32     ? TS_PREC_TF32
                                         : op == TS_OP_SINR_SVD_TF32X3 ? TS_PREC_TF32X3
                                                                       : TS_PREC_BF16X2)
               : 0;
  if (op != TS_OP_SINR_SVD && op != TS_OP_SINR_MMSE) return 0;
  return carve(d, op).total;
}

int ts_coefficients(const ts_dims* d, const ts_c64* alpha, const float* tau_s, ts_c64* c,
                    void* stream) {
  if (d == nullptr || alpha == nullptr || tau_s == nullptr || c == nullptr) return TS_ERR_NULL;
  if (d->J < 1 || d->K < 1 || d->P < 1) return TS_ERR_DIMS;
  if (!aligned8(alpha) || !aligned8(c) || ((uintptr_t)tau_s & 3u)) return TS_ERR_ALIGN;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nch = d->J * d->J;
  return cuda_status(ts::launch_coefficients(reinterpret_cast<const float2*>(alpha), tau_s,
                                             d->delta_f_hz, nch, d->K, d->P,
                                             reinterpret_cast<float2*>(c), s));
}

int ts_project_precoder(const ts_dims* d, const ts_c64* B, const ts_c64* Pfull, ts_c64* Pt,
                        void* stream) {
  int st = check_dims(d);
  if (st != TS_OK) return st;
  if (B == nullptr || Pfull == nullptr || Pt == nullptr) return TS_ERR_NULL;
  if (!aligned8(B) || !aligned8(Pfull) || !aligned8(Pt)) return TS_ERR_ALIGN;
  return cuda_status(ts::launch_project_precoder(
      reinterpret_cast<const float2*>(B), reinterpret_cast<const float2*>(Pfull), d->J, d->N, d->n,
      d->L, reinterpret_cast<float2*>(Pt), static_cast<cudaStream_t>(stream)));
}

}  // extern "C"

namespace {

int adjoint_impl(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                 const ts_c64* Pt, const float* sigma2, const float* dsinr, ts_c64* dG, ts_c64* dC,
                 ts_c64* dPt, float* sinr, void* ws, size_t ws_bytes, void* stream) {
  const bool svd = Pt == nullptr;
  int st = check_narrow(d);
  if (st != TS_OK) return st;
  st = check_coef(coef);
  if (st != TS_OK) return st;
  if (G == nullptr || C == nullptr || sigma2 == nullptr || dsinr == nullptr || dG == nullptr ||
      dC == nullptr || (!svd && dPt == nullptr))
    return TS_ERR_NULL;
  if (!aligned8(G) || !aligned8(C) || !aligned8(Pt) || !aligned8(dG) || !aligned8(dC) ||
      !aligned8(dPt) || ((uintptr_t)sigma2 & 3u) || ((uintptr_t)dsinr & 3u) ||
      ((uintptr_t)sinr & 3u))
    return TS_ERR_ALIGN;
  const AdjWorkspace w = carve_adjoint(d, svd);
  if (ws == nullptr || ws_bytes < w.total) return TS_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return TS_ERR_ALIGN;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  Workspace fw;
  fw.turns = w.turns;
  ts::SinrArgs a = base_args(d, coef, G, C, sigma2, sinr, nullptr, base, fw);
  a.rlist = nullptr;                 // no finalize pass here
  a.rcount = nullptr;
  a.Hserv = reinterpret_cast<float2*>(base + w.Hall);
  a.serv_stride = d->J + 1;          // serving link (k, k) inside the all-link layout
  cudaError_t e = cudaSuccess;
  if (coef->mode == TS_COEF_PATHS)
    e = ts::launch_turns(coef->tau_s, d->delta_f_hz, d->J * d->J * d->P,
                         reinterpret_cast<unsigned long long*>(base + w.turns), s);
  if (e == cudaSuccess) e = ts::launch_sinr_rebuild(a, s);
  if (svd && e == cudaSuccess) {
    a.V = reinterpret_cast<float2*>(base + w.V);
    a.Eserv = reinterpret_cast<float2*>(base + w.Eserv);
    a.pflag = reinterpret_cast<uint8_t*>(base + w.pflag);
    a.Uout = reinterpret_cast<float2*>(base + w.U);
    a.Sout = reinterpret_cast<float*>(base + w.S);
    a.Vmout = reinterpret_cast<float2*>(base + w.Vm);
    e = ts::launch_svd_precoder(a, s);
  }
  if (e == cudaSuccess) {
    ts::AdjointWork aw{};
    aw.Pt = reinterpret_cast<const float2*>(Pt);
    aw.dsinr = dsinr;
    aw.sinr = sinr;
    aw.W = reinterpret_cast<float2*>(base + w.W);
    aw.E = reinterpret_cast<float2*>(base + w.E);
    aw.gE = reinterpret_cast<float2*>(base + w.gE);
    aw.gH = reinterpret_cast<float2*>(base + w.gH);
    aw.gV = reinterpret_cast<float2*>(base + w.gV);
    aw.gw = reinterpret_cast<float2*>(base + w.gw);
    aw.dG = reinterpret_cast<float2*>(dG);
    aw.dC = reinterpret_cast<float2*>(dC);
    aw.part = reinterpret_cast<float2*>(base + w.part);
    aw.dPt = reinterpret_cast<float2*>(dPt);
    e = ts::launch_adjoint(a, aw, s);
  }
  return cuda_status(e);
}

}  // namespace

extern "C" {

int ts_sinr_svd_adjoint(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                        const float* sigma2, const float* dsinr, ts_c64* dG, ts_c64* dC,
                        float* sinr, void* ws, size_t ws_bytes, void* stream) {
  return adjoint_impl(d, coef, G, C, nullptr, sigma2, dsinr, dG, dC, nullptr, sinr, ws, ws_bytes,
                      stream);
}

int ts_sinr_mmse_adjoint(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                         const ts_c64* Pt, const float* sigma2, const float* dsinr, ts_c64* dG,
                         ts_c64* dC, ts_c64* dPt, float* sinr, void* ws, size_t ws_bytes,
                         void* stream) {
  if (Pt == nullptr) return TS_ERR_NULL;
  return adjoint_impl(d, coef, G, C, Pt, sigma2, dsinr, dG, dC, dPt, sinr, ws, ws_bytes, stream);
}

int ts_tucker_fit(const ts_dims* d, const ts_c64* X, int S, int init, ts_c64* A, ts_c64* B,
                  ts_c64* C, ts_c64* G, double* g_hist, void* ws, size_t ws_bytes, void* stream) {
  return ts_tucker_fit_model(d, X, S, init, TS_MODEL_GROUPWISE, A, B, C, G, g_hist, ws, ws_bytes,
                             stream);
}

int ts_tucker_fit_model(const ts_dims* d, const ts_c64* X, int S, int init, int model, ts_c64* A,
                        ts_c64* B, ts_c64* C, ts_c64* G, double* g_hist, void* ws, size_t ws_bytes,
                        void* stream) {
  int st = fit_checks(d);
  if (st != TS_OK) return st;
  if (model != TS_MODEL_GROUPWISE && model != TS_MODEL_SHARED && model != TS_MODEL_INDIVIDUAL)
    return TS_ERR_MODE;
  if (S < 0 || (init != 0 && init != 1)) return TS_ERR_MODE;
  if (X == nullptr || A == nullptr || B == nullptr || C == nullptr || G == nullptr) return TS_ERR_NULL;
  if (!aligned8(X) || !aligned8(A) || !aligned8(B) || !aligned8(C) || !aligned8(G) || !aligned8(g_hist))
    return TS_ERR_ALIGN;
  const ts::FitDims f = fit_dims(d, model);
  if (ws == nullptr || ws_bytes < ts::fit_workspace_bytes(f)) return TS_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return TS_ERR_ALIGN;
  return cuda_status(ts::launch_fit(f, reinterpret_cast<const float2*>(X), S, init,
                                    reinterpret_cast<float2*>(A), reinterpret_cast<float2*>(B),
                                    reinterpret_cast<float2*>(C), reinterpret_cast<float2*>(G),
                                    g_hist, ws, static_cast<cudaStream_t>(stream)));
}

int ts_tucker_reconstruct(const ts_dims* d, int model, const ts_c64* A, const ts_c64* B,
                          const ts_c64* C, const ts_c64* G, ts_c64* Xhat, void* ws, size_t ws_bytes,
                          void* stream) {
  int st = reconstruct_checks(d);
  if (st != TS_OK) return st;
  if (model != TS_MODEL_GROUPWISE && model != TS_MODEL_SHARED && model != TS_MODEL_INDIVIDUAL)
    return TS_ERR_MODE;
  if (A == nullptr || B == nullptr || C == nullptr || G == nullptr || Xhat == nullptr) return TS_ERR_NULL;
  if (!aligned8(A) || !aligned8(B) || !aligned8(C) || !aligned8(G) || !aligned8(Xhat)) return TS_ERR_ALIGN;
  const ts::FitDims f = fit_dims(d, model);
  if (ws == nullptr || ws_bytes < ts::reconstruct_workspace_bytes(f)) return TS_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return TS_ERR_ALIGN;
  return cuda_status(ts::launch_reconstruct(
      f, reinterpret_cast<const float2*>(A), reinterpret_cast<const float2*>(B),
      reinterpret_cast<const float2*>(C), reinterpret_cast<const float2*>(G),
      reinterpret_cast<float2*>(Xhat), ws, static_cast<cudaStream_t>(stream)));
}

int ts_project_precoder_adjoint(const ts_dims* d, const ts_c64* Pfull, const ts_c64* dPt,
                                ts_c64* dB, void* stream) {
  int st = check_dims(d);
  if (st != TS_OK) return st;
  if (Pfull == nullptr || dPt == nullptr || dB == nullptr) return TS_ERR_NULL;
  if (!aligned8(Pfull) || !aligned8(dPt) || !aligned8(dB)) return TS_ERR_ALIGN;
  return cuda_status(ts::launch_project_precoder_adjoint(
      reinterpret_cast<const float2*>(Pfull), reinterpret_cast<const float2*>(dPt), d->J, d->N,
      d->n, d->L, reinterpret_cast<float2*>(dB), static_cast<cudaStream_t>(stream)));
}

}  // extern "C"

namespace {

// The dense-channel comparator runs the compressed path on the trivial
// factorisation G = X, C = I: (m, n, p) = (M, N, P).
ts_dims dense_dims(const ts_dims* d) {
  ts_dims e = *d;
  e.m = d->M;
  e.n = d->N;
  e.p = d->P;
  return e;
}

int sinr_common_checks(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                       bool identity, const float* sigma2, float* sinr, void* ws, size_t ws_bytes,
                       int op) {
  int st = op == TS_OP_SINR_MMSE ? check_narrow(d) : check_dims(d, identity);
  if (st != TS_OK) return st;
  st = check_coef(coef);
  if (st != TS_OK) return st;
  if (G == nullptr || (!identity && C == nullptr) || sigma2 == nullptr || sinr == nullptr)
    return TS_ERR_NULL;
  if (!aligned8(G) || !aligned8(C) || ((uintptr_t)sigma2 & 3u) || ((uintptr_t)sinr & 3u))
    return TS_ERR_ALIGN;
  const size_t need = carve(d, op).total;
  if (ws == nullptr || ws_bytes < need) return TS_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return TS_ERR_ALIGN;
  return TS_OK;
}

int sinr_mmse_impl(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                   bool identity, const ts_c64* Pt, const float* sigma2, float* sinr,
                   uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  int st = sinr_common_checks(d, coef, G, C, identity, sigma2, sinr, ws, ws_bytes, TS_OP_SINR_MMSE);
  if (st != TS_OK) return st;
  if (Pt == nullptr) return TS_ERR_NULL;
  if (!aligned8(Pt)) return TS_ERR_ALIGN;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace w = carve(d, TS_OP_SINR_MMSE);
  char* base = static_cast<char*>(ws);
  ts::SinrArgs a = base_args(d, coef, G, C, sigma2, sinr, flags, base, w);
  a.identity_C = identity;
  float2* F = reinterpret_cast<float2*>(base + w.F);
  a.F = F;
  cudaError_t e = cudaSuccess;
  if (coef->mode == TS_COEF_PATHS)
    e = ts::launch_turns(coef->tau_s, d->delta_f_hz, d->J * d->J * d->P,
                         reinterpret_cast<unsigned long long*>(base + w.turns), s);
  if (e == cudaSuccess)
    e = ts::launch_mmse_fold(a.G, reinterpret_cast<const float2*>(Pt), d->J, d->m, d->n, d->p,
                             d->L, F, s);
  if (e == cudaSuccess) e = links_then_finalize(a, false, s);
  return cuda_status(e);
}

// The SVD precoders into the workspace.  With tc_prep (TF32X3, a core that
// the precoder does not contract itself) the tensor-core operands are
// prepared into tc_prep first, the serving links' projections included, and
// the serving pass runs on the tensor cores.
int svd_precoders_impl(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                       bool identity, void* ws, size_t ws_bytes, void* stream,
                       void* tc_prep = nullptr) {
  static const float kOne = 1.f;
  static float dummy_out;
  int st = sinr_common_checks(d, coef, G, C, identity, &kOne, &dummy_out, ws, ws_bytes,
                              TS_OP_SINR_SVD);
  if (st != TS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace w = carve(d, TS_OP_SINR_SVD);
  char* base = static_cast<char*>(ws);
  ts::SinrArgs a = base_args(d, coef, G, C, nullptr, nullptr, nullptr, base, w);
  a.identity_C = identity;
  a.V = reinterpret_cast<float2*>(base + w.V);
  a.pflag = reinterpret_cast<uint8_t*>(base + w.pflag);
  cudaError_t e = cudaSuccess;
  if (coef->mode == TS_COEF_PATHS)
    e = ts::launch_turns(coef->tau_s, d->delta_f_hz, d->J * d->J * d->P,
                         reinterpret_cast<unsigned long long*>(base + w.turns), s);
  a.fuse_serve = fuses_serve(d) ? 1 : 0;
  if (!a.fuse_serve) {
    a.Hserv = reinterpret_cast<float2*>(base + w.Hserv);
    if (w.Ueig != 0) {
      a.Ueig = reinterpret_cast<float2*>(base + w.Ueig);
      a.lam_eig = reinterpret_cast<float*>(base + w.lam);
      a.conv_eig = reinterpret_cast<uint8_t*>(base + w.conv);
    }
    a.serv_stride = 1;
    if (w.Wserv != 0 && !identity) a.Wserv = reinterpret_cast<float2*>(base + w.Wserv);
    if (tc_prep != nullptr) {
      if (e == cudaSuccess) e = ts::launch_tc_operands(a, TS_PREC_TF32X3, true, tc_prep, s);
      if (e == cudaSuccess) e = ts::launch_serving_tc(a, tc_prep, s);
    } else if (e == cudaSuccess) {
      e = ts::launch_sinr_serving(a, s);
    }
  }
  // units with a close pair of singular values are listed by the precoder
  // kernels and their precoders refined from H~ in double-float (off with
  // the refinement)
  a.list_close = a.refine_sens < INFINITY && w.Uclose != 0 ? 1 : 0;
  if (a.list_close) {
    a.Uclose = reinterpret_cast<float2*>(base + w.Uclose);
    a.close_mask = reinterpret_cast<int*>(base + w.cmask);
  }
  if (e == cudaSuccess && a.list_close) e = cudaMemsetAsync(a.rcount, 0, sizeof(int), s);
  if (e == cudaSuccess) e = ts::launch_svd_precoder(a, s);
  if (e == cudaSuccess && a.list_close) e = ts::launch_precoder_refine(a, s);
  if (e == cudaSuccess && g_ev_phase != nullptr && !g_timing_suspended) e = cudaEventRecord(g_ev_phase, s);
  return cuda_status(e);
}

// operands_ready: svd_precoders_impl prepared the operands (all but the
// precoder rows) into the same buffer
int svd_from_precoders_prec_impl(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                                 const ts_c64* C, const float* sigma2, int prec, float* sinr,
                                 uint8_t* flags, void* ws, size_t ws_bytes, void* stream,
                                 bool operands_ready = false) {
  int st = sinr_common_checks(d, coef, G, C, false, sigma2, sinr, ws, ws_bytes, TS_OP_SINR_SVD);
  if (st != TS_OK) return st;
  if (ws_bytes < prec_workspace_bytes(d, prec)) return TS_ERR_WORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace w = carve(d, TS_OP_SINR_SVD);
  char* base = static_cast<char*>(ws);
  ts::SinrArgs a = base_args(d, coef, G, C, sigma2, sinr, flags, base, w);
  a.V = reinterpret_cast<float2*>(base + w.V);
  a.pflag = reinterpret_cast<uint8_t*>(base + w.pflag);
  void* prep = base + w.total;
  const bool timed = g_ev_start != nullptr && g_ev_stop != nullptr && !g_timing_suspended;
  cudaError_t e = operands_ready ? ts::launch_tc_vtiles(a, prec, prep, s) : ts::launch_core_prep(a, prec, prep, s);
  if (e == cudaSuccess && timed) e = cudaEventRecord(g_ev_start, s);
  if (e == cudaSuccess) e = ts::launch_sinr_links_tc(a, prec, prep, s);
  if (e == cudaSuccess && timed) e = cudaEventRecord(g_ev_stop, s);
  if (e == cudaSuccess) e = finalize_refined(a, true, s);
  return cuda_status(e);
}

int check_prec(const ts_dims* d, int precision) {
  if (precision != TS_PREC_TF32 && precision != TS_PREC_BF16X2 && precision != TS_PREC_TF32X3)
    return TS_ERR_MODE;
  int st = check_narrow(d);
  if (st != TS_OK) return st;
  return ts::tc_supported(d->m, d->L, d->p) ? TS_OK : TS_ERR_MODE;
}

int svd_from_precoders_impl(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                            const ts_c64* C, bool identity, const float* sigma2, float* sinr,
                            uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  int st = sinr_common_checks(d, coef, G, C, identity, sigma2, sinr, ws, ws_bytes, TS_OP_SINR_SVD);
  if (st != TS_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Workspace w = carve(d, TS_OP_SINR_SVD);
  char* base = static_cast<char*>(ws);
  ts::SinrArgs a = base_args(d, coef, G, C, sigma2, sinr, flags, base, w);
  a.identity_C = identity;
  a.V = reinterpret_cast<float2*>(base + w.V);
  a.pflag = reinterpret_cast<uint8_t*>(base + w.pflag);
  return cuda_status(links_then_finalize(a, true, s));
}

// U UEs per cell (Section 4): UE group u holds UE u of every cell, its links
// at G + u J^2 p m n (likewise C, the coefficients, sigma2, sinr, flags).
// Every BS k interferes with its first UE's precoder, so group 0's
// precoders V_0 stay in the first single-UE workspace and every group reads
// them for its interfering links.  With two single-UE workspaces the groups
// run one after the other, the later ones reusing the second; with one per
// group (U of them) groups 1.. run concurrently on side streams once V_0 is
// ready, each in its own, and the caller's stream waits for all of them.
int svd_multiuser_impl(const ts_dims* d, int U, const ts_coef* coef, const ts_c64* G,
                       const ts_c64* C, bool identity, const float* sigma2, float* sinr,
                       uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  if (U < 1) return TS_ERR_DIMS;
  int st = sinr_common_checks(d, coef, G, C, identity, sigma2, sinr, ws, ws_bytes, TS_OP_SINR_SVD);
  if (st != TS_OK) return st;
  const Workspace w = carve(d, TS_OP_SINR_SVD);
  if (ws_bytes < 2 * w.total) return TS_ERR_WORKSPACE;
  const bool concurrent = U > 1 && ws_bytes >= (size_t)U * w.total;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t nch = (size_t)d->J * d->J;
  char* base0 = static_cast<char*>(ws);
  auto group_coef = [&](int u) {
    ts_coef cu = *coef;
    if (cu.mode == TS_COEF_DENSE) {
      cu.c = coef->c + (size_t)u * nch * d->K * d->P;
    } else {
      cu.alpha = coef->alpha + (size_t)u * nch * d->P;
      cu.tau_s = coef->tau_s + (size_t)u * nch * d->P;
    }
    return cu;
  };
  // one UE group: its precoders (serving effective channels, flags) in
  // `base`, its links against V_0, its finalisation
  auto run_group = [&](int u, char* base, cudaStream_t gs) -> int {
    const ts_coef cu = group_coef(u);
    const ts_c64* Gu = G + (size_t)u * nch * d->p * d->m * d->n;
    const ts_c64* Cu = identity ? nullptr : C + (size_t)u * nch * d->P * d->p;
    int r = svd_precoders_impl(d, &cu, Gu, Cu, identity, base, w.total, gs);
    if (r != TS_OK) return r;
    ts::SinrArgs a = base_args(d, &cu, Gu, Cu, sigma2 + (size_t)u * d->J,
                               sinr + (size_t)u * d->J * d->K * d->L,
                               flags == nullptr ? nullptr : flags + (size_t)u * d->J * d->K, base, w);
    a.identity_C = identity;
    a.V = reinterpret_cast<float2*>(base0 + w.V);
    a.pflag = reinterpret_cast<uint8_t*>(base + w.pflag);
    return cuda_status(links_then_finalize(a, true, gs));
  };
  if (!concurrent) {
    for (int u = 0; u < U; ++u) {
      const int r = run_group(u, base0 + (u == 0 ? 0 : w.total), s);
      if (r != TS_OK) return r;
    }
    return TS_OK;
  }
  cudaStream_t side[kSideStreams];
  cudaError_t e = side_streams(side);
  if (e != cudaSuccess) return cuda_status(e);
  const int nside = U - 1 < kSideStreams ? U - 1 : kSideStreams;
  // group 0: precoders, then V_0 is published to the side streams
  const ts_coef c0 = group_coef(0);
  st = svd_precoders_impl(d, &c0, G, C, identity, base0, w.total, stream);
  if (st != TS_OK) return st;
  cudaEvent_t ev[kSideStreams + 1] = {};
  for (int j = 0; j <= nside && e == cudaSuccess; ++j)
    e = cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  for (int j = 0; j < nside && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(side[j], ev[0], 0);
  if (e == cudaSuccess) {
    ts::SinrArgs a = base_args(d, &c0, G, C, sigma2, sinr, flags, base0, w);
    a.identity_C = identity;
    a.V = reinterpret_cast<float2*>(base0 + w.V);
    a.pflag = reinterpret_cast<uint8_t*>(base0 + w.pflag);
    e = links_then_finalize(a, true, s);
  }
  for (int u = 1; u < U && e == cudaSuccess; ++u) {
    st = run_group(u, base0 + (size_t)u * w.total, side[(u - 1) % nside]);
    if (st != TS_OK) break;
  }
  // the caller's stream waits for every side stream, also after a failed
  // group (work already queued there must not outlive the caller's buffers)
  for (int j = 0; j < nside; ++j) {
    if (ev[1 + j] == nullptr) continue;
    const cudaError_t er = cudaEventRecord(ev[1 + j], side[j]);
    const cudaError_t ew = er == cudaSuccess ? cudaStreamWaitEvent(s, ev[1 + j], 0) : er;
    if (e == cudaSuccess) e = ew;
  }
  for (int j = 0; j <= nside; ++j)
    if (ev[j] != nullptr) cudaEventDestroy(ev[j]);       // released once complete
  if (e != cudaSuccess) return cuda_status(e);
  return st;
}

}  // namespace

extern "C" {

int ts_sinr_svd_multiuser(const ts_dims* d, int U, const ts_coef* coef, const ts_c64* G,
                          const ts_c64* C, const float* sigma2, float* sinr, uint8_t* flags,
                          void* ws, size_t ws_bytes, void* stream) {
  return svd_multiuser_impl(d, U, coef, G, C, false, sigma2, sinr, flags, ws, ws_bytes, stream);
}

int ts_dense_sinr_svd_multiuser(const ts_dims* d, int U, const ts_coef* coef, const ts_c64* X,
                                const float* sigma2, float* sinr, uint8_t* flags, void* ws,
                                size_t ws_bytes, void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  const ts_dims e = dense_dims(d);
  return svd_multiuser_impl(&e, U, coef, X, nullptr, true, sigma2, sinr, flags, ws, ws_bytes,
                            stream);
}

int ts_sinr_mmse(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                 const ts_c64* Pt, const float* sigma2, float* sinr, uint8_t* flags, void* ws,
                 size_t ws_bytes, void* stream) {
  return sinr_mmse_impl(d, coef, G, C, false, Pt, sigma2, sinr, flags, ws, ws_bytes, stream);
}

int ts_svd_precoders(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                     void* ws, size_t ws_bytes, void* stream) {
  return svd_precoders_impl(d, coef, G, C, false, ws, ws_bytes, stream);
}

int ts_sinr_svd_from_precoders(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                               const ts_c64* C, const float* sigma2, float* sinr, uint8_t* flags,
                               void* ws, size_t ws_bytes, void* stream) {
  return svd_from_precoders_impl(d, coef, G, C, false, sigma2, sinr, flags, ws, ws_bytes, stream);
}

int ts_sinr_svd(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                const float* sigma2, float* sinr, uint8_t* flags, void* ws, size_t ws_bytes,
                void* stream) {
  int st = svd_precoders_impl(d, coef, G, C, false, ws, ws_bytes, stream);
  if (st != TS_OK) return st;
  return svd_from_precoders_impl(d, coef, G, C, false, sigma2, sinr, flags, ws, ws_bytes, stream);
}

int ts_sinr_svd_prec(const ts_dims* d, const ts_coef* coef, const ts_c64* G, const ts_c64* C,
                     const float* sigma2, int precision, float* sinr, uint8_t* flags, void* ws,
                     size_t ws_bytes, void* stream) {
  if (precision == TS_PREC_FP32)
    return ts_sinr_svd(d, coef, G, C, sigma2, sinr, flags, ws, ws_bytes, stream);
  int st = check_prec(d, precision);
  if (st != TS_OK) return st;
  if (ws != nullptr && ws_bytes < prec_workspace_bytes(d, precision)) return TS_ERR_WORKSPACE;
  // TF32X3 also forms the serving channels on the tensor cores (where the
  // precoder reads them from the serving pass)
  const bool tc_serve = precision == TS_PREC_TF32X3 && ws != nullptr && !fuses_serve(d);
  void* prep = tc_serve ? static_cast<char*>(ws) + carve(d, TS_OP_SINR_SVD).total : nullptr;
  st = svd_precoders_impl(d, coef, G, C, false, ws, ws_bytes, stream, prep);
  if (st != TS_OK) return st;
  return svd_from_precoders_prec_impl(d, coef, G, C, sigma2, precision, sinr, flags, ws, ws_bytes,
                                      stream, tc_serve);
}

int ts_sinr_svd_from_precoders_prec(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                                    const ts_c64* C, const float* sigma2, int precision,
                                    float* sinr, uint8_t* flags, void* ws, size_t ws_bytes,
                                    void* stream) {
  if (precision == TS_PREC_FP32)
    return ts_sinr_svd_from_precoders(d, coef, G, C, sigma2, sinr, flags, ws, ws_bytes, stream);
  int st = check_prec(d, precision);
  if (st != TS_OK) return st;
  return svd_from_precoders_prec_impl(d, coef, G, C, sigma2, precision, sinr, flags, ws, ws_bytes,
                                      stream);
}

int ts_dense_sinr_svd(const ts_dims* d, const ts_coef* coef, const ts_c64* X, const float* sigma2,
                      float* sinr, uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  const ts_dims e = dense_dims(d);
  int st = svd_precoders_impl(&e, coef, X, nullptr, true, ws, ws_bytes, stream);
  if (st != TS_OK) return st;
  return svd_from_precoders_impl(&e, coef, X, nullptr, true, sigma2, sinr, flags, ws, ws_bytes,
                                 stream);
}

int ts_dense_sinr_mmse(const ts_dims* d, const ts_coef* coef, const ts_c64* X, const ts_c64* Pfull,
                       const float* sigma2, float* sinr, uint8_t* flags, void* ws, size_t ws_bytes,
                       void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  const ts_dims e = dense_dims(d);
  return sinr_mmse_impl(&e, coef, X, nullptr, true, Pfull, sigma2, sinr, flags, ws, ws_bytes,
                        stream);
}

int ts_sinr_svd_range(const ts_dims* d, int kappa0, int count, const ts_coef* coef, const ts_c64* G,
                      const ts_c64* C, const float* sigma2, int precision, float* sinr,
                      uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  if (kappa0 < 0 || count < 1 || (int64_t)kappa0 + count > d->K) return TS_ERR_DIMS;
  ts_dims r = *d;
  r.K = count;
  RangeScope scope(kappa0, d->K);
  return ts_sinr_svd_prec(&r, coef, G, C, sigma2, precision, sinr, flags, ws, ws_bytes, stream);
}

int ts_sinr_mmse_range(const ts_dims* d, int kappa0, int count, const ts_coef* coef, const ts_c64* G,
                       const ts_c64* C, const ts_c64* Pt, const float* sigma2, float* sinr,
                       uint8_t* flags, void* ws, size_t ws_bytes, void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  if (kappa0 < 0 || count < 1 || (int64_t)kappa0 + count > d->K) return TS_ERR_DIMS;
  ts_dims r = *d;
  r.K = count;
  RangeScope scope(kappa0, d->K);
  return ts_sinr_mmse(&r, coef, G, C, Pt, sigma2, sinr, flags, ws, ws_bytes, stream);
}

}  // extern "C"
