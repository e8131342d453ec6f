// Batched evaluation of many independent systems with their own sizes: the
// planner checks every instance, optionally autotunes the launch shapes of
// each new shape class, and captures all instances' kernels into one CUDA
// graph (instances spread over four parallel branches, so that small systems
// overlap; the instances of a branch share its workspace slot);
// ts_batch_launch replays it with one graph launch.
//
// Autotuning knobs (SinrArgs): the interfering-link kernel of the FP32 SVD
// path (two rows x two subcarriers per lane, or one row per lane) and the
// precoder tile (subcarriers per CTA halved 0 or 1 times).  Each candidate is
// timed with CUDA events on the instance's own data (one warm-up and three
// timed evaluations) and the fastest is kept in a process-wide table keyed by
// the shape class.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.h"
#include "tuckersinr.h"

struct ts_batch_plan {
  std::vector<ts_instance> inst;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

constexpr int kBranches = 4;

std::mutex g_table_mutex;
std::map<std::string, ts::Tuning> g_table;

int ws_op(const ts_instance& x) {
  if (x.op == TS_OP_SINR_MMSE) return TS_OP_SINR_MMSE;
  if (x.precision == TS_PREC_TF32) return TS_OP_SINR_SVD_TF32;
  if (x.precision == TS_PREC_BF16X2) return TS_OP_SINR_SVD_BF16X2;
  if (x.precision == TS_PREC_TF32X3) return TS_OP_SINR_SVD_TF32X3;
  return TS_OP_SINR_SVD;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace slots: instance j runs on branch j % kBranches, and the instances
// of one branch run one after the other, so they share that branch's slot
// (each call writes every byte of scratch it reads before reading it).
// slot[b] = offset of branch b's slot; returns the total, 0 if an instance
// is invalid.
size_t slot_layout(const ts_instance* inst, int n, size_t* slot, size_t* slot_bytes) {
  size_t need[kBranches] = {};
  for (int j = 0; j < n; ++j) {
    const size_t b = ts_workspace_bytes(&inst[j].d, ws_op(inst[j]));
    if (b == 0) return 0;
    if (b > need[j % kBranches]) need[j % kBranches] = b;
  }
  size_t o = 0;
  for (int b = 0; b < kBranches; ++b) {
    slot[b] = o;
    slot_bytes[b] = need[b];
    o += align256(need[b]);
  }
  return o;
}

std::string class_key(const ts_instance& x) {
  char buf[160];
  snprintf(buf, sizeof buf, "op%d_prec%d_J%d_m%d_n%d_p%d_P%d_L%d_K%d_coef%d", x.op, x.precision,
           x.d.J, x.d.m, x.d.n, x.d.p, x.d.P, x.d.L, x.d.K, x.coef.mode);
  return buf;
}

// Sizes, operation, precision and pointers, checked without touching the
// device.
int check_instance(const ts_instance& x) {
  if (x.op != TS_OP_SINR_SVD && x.op != TS_OP_SINR_MMSE) return TS_ERR_MODE;
  if (x.precision != TS_PREC_FP32 && x.precision != TS_PREC_TF32 && x.precision != TS_PREC_BF16X2 &&
      x.precision != TS_PREC_TF32X3)
    return TS_ERR_MODE;
  if (x.op == TS_OP_SINR_MMSE && x.precision != TS_PREC_FP32) return TS_ERR_MODE;
  if (ts_workspace_bytes(&x.d, ws_op(x)) == 0) return TS_ERR_DIMS;
  if (x.G == nullptr || x.C == nullptr || x.sigma2 == nullptr || x.sinr == nullptr) return TS_ERR_NULL;
  if (x.op == TS_OP_SINR_MMSE && x.Pt == nullptr) return TS_ERR_NULL;
  if (x.coef.mode != TS_COEF_DENSE && x.coef.mode != TS_COEF_PATHS) return TS_ERR_MODE;
  if (x.coef.mode == TS_COEF_DENSE && x.coef.c == nullptr) return TS_ERR_NULL;
  if (x.coef.mode == TS_COEF_PATHS && (x.coef.alpha == nullptr || x.coef.tau_s == nullptr))
    return TS_ERR_NULL;
  return TS_OK;
}

int run_instance(const ts_instance& x, void* ws, size_t bytes, cudaStream_t s) {
  if (x.op == TS_OP_SINR_MMSE)
    return ts_sinr_mmse(&x.d, &x.coef, x.G, x.C, x.Pt, x.sigma2, x.sinr, x.flags, ws, bytes, s);
  return ts_sinr_svd_prec(&x.d, &x.coef, x.G, x.C, x.sigma2, x.precision, x.sinr, x.flags, ws, bytes,
                          s);
}

// Launch-shape candidates of an instance's shape class.
std::vector<ts::Tuning> candidates(const ts_instance& x) {
  std::vector<ts::Tuning> c;
  if (x.op != TS_OP_SINR_SVD) return c;
  const bool two_link = x.precision == TS_PREC_FP32 && x.d.m > 2 && x.d.J > 1;
  for (int sp = 0; sp < 2; ++sp) {
    if (two_link) {
      c.push_back({1, sp});
      c.push_back({2, sp});
    } else {
      c.push_back({0, sp});
    }
  }
  return c;
}

int autotune(const ts_instance& x, void* ws, size_t bytes) {
  const std::string key = class_key(x);
  {
    std::lock_guard<std::mutex> lk(g_table_mutex);
    if (g_table.count(key)) return TS_OK;
  }
  const std::vector<ts::Tuning> cand = candidates(x);
  if (cand.empty()) return TS_OK;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int st = e == cudaSuccess ? TS_OK : ts::record_cuda_error(e);
  ts::Tuning best = cand[0];
  float best_ms = 1e30f;
  for (size_t c = 0; c < cand.size() && st == TS_OK; ++c) {
    ts::set_tuning(cand[c]);
    st = run_instance(x, ws, bytes, s);                   // warm-up
    if (st == TS_OK) e = cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == TS_OK && e == cudaSuccess; ++r) st = run_instance(x, ws, bytes, s);
    if (st == TS_OK && e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (st == TS_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (st == TS_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (st == TS_OK && e != cudaSuccess) st = ts::record_cuda_error(e);
    if (st == TS_OK && ms < best_ms) {
      best_ms = ms;
      best = cand[c];
    }
  }
  ts::set_tuning({0, 0});
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (st == TS_OK) {
    std::lock_guard<std::mutex> lk(g_table_mutex);
    g_table[key] = best;
  }
  return st;
}

ts::Tuning tuning_of(const ts_instance& x) {
  std::lock_guard<std::mutex> lk(g_table_mutex);
  auto it = g_table.find(class_key(x));
  return it == g_table.end() ? ts::Tuning{0, 0} : it->second;
}

}  // namespace

extern "C" {

size_t ts_batch_workspace_bytes(const ts_instance* inst, int n) {
  if (inst == nullptr || n < 1) return 0;
  for (int j = 0; j < n; ++j)
    if (check_instance(inst[j]) != TS_OK) return 0;
  size_t slot[kBranches], slot_bytes[kBranches];
  return slot_layout(inst, n, slot, slot_bytes);
}

int ts_batch_plan_create(const ts_instance* inst, int n, void* ws, size_t ws_bytes, int options,
                         ts_batch_plan** plan) {
  if (plan == nullptr || inst == nullptr || ws == nullptr) return TS_ERR_NULL;
  *plan = nullptr;
  if (n < 1) return TS_ERR_DIMS;
  for (int j = 0; j < n; ++j) {
    const int st = check_instance(inst[j]);
    if (st != TS_OK) return st;
  }
  size_t slot[kBranches], slot_bytes[kBranches];
  const size_t o = slot_layout(inst, n, slot, slot_bytes);
  std::vector<size_t> off(n), bytes(n);
  for (int j = 0; j < n; ++j) {
    off[j] = slot[j % kBranches];
    bytes[j] = slot_bytes[j % kBranches];
  }
  if (ws_bytes < o) return TS_ERR_WORKSPACE;
  if (((uintptr_t)ws & 255u) != 0) return TS_ERR_ALIGN;
  char* base = static_cast<char*>(ws);

  if (options & TS_BATCH_AUTOTUNE)
    for (int j = 0; j < n; ++j) {
      const int st = autotune(inst[j], base + off[j], bytes[j]);
      if (st != TS_OK) return st;
    }

  ts_batch_plan* p = new ts_batch_plan;
  p->inst.assign(inst, inst + n);
  cudaStream_t origin = nullptr, br[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
  for (int b = 0; b < kBranches && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&br[b], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int b = 0; b < kBranches && e == cudaSuccess; ++b) e = cudaEventCreateWithFlags(&join[b], cudaEventDisableTiming);
  int st = e == cudaSuccess ? TS_OK : ts::record_cuda_error(e);
  bool capturing = false;
  if (st == TS_OK) {
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeRelaxed);
    capturing = e == cudaSuccess;
    if (e == cudaSuccess) e = cudaEventRecord(fork, origin);
    for (int b = 0; b < kBranches && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(br[b], fork, 0);
    if (e != cudaSuccess) st = ts::record_cuda_error(e);
  }
  ts::suspend_timing(true);
  for (int j = 0; j < n && st == TS_OK; ++j) {
    ts::set_tuning(tuning_of(inst[j]));
    st = run_instance(inst[j], base + off[j], bytes[j], br[j % kBranches]);
  }
  ts::set_tuning({0, 0});
  ts::suspend_timing(false);
  if (capturing) {
    // join every branch (also after an error, so that the capture ends)
    for (int b = 0; b < kBranches; ++b) {
      if (cudaEventRecord(join[b], br[b]) == cudaSuccess) cudaStreamWaitEvent(origin, join[b], 0);
    }
    e = cudaStreamEndCapture(origin, &p->graph);
    if (st == TS_OK && e != cudaSuccess) st = ts::record_cuda_error(e);
  }
  if (st == TS_OK) {
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) st = ts::record_cuda_error(e);
  }
  for (int b = 0; b < kBranches; ++b) {
    if (join[b]) cudaEventDestroy(join[b]);
    if (br[b]) cudaStreamDestroy(br[b]);
  }
  if (fork) cudaEventDestroy(fork);
  if (origin) cudaStreamDestroy(origin);
  if (st != TS_OK) {
    ts_batch_plan_destroy(p);
    return st;
  }
  *plan = p;
  return TS_OK;
}

int ts_batch_launch(ts_batch_plan* plan, void* stream) {
  if (plan == nullptr || plan->exec == nullptr) return TS_ERR_NULL;
  const cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TS_OK : ts::record_cuda_error(e);
}

void ts_batch_plan_destroy(ts_batch_plan* plan) {
  if (plan == nullptr) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
}

int ts_autotune_save(const char* path) {
  if (path == nullptr) return TS_ERR_NULL;
  FILE* f = fopen(path, "w");
  if (f == nullptr) return TS_ERR_MODE;
  std::lock_guard<std::mutex> lk(g_table_mutex);
  for (const auto& kv : g_table)
    fprintf(f, "%s %d %d\n", kv.first.c_str(), kv.second.link_variant, kv.second.precoder_split);
  fclose(f);
  return TS_OK;
}

int ts_autotune_load(const char* path) {
  if (path == nullptr) return TS_ERR_NULL;
  FILE* f = fopen(path, "r");
  if (f == nullptr) return TS_ERR_MODE;
  char key[160];
  int lv = 0, sp = 0;
  std::lock_guard<std::mutex> lk(g_table_mutex);
  while (fscanf(f, "%159s %d %d", key, &lv, &sp) == 3) {
    if (lv < 0 || lv > 2 || sp < 0 || sp > 1) continue;
    g_table[key] = ts::Tuning{lv, sp};
  }
  fclose(f);
  return TS_OK;
}

}  // extern "C"
