// Allocation-free MMSE SINR entry point.
//
// Some callers cannot allocate device memory at the moment they evaluate SINR:
// a per-slot scheduler loop with a fixed latency budget (cudaMalloc and
// cudaFree may synchronise the device and take milliseconds), or a plug-in
// running inside a host framework that owns and pre-reserves all device
// memory.  ts_sinr_mmse_noalloc serves them: its scratch is a fixed array in
// the library's own device memory, so the caller passes only inputs and
// outputs.
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tuckersinr.h"

namespace {

// The scratch array.  Every GPU that loads the library holds it until the
// process exits (it is committed when the library's module is loaded on the
// device, at the first call there).  Host code must not use the name as a
// device address: the address comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_scratch[TS_NOALLOC_SCRATCH_BYTES];

// Device address of g_scratch on the current device, looked up on every
// call with the call's device current.  Once the library's module is loaded
// on a device the lookup is a host-side table read; looking up again rather
// than caching keeps the address right after the device's context was reset
// and recreated (cudaDeviceReset), when the module and its array move.
// Returns a cudaError_t.
cudaError_t scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" int ts_sinr_mmse_noalloc(const ts_dims* d, const ts_coef* coef, const ts_c64* G,
                                    const ts_c64* C, const ts_c64* Pt, const float* sigma2,
                                    float* sinr, uint8_t* flags, void* stream) {
  if (d == nullptr) return TS_ERR_NULL;
  const size_t need = ts_workspace_bytes(d, TS_OP_SINR_MMSE);
  if (need == 0) return TS_ERR_DIMS;
  if (need > TS_NOALLOC_SCRATCH_BYTES) return TS_ERR_WORKSPACE;
  void* ws = nullptr;
  const cudaError_t e = scratch_address(&ws);
  if (e != cudaSuccess) return ts::record_cuda_error(e);   // kept for ts_last_cuda_error()
  // every byte of scratch the MMSE path reads is written earlier in the same
  // call, so the previous call's contents need no clearing
  return ts_sinr_mmse(d, coef, G, C, Pt, sigma2, sinr, flags, ws, TS_NOALLOC_SCRATCH_BYTES, stream);
}
