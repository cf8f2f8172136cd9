// Optimality-criteria update for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: code that runs inside
// another runtime's memory pool or allocator hook, plugins whose host
// application owns every device allocation, or a step recorded while the
// caller's memory budget is frozen.  to_oc_update needs a context, and a
// context needs a caller-allocated workspace.  to_oc_update_noalloc runs the
// same OC kernels without either: its scratch memory (the per-element
// factors, the bisection bracket and the reduction partials) lives in the
// file-scope device array below, which every GPU that loads libtopo.so holds
// until the process exits.
#include <cuda.h>

#include <mutex>

#include "kernels.h"

namespace {

using namespace topo;

constexpr long long NOALLOC_MAX_NEL = 1LL << 21;              // 2,097,152 elements
constexpr size_t NA_A = 0;                                    // double[NOALLOC_MAX_NEL]
constexpr size_t NA_PARTIALS = NA_A + sizeof(double) * NOALLOC_MAX_NEL;
constexpr size_t NA_SCAL = NA_PARTIALS + sizeof(double) * RED_BLOCKS;
constexpr size_t NA_COUNTERS = NA_SCAL + sizeof(double) * S_NSLOTS;
constexpr size_t NA_BYTES = NA_COUNTERS + 256;                // ~16 MiB in total
// Bisection steps launched per call.  A step is a no-op once the bracket is
// within 1e-13 relative; 192 steps cover multipliers down to ~1e-30.
constexpr int NOALLOC_OC_STEPS = 192;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// The array's device address belongs to a CUDA context: each context that
// loads the library (the primary context of every device, a context the
// host application created and made current, the new primary context after
// a cudaDeviceReset) has its own copy.  In host code the array's name is
// only a host-side stand-in, so the address is resolved with the context
// current, once per context, and cached under the context's unique ID
// (cuCtxGetId; a context's handle may be reused after it is destroyed, its
// ID never is).  The two driver functions are fetched through the runtime,
// so the library needs no link to the driver library.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

constexpr int CACHE_SLOTS = 64;
std::mutex g_mu;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
unsigned long long g_ctx_id[CACHE_SLOTS] = {0};
unsigned char* g_ctx_ptr[CACHE_SLOTS] = {nullptr};
int g_next_slot = 0;

cudaError_t driver_functions() {
  if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
  void* f1 = nullptr;
  void* f2 = nullptr;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                   cudaEnableDefault, &q1);
  if (e != cudaSuccess) return e;
  e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
  if (e != cudaSuccess) return e;
  if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
    return cudaErrorSymbolNotFound;
  g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  return cudaSuccess;
}

// Device address of the scratch array in the calling thread's current
// context (the runtime binds the current device's primary context first if
// none is current).
cudaError_t scratch_for_current_context(unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  cudaError_t e = driver_functions();
  if (e != cudaSuccess) return e;
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  void* p = nullptr;
  if (!ctx) {
    // nothing current yet: resolving the symbol binds the primary context
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  for (int i = 0; i < CACHE_SLOTS; ++i)
    if (g_ctx_ptr[i] && g_ctx_id[i] == id) {
      *out = g_ctx_ptr[i];
      return cudaSuccess;
    }
  if (!p && (e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
  const int slot = g_next_slot;
  g_next_slot = (g_next_slot + 1) % CACHE_SLOTS;
  g_ctx_id[slot] = id;
  g_ctx_ptr[slot] = static_cast<unsigned char*>(p);
  *out = g_ctx_ptr[slot];
  return cudaSuccess;
}

to_status cuda_err(const char* what, cudaError_t e) {
  set_global_error(std::string(what) + ": " + cudaGetErrorString(e));
  return TO_E_CUDA;
}

}  // namespace

extern "C" to_status to_oc_update_noalloc(int64_t nel, double volfrac, double move,
                                          const double* dc_f, const double* dv_f, double* rho,
                                          double* change_dev, void* stream) {
  if (nel < 1) return set_global_error("nel must be positive"), TO_E_INVALID;
  if (nel > NOALLOC_MAX_NEL)
    return set_global_error("nel exceeds the no-alloc scratch capacity of 2097152 elements"),
           TO_E_INVALID;
  if (!dc_f || !dv_f || !rho) return set_global_error("NULL argument"), TO_E_INVALID;
  if (!(volfrac > 0.0 && volfrac <= 1.0) || !(move > 0.0 && move <= 1.0))
    return set_global_error("bad volfrac/move"), TO_E_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  cudaError_t e = scratch_for_current_context(&base);
  if (e != cudaSuccess) return cuda_err("scratch address", e);
  double* a = reinterpret_cast<double*>(base + NA_A);
  double* partials = reinterpret_cast<double*>(base + NA_PARTIALS);
  double* scal = reinterpret_cast<double*>(base + NA_SCAL);
  unsigned* counters = reinterpret_cast<unsigned*>(base + NA_COUNTERS);
  // The array keeps the previous call's contents: the reduction counters
  // must start at zero (the bracket and factors are rewritten below).
  if ((e = cudaMemsetAsync(counters, 0, 256, s)) != cudaSuccess) return cuda_err("clear", e);
  const double target = volfrac * (double)nel;
  if ((e = launch_oc_prep(nel, rho, dc_f, dv_f, a, scal, s)) != cudaSuccess)
    return cuda_err("oc prep", e);
  for (int q = 0; q < NOALLOC_OC_STEPS; ++q)
    if ((e = launch_oc_step(nel, rho, a, dv_f, move, target, scal, partials, counters + 0, s)) !=
        cudaSuccess)
      return cuda_err("oc step", e);
  if ((e = launch_oc_final(nel, rho, a, move, scal, change_dev, partials, counters + 1, s)) !=
      cudaSuccess)
    return cuda_err("oc final", e);
  return TO_OK;
}
