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

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so its device address is
// resolved once per device (with that device current) and cached.
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_dev_ptr[dev];
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
  cudaError_t e = scratch_for_current_device(&base);
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
