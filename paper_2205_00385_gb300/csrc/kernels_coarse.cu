// Persistent coarse-grid cycle (Algorithm 2 below level 1).
//
// Below the first coarse level every step of the V-cycle is small (tens of
// thousands of nodes at most) and the standalone launches are bound by launch
// latency and grid ramp-up rather than by memory.  This kernel runs all of
// them in one co-resident grid, phase after phase, separated by a grid-wide
// barrier:
//
//   for l = 2 .. L-1:  b_l = Pm^T r_{l-1}, z_l = omega D_l^-1 b_l (l < L-1)
//                      r_l = b_l - K_l z_l                          (l < L-1)
//   z2_{L-1} = K_{L-1}^-1 b_{L-1}       (stored inverse of the coarsest grid)
//   for l = L-2 .. 2:  z_l += Pm z2_{l+1}
//                      z2_l = z_l + omega D_l^-1 (b_l - K_l z_l)
//   z_1 += Pm z2_2
//
// Each phase calls the same per-item bodies as the standalone kernels, in
// the same order, so the two paths give identical values.
//
// The grid barrier is one 32-bit word: block 0 adds 2^31 - (nblocks - 1),
// every other block adds 1, so one full round adds exactly 2^31 and the top
// bit flips when the last block arrives (no reset between rounds).  The wait
// is bounded: after SPIN_LIMIT polls the block raises the abort word and
// records TO_E_TIMEOUT in the status word; every waiting block sees the abort
// word and returns, so the kernel always ends.  The host clears both words
// when it reports the error.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.h"
#include "mgdev.cuh"

namespace topo {

namespace {

constexpr int CC_THREADS = 256;
constexpr int CC_WARPS = CC_THREADS / 32;
constexpr unsigned SPIN_LIMIT = 1u << 21;   // polls of about 0.1-1 us each

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// false when the cycle was aborted (this block's or another block's wait
// expired); the caller then returns
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned* abort_w, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    __threadfence();
    const unsigned old = atomicAdd(bar, add);
    int ok = 1;
    unsigned spins = 0;
    while (((ld_acquire(bar) ^ old) & 0x80000000u) == 0u) {
      if (ld_acquire(abort_w)) {
        ok = 0;
        break;
      }
      if (++spins > SPIN_LIMIT) {
        atomicExch(abort_w, 1u);
        atomicCAS(status, 0, (int)TO_E_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ void node_ijk(const GridP& g, int n, int& i, int& j, int& k) {
  i = n % g.nnx;
  const int q = n / g.nnx;
  j = q % g.nny;
  k = q / g.nny;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(CC_THREADS, 4) k_coarse_cycle(CoarseCycleP P) {
  constexpr int NT = tri_len(Geo<DIM>::ND);
  __shared__ __align__(16) T sk[CC_WARPS][NT];
  if (ld_acquire(P.abort_w)) return;   // an earlier cycle failed; nothing is trusted
  const int L = P.L;
  const T omega = T(P.omega);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int tid = blockIdx.x * CC_THREADS + threadIdx.x, nthr = gridDim.x * CC_THREADS;
  const int gwarp = tid >> 5, nwarps = nthr >> 5;
  auto V = [](void* p) { return static_cast<T*>(p); };
  auto C = [](const void* p) { return static_cast<const T*>(p); };
  // stored-level operator: element rows of K_l z_l, then the node epilogue
  auto gemv = [&](int l) {
    const GridP& g = P.lv[l].g;
    for (int e = gwarp; e < (int)g.nel; e += nwarps)
      gemv_elem<DIM, T>(g, P.lv[l].mask, C(P.lv[l].Kc), C(P.lv[l].z), V(P.lv[l].eo), e, lane,
                        sk[wib]);
  };
  // ---- downward: restrict, pre-smooth from zero, residual ----
  for (int l = 2; l < L; ++l) {
    const GridP& gc = P.lv[l].g;
    const bool smooth = l < L - 1;
    for (int n = tid; n < (int)gc.nn; n += nthr) {
      int I, J, K;
      node_ijk(gc, n, I, J, K);
      restrict_at<DIM, T>(P.lv[l - 1].g, P.lv[l - 1].mask, gc, P.lv[l].mask, C(P.lv[l - 1].r),
                          V(P.lv[l].b), smooth ? C(P.lv[l].dinv) : nullptr, omega,
                          smooth ? V(P.lv[l].z) : nullptr, I, J, K);
    }
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
    if (!smooth) break;
    gemv(l);
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
    for (int n = tid; n < (int)gc.nn; n += nthr) {
      int i, j, k;
      node_ijk(gc, n, i, j, k);
      gather_at<DIM, T, EPI_RESID>(gc, P.lv[l].mask, C(P.lv[l].eo), C(P.lv[l].z), V(P.lv[l].r),
                                   C(P.lv[l].b), nullptr, omega, T(1), i, j, k);
    }
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
  }
  // ---- coarsest grid: exact solve with the stored inverse ----
  for (int row = gwarp; row < P.nc; row += nwarps)
    dense_row<T>(P.nc, C(P.Ainv), C(P.lv[L - 1].b), V(P.lv[L - 1].z2), row, lane);
  if (!grid_sync(P.bar, P.abort_w, P.status)) return;
  // ---- upward: interpolate, post-smooth ----
  for (int l = L - 2; l >= 1; --l) {
    const GridP& g = P.lv[l].g;
    for (int n = tid; n < (int)g.nn; n += nthr) {
      int i, j, k;
      node_ijk(g, n, i, j, k);
      prolong_at<DIM, T>(g, P.lv[l].mask, P.lv[l + 1].g, C(P.lv[l + 1].z2), V(P.lv[l].z), i, j, k);
    }
    if (l == 1) break;   // level 1 is smoothed by the caller
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
    gemv(l);
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
    for (int n = tid; n < (int)g.nn; n += nthr) {
      int i, j, k;
      node_ijk(g, n, i, j, k);
      gather_at<DIM, T, EPI_SMOOTH>(g, P.lv[l].mask, C(P.lv[l].eo), C(P.lv[l].z), V(P.lv[l].z2),
                                    C(P.lv[l].b), C(P.lv[l].dinv), omega, T(1), i, j, k);
    }
    if (!grid_sync(P.bar, P.abort_w, P.status)) return;
  }
}

template <int DIM, typename T>
int cc_blocks() {
  static int nb = 0;
  if (nb == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coarse_cycle<DIM, T>, CC_THREADS,
                                                      0) != cudaSuccess)
      return 0;
    nb = sms * (per_sm < 4 ? per_sm : 4);
  }
  return nb;
}

template <int DIM, typename T>
cudaError_t coarse_cycle_t(const CoarseCycleP& P, cudaStream_t s) {
  const int nb = cc_blocks<DIM, T>();
  if (nb <= 0) return cudaErrorCooperativeLaunchTooLarge;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nb);
  cfg.blockDim = dim3(CC_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_coarse_cycle<DIM, T>, P);
}

}  // namespace

bool coarse_cycle_ok(int dim, const CoarseCycleP& P) {
  if (P.L < 3 || P.L > MAXL || (dim != 2 && dim != 3)) return false;
  // node and element indices of levels 1 .. L-1 are 32-bit in the kernel
  for (int l = 1; l < P.L; ++l)
    if (P.lv[l].g.nn >= (1ll << 30) || P.lv[l].g.nel >= (1ll << 30)) return false;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return false;
  return coop != 0;
}

cudaError_t launch_coarse_cycle(int dim, int t, const CoarseCycleP& P, cudaStream_t s) {
  if (dim == 2) return t == T_F64 ? coarse_cycle_t<2, double>(P, s) : coarse_cycle_t<2, float>(P, s);
  return t == T_F64 ? coarse_cycle_t<3, double>(P, s) : coarse_cycle_t<3, float>(P, s);
}

}  // namespace topo
