// The coarse end of the V-cycle (Algorithm 2) in one launch (option
// TO_OPERATOR_FUSED_COARSE; off by default).
//
// Below a few thousand nodes a level's kernels carry almost no work: at
// 192 x 96 x 96 the levels from 24 x 12 x 12 down to the 6 x 3 x 3
// coarsest grid take eleven launches per V-cycle.  Here one thread-block
// cluster runs that whole stretch -- restriction into level l0, the
// residual and restriction of every level below it, the exact coarsest
// solve, and on the way up each level's interpolation and post-smoothing --
// with a cluster barrier between the steps.  The barrier is the hardware
// one (barrier.cluster, release / acquire at cluster scope): the cluster's
// CTAs are co-scheduled by construction, so nothing spins in software, and
// the vectors the CTAs exchange between steps are read through L2
// (ld.global.cg).  Every step uses the per-item bodies of the
// one-kernel-per-step path (mg_device.cuh) and the same per-row summation
// order in the coarsest product, so the result is bit for bit the same.
// Measured, it is slower than the separate launches (277 against 247 us
// per V-cycle at 192 x 96 x 96): inside a captured graph with programmatic
// dependent launch the separate kernels' launch cost is hidden, and each
// of their steps spreads over the whole GPU, where the cluster's 8-16 SMs
// need one memory round trip or more per step per thread.
#include <mutex>

#include "kernels.h"
#include "mg_device.cuh"

namespace topo {
namespace {

constexpr int VF_THREADS = 384;

__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_nctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}

template <int DIM, typename T, typename TA>
__global__ void __launch_bounds__(VF_THREADS, 1) k_vcycle_coarse(VFuseArgs a) {
  const long long nthr = (long long)cluster_nctarank() * blockDim.x;
  const long long tid = (long long)cluster_ctarank() * blockDim.x + threadIdx.x;
  const T omega = T(a.omega);
  const int L = a.L;
  pdl_wait();

  // restriction into level l (pre-smoothing it from zero unless coarsest)
  auto restrict_into = [&](int l) {
    const VFLevel& f = a.lv[l - 1];
    const VFLevel& c = a.lv[l];
    const bool smooth = l < L - 1;
    const long long plane = (long long)c.g.nnx * c.g.nny;
    for (long long n = tid; n < c.g.nn; n += nthr) {
      const int K = DIM == 3 ? (int)(n / plane) : 0;
      const long long rem = n - (long long)K * plane;
      const int J = (int)(rem / c.g.nnx), I = (int)(rem - (long long)J * c.g.nnx);
      restrict_node<DIM, T, true>(f.g, f.mask, c.g, c.mask, static_cast<const T*>(f.r),
                                  static_cast<T*>(c.b),
                                  smooth ? static_cast<const T*>(c.dinv) : nullptr, omega,
                                  smooth ? static_cast<T*>(c.z) : nullptr, I, J, K);
    }
  };
  // level l's operator on its stored stencil, residual or smoothing epilogue
  auto residual = [&](int l) {
    const VFLevel& v = a.lv[l];
    for (long long r = tid; r < DIM * v.g.nn; r += nthr)
      stencil_row<DIM, T, EPI_RESID, true>(v.g, static_cast<const T*>(v.S),
                                           static_cast<const T*>(v.z), static_cast<T*>(v.r),
                                           static_cast<const T*>(v.b),
                                           static_cast<const T*>(v.dinv), omega, r);
  };
  auto smooth = [&](int l) {
    const VFLevel& v = a.lv[l];
    for (long long r = tid; r < DIM * v.g.nn; r += nthr)
      stencil_row<DIM, T, EPI_SMOOTH, true>(v.g, static_cast<const T*>(v.S),
                                            static_cast<const T*>(v.z), static_cast<T*>(v.z2),
                                            static_cast<const T*>(v.b),
                                            static_cast<const T*>(v.dinv), omega, r);
  };
  // z_l += P z2_{l+1}
  auto prolong = [&](int l) {
    const VFLevel& f = a.lv[l];
    const VFLevel& c = a.lv[l + 1];
    const int nq = DIM == 3 ? (f.g.nnz + 1) / 2 : 1;
    const long long plane = (long long)f.g.nnx * f.g.nny, items = plane * nq;
    for (long long it = tid; it < items; it += nthr) {
      const int q = (int)(it / plane);
      const long long rem = it - (long long)q * plane;
      const int j = (int)(rem / f.g.nnx), i = (int)(rem - (long long)j * f.g.nnx);
      prolong_pair<DIM, T, true>(f.g, f.mask, c.g, static_cast<const T*>(c.z2),
                                 static_cast<T*>(f.z), i, j, q);
    }
  };

  restrict_into(a.l0);
  cluster_sync_all();
  for (int l = a.l0; l < L - 1; ++l) {
    residual(l);
    cluster_sync_all();
    restrict_into(l + 1);
    cluster_sync_all();
  }
  {
    // coarsest grid: z2 = Ainv b, one warp per row, lanes strided over the
    // columns and summed by the same shuffle tree as the one-kernel path
    const VFLevel& v = a.lv[L - 1];
    const TA* A = static_cast<const TA*>(a.Ainv);
    const T* x = static_cast<const T*>(v.b);
    T* y = static_cast<T*>(v.z2);
    const int lane = threadIdx.x & 31;
    const long long nw = nthr >> 5;
    for (long long row = tid >> 5; row < a.nc; row += nw) {
      TA s = TA(0);
      for (int m = lane; m < a.nc; m += 32) s += A[(size_t)row * a.nc + m] * (TA)__ldcg(x + m);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) y[row] = (T)s;
    }
  }
  cluster_sync_all();
  for (int l = L - 2; l >= a.l0; --l) {
    prolong(l);
    cluster_sync_all();
    smooth(l);
    if (l > a.l0) cluster_sync_all();
  }
  pdl_launch_dependents();
}

// largest cluster (16, else 8) of which one can be resident on the device;
// 0 if none.  Queried once per kernel and device.
template <int DIM, typename T, typename TA>
int cluster_for() {
  static int cache[64];
  static bool done[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return cache[dev];
  int best = 0;
  auto kern = k_vcycle_coarse<DIM, T, TA>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
      cudaSuccess)
    (void)cudaGetLastError();
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(VF_THREADS);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n >= 1) {
      best = cs;
      break;
    }
    (void)cudaGetLastError();
  }
  cache[dev] = best;
  done[dev] = true;
  return best;
}

template <int DIM, typename T, typename TA>
cudaError_t launch_t(const VFuseArgs& a, cudaStream_t s) {
  const int cs = cluster_for<DIM, T, TA>();
  if (cs <= 0) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cs);
  cfg.blockDim = dim3(VF_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_vcycle_coarse<DIM, T, TA>, a);
}

}  // namespace

int vcycle_coarse_cluster(int dim, int t, int ta) {
  if (dim == 2) {
    if (t == T_F64) return ta == T_F64 ? cluster_for<2, double, double>() : 0;
    return ta == T_F64 ? cluster_for<2, float, double>() : cluster_for<2, float, float>();
  }
  if (t == T_F64) return ta == T_F64 ? cluster_for<3, double, double>() : 0;
  return ta == T_F64 ? cluster_for<3, float, double>() : cluster_for<3, float, float>();
}

cudaError_t launch_vcycle_coarse(int dim, int t, int ta, const VFuseArgs& a, cudaStream_t s) {
  if (a.l0 < 1 || a.L > VF_MAXL || a.l0 > a.L - 1 || a.nc <= 0) return cudaErrorInvalidValue;
  if (dim == 2) {
    if (t == T_F64) return ta == T_F64 ? launch_t<2, double, double>(a, s) : cudaErrorInvalidValue;
    return ta == T_F64 ? launch_t<2, float, double>(a, s) : launch_t<2, float, float>(a, s);
  }
  if (t == T_F64) return ta == T_F64 ? launch_t<3, double, double>(a, s) : cudaErrorInvalidValue;
  return ta == T_F64 ? launch_t<3, float, double>(a, s) : launch_t<3, float, float>(a, s);
}

}  // namespace topo
