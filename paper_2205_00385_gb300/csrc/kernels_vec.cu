// Float64-accurate long-vector kernels: the CG recursion of the mixed path,
// the PARM/CARM Gram matrices and combinations, and Gram-Schmidt.
//
// A vector is stored either as float64 (the FP64 path: float64 arithmetic)
// or as double-float pairs float2 {hi, lo} (the mixed path: every operation
// in double-float on the FP32 pipe, ~2^-48 relative).  GB300 executes one
// float64 FMA per clock per SM against 128 float32 FMAs, so the mixed path
// keeps its float64-accurate vectors in the pair format: loads and stores
// need no conversion and the FP64 pipe is left idle.  Reductions use a
// fixed grid and fixed summation orders, so results do not depend on
// scheduling.
#include <mutex>
#include <type_traits>

#include "dfmath.cuh"
#include "kernels.h"

namespace topo {

// Arithmetic of a storage type: T is the register type.
template <typename S>
struct Ar;
template <>
struct Ar<double> {
  using T = double;
  __device__ static T ld(const double* p, long long i) { return p[i]; }
  __device__ static void st(double* p, long long i, T v) { p[i] = v; }
  __device__ static T zero() { return 0.0; }
  __device__ static T from_d(double x) { return x; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static T fma3(T a, T b, T c) { return fma(a, b, c); }
  __device__ static T mulf(T a, float b) { return a * (double)b; }
  __device__ static double to_d(T a) { return a; }
  __device__ static T shfl_down(T a, int o) { return __shfl_down_sync(0xffffffffu, a, o); }
  // dot-product accumulation (acc += a b) and its final normalisation
  __device__ static void dacc(T& acc, T a, T b) { acc = fma(a, b, acc); }
  __device__ static T dfin(T a) { return a; }
};
template <>
struct Ar<float2> {
  using T = dfl;
  __device__ static T ld(const float2* p, long long i) {
    const float2 v = p[i];
    return {v.x, v.y};
  }
  __device__ static void st(float2* p, long long i, T v) { p[i] = make_float2(v.h, v.l); }
  __device__ static T zero() { return {0.f, 0.f}; }
  __device__ static T from_d(double x) { return split_d(x); }
  __device__ static T add(T a, T b) { return df_add(a, b); }
  __device__ static T fma3(T a, T b, T c) { return df_fma(a, b, c); }
  // a * b for a float b (b exact): TwoProduct on hi plus the lo term
  __device__ static T mulf(T a, float b) {
    const float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    const float h = p + e;
    return {h, e - (h - p)};
  }
  __device__ static double to_d(T a) { return df_to_d(a); }
  __device__ static T shfl_down(T a, int o) {
    return {__shfl_down_sync(0xffffffffu, a.h, o), __shfl_down_sync(0xffffffffu, a.l, o)};
  }
  __device__ static void dacc(T& acc, T a, T b) { df_dot_acc(acc, a, b); }
  __device__ static T dfin(T a) { return df_norm(a); }
};

// store a register value into a (possibly different) storage type
__device__ __forceinline__ void st_any(double* p, long long i, double v) { p[i] = v; }
__device__ __forceinline__ void st_any(double* p, long long i, dfl v) { p[i] = df_to_d(v); }
__device__ __forceinline__ void st_any(float2* p, long long i, dfl v) { p[i] = make_float2(v.h, v.l); }

// Block sum of NV per-thread values: warps reduce in the storage's
// arithmetic, lane 0 widens once, warp 0 adds the warp results in float64
// in warp order.  Valid in thread 0.
template <typename S, int NV>
__device__ __forceinline__ void block_sum_v(typename Ar<S>::T (&v)[NV], double (&out)[NV],
                                            double* sh /* >= NV*32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    typename Ar<S>::T x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = Ar<S>::add(x, Ar<S>::shfl_down(x, o));
    if (lane == 0) sh[q * 32 + warp] = Ar<S>::to_d(x);
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      out[q] = s;
    }
  }
  __syncthreads();
}

// single-value reduction finished by the last block: *out = sum
template <typename S>
__device__ __forceinline__ void reduce_to(typename Ar<S>::T v, double* out, double* partials,
                                          unsigned* counter, double* sh) {
  typename Ar<S>::T vv[1] = {v};
  double o1[1];
  block_sum_v<S, 1>(vv, o1, sh);
  if (publish_partials<1>(o1, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *out = o[0];
  }
}

#define GRID_LOOP(k, n)                                                 \
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; \
       k < (n); k += (long long)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// Basic vector operations
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(RED_THREADS)
    k_vdot(long long n, const S* __restrict__ a, const S* __restrict__ b, double* partials,
           unsigned* counter, double* out) {
  using A = Ar<S>;
  __shared__ double sh[32];
  typename A::T v[2] = {A::zero(), A::zero()};
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + 3 * stride < n; k += 4 * stride) {
    typename A::T av[4], bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      av[u] = A::ld(a, k + u * stride);
      bv[u] = A::ld(b, k + u * stride);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) A::dacc(v[u & 1], av[u], bv[u]);
  }
  for (; k < n; k += stride) A::dacc(v[0], A::ld(a, k), A::ld(b, k));
  reduce_to<S>(A::add(A::dfin(v[0]), A::dfin(v[1])), out, partials, counter, sh);
}

__global__ void __launch_bounds__(256) k_split(long long n, const double* __restrict__ in,
                                               float2* __restrict__ out) {
  GRID_LOOP(k, n) {
    const dfl v = split_d(in[k]);
    out[k] = make_float2(v.h, v.l);
  }
}

__global__ void __launch_bounds__(256) k_join(long long n, const float2* __restrict__ in,
                                              double* __restrict__ out) {
  GRID_LOOP(k, n) {
    const float2 v = in[k];
    out[k] = df_to_d({v.x, v.y});
  }
}

template <typename S>
__global__ void __launch_bounds__(256) k_vcopy(long long n, const S* __restrict__ a,
                                               S* __restrict__ b) {
  GRID_LOOP(k, n) b[k] = a[k];
}

// a *= 1/sqrt(*s2) (0 when *s2 <= 0); the scale is formed once per block
template <typename S>
__global__ void __launch_bounds__(256) k_vscale_inv_sqrt(long long n, S* __restrict__ a,
                                                         const double* __restrict__ s2) {
  using A = Ar<S>;
  __shared__ double s_sc;
  if (threadIdx.x == 0) s_sc = (*s2 > 0.0) ? 1.0 / sqrt(*s2) : 0.0;
  __syncthreads();
  const typename A::T sc = A::from_d(s_sc);
  GRID_LOOP(k, n) A::st(a, k, A::fma3(A::ld(a, k), sc, A::zero()));
}

// ---------------------------------------------------------------------------
// Gram matrix G[i + ldg*j] = sum_k A[k + i*n] B[k + j*n] (i < na, j < nb,
// both <= MAXB) in one pass over the data: a block stages a chunk of MD_CH
// indices of every column in shared memory, then its threads accumulate
// 2 x 2 tiles of G over interleaved index subsets.  Per-block partials are
// summed by the last block in block order.
// ---------------------------------------------------------------------------
constexpr int MD_CH = 128;   // indices per chunk = threads per block

__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}

template <typename S>
__global__ void __launch_bounds__(MD_CH)
    k_gram(long long n, const S* __restrict__ A, int na, const int* na_dev,
           const S* __restrict__ B, int nb, const int* nb_dev, double* G, int ldg,
           double* partials, unsigned* counter, bool sym) {
  using Rg = Ar<S>;
  using V = typename Rg::T;
  static_assert(sizeof(V) == sizeof(S), "staged values keep the storage layout");
  extern __shared__ unsigned char md_smem[];
  V* sv = reinterpret_cast<V*>(md_smem);   // [2][nv][MD_CH]
  __shared__ bool s_last;
  const int ma = na_dev ? min(max(*na_dev, 0), na) : na;
  const int mb = nb_dev ? min(max(*nb_dev, 0), nb) : nb;
  const int nv = ma + mb;
  const int tr = (ma + 1) / 2, tc = (mb + 1) / 2;
  // sym (a symmetric product, ma == mb): only the 2 x 2 tiles on or above
  // the diagonal, numbered column by column (tile = tj (tj+1)/2 + ti)
  const int ntt = sym ? tr * (tr + 1) / 2 : tr * tc;
  const int ntile = ntt > 0 ? ntt : 1;
  const int S_ = MD_CH / ntile;   // index subsets per tile (>= 2)
  const int t = threadIdx.x;
  const int tile = t % ntile, sub = t / ntile;
  const bool active = ntt > 0 && sub < S_;
  int ti = tile % (tr > 0 ? tr : 1), tj = tile / (tr > 0 ? tr : 1);
  if (sym) {
    tj = 0;
    while ((tj + 1) * (tj + 2) / 2 <= tile) ++tj;
    ti = tile - tj * (tj + 1) / 2;
  }
  const int i0 = active ? 2 * ti : 0, j0 = active ? 2 * tj : 0;
  V acc[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) acc[p][q] = Rg::zero();
  const long long cstride = (long long)gridDim.x * MD_CH;
  // chunk k0 -> stage buffer st: thread t copies index k0 + t of every column
  auto issue = [&](long long k0, int st) {
    const long long k = k0 + t;
    const bool ok = k < n;
    for (int v = 0; v < nv; ++v) {
      const S* col = v < ma ? A + (size_t)v * n : B + (size_t)(v - ma) * n;
      cp_async8(sv + ((size_t)st * nv + v) * MD_CH + t, ok ? col + k : col, ok);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  long long k0 = (long long)blockIdx.x * MD_CH;
  int st = 0;
  if (k0 < n) issue(k0, 0);
  for (; k0 < n; k0 += cstride) {
    if (k0 + cstride < n) {
      issue(k0 + cstride, st ^ 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    if (active) {
      const V* base = sv + (size_t)st * nv * MD_CH;
      const V* a0 = base + i0 * MD_CH;
      const V* a1 = base + (i0 + 1 < ma ? i0 + 1 : i0) * MD_CH;
      const V* b0 = base + (ma + j0) * MD_CH;
      const V* b1 = base + (ma + (j0 + 1 < mb ? j0 + 1 : j0)) * MD_CH;
      for (int idx = sub; idx < MD_CH; idx += S_) {
        const V x0 = a0[idx], x1 = a1[idx], y0 = b0[idx], y1 = b1[idx];
        Rg::dacc(acc[0][0], x0, y0);
        Rg::dacc(acc[1][0], x1, y0);
        Rg::dacc(acc[0][1], x0, y1);
        Rg::dacc(acc[1][1], x1, y1);
      }
      // renormalise the double-float accumulators once per chunk, so that
      // their error terms never grow over more than one chunk's products
#pragma unroll
      for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) acc[p][q] = Rg::dfin(acc[p][q]);
    }
    __syncthreads();
    st ^= 1;
  }
  double* red = reinterpret_cast<double*>(md_smem);   // ntile * 4 * S_ <= 4 * MD_CH doubles
  if (active) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q)
        red[(tile * 4 + p + 2 * q) * S_ + sub] = Rg::to_d(Rg::dfin(acc[p][q]));
  }
  __syncthreads();
  const int np = ma * mb;
  double* part = partials + (size_t)blockIdx.x * (MAXB * MAXB);
  for (int e = t; e < np; e += MD_CH) {
    const int i = e % ma, j = e / ma;
    if (sym && i > j) continue;
    const int tl = sym ? (j / 2) * (j / 2 + 1) / 2 + i / 2 : (i / 2) + tr * (j / 2);
    const int qq = (i & 1) + 2 * (j & 1);
    double sum = 0.0;
    for (int u = 0; u < S_; ++u) sum += red[(tl * 4 + qq) * S_ + u];
    part[e] = sum;
  }
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int e = t; e < np; e += MD_CH) {
    const int i = e % ma, j = e / ma;
    if (sym && i > j) continue;
    double sum = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) sum += partials[(size_t)bl * (MAXB * MAXB) + e];
    G[i + (size_t)ldg * j] = sum;
    if (sym) G[j + (size_t)ldg * i] = sum;
  }
  if (t == 0) *counter = 0u;
}

// Column case: g[i] = sum_k A[k + i*n] b[k].  Warp w of a block
// accumulates column w % na over its own share of the indices, wpc = blockDim
// / (32 na) warps per column (more warps for few columns, so that a launch
// with one or two columns still keeps enough loads outstanding); one
// accumulator set per lane, four indices in flight.  Lanes, the warps of a
// column, and blocks are summed in a fixed order.
template <typename S>
__global__ void __launch_bounds__(32 * MAXB)
    k_gram_col(long long n, const S* __restrict__ A, int na, const int* na_dev,
               const S* __restrict__ b, double* g, double* partials, unsigned* counter) {
  using Rg = Ar<S>;
  using V = typename Rg::T;
  __shared__ double sh[32 * MAXB / 32];
  __shared__ bool s_last;
  const int ma = na_dev ? min(max(*na_dev, 0), na) : na;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int wpc = nw / na, ci = wi % na, sub = wi / na;
  V acc = Rg::zero(), acc2 = Rg::zero();
  if (ci < ma) {
    const S* col = A + (size_t)ci * n;
    const long long stride = (long long)gridDim.x * wpc * 32;
    long long k = ((long long)blockIdx.x * wpc + sub) * 32 + lane;
    V acc3 = Rg::zero(), acc4 = Rg::zero();
    for (; k + 3 * stride < n; k += 4 * stride) {
      const V a0 = Rg::ld(col, k), b0 = Rg::ld(b, k);
      const V a1 = Rg::ld(col, k + stride), b1 = Rg::ld(b, k + stride);
      const V a2 = Rg::ld(col, k + 2 * stride), b2 = Rg::ld(b, k + 2 * stride);
      const V a3 = Rg::ld(col, k + 3 * stride), b3 = Rg::ld(b, k + 3 * stride);
      Rg::dacc(acc, a0, b0);
      Rg::dacc(acc2, a1, b1);
      Rg::dacc(acc3, a2, b2);
      Rg::dacc(acc4, a3, b3);
    }
    for (; k < n; k += stride) Rg::dacc(acc, Rg::ld(col, k), Rg::ld(b, k));
    acc = Rg::add(Rg::add(Rg::dfin(acc), Rg::dfin(acc2)), Rg::add(Rg::dfin(acc3), Rg::dfin(acc4)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = Rg::add(acc, Rg::shfl_down(acc, o));
  }
  if (lane == 0) sh[wi] = ci < ma ? Rg::to_d(acc) : 0.0;
  __syncthreads();
  if ((int)threadIdx.x < MAXB) {
    double v = 0.0;
    if ((int)threadIdx.x < na)
      for (int u = 0; u < wpc; ++u) v += sh[u * na + threadIdx.x];
    partials[(size_t)blockIdx.x * MAXB + threadIdx.x] = v;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if ((int)threadIdx.x < ma) {
    double sum = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) sum += partials[(size_t)bl * MAXB + threadIdx.x];
    g[threadIdx.x] = sum;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// y = beta*y + sign*sum_i c[i] A[:, i] (i < m <= MMAX); optional
// |y - w|^2 -> *rr.  A, w (and y when SY = S) in storage S; y may be
// float64 when S is the pair format (one float64 add per stored value).
// The coefficients sit in shared memory; each thread keeps two indices in
// flight so that enough loads are outstanding to cover DRAM latency.
template <typename S, typename SY, int MMAX>
__global__ void __launch_bounds__(RED_THREADS, 4)
    k_combine(long long n, const S* __restrict__ A, int m, const int* m_dev,
              const double* __restrict__ c, double sign, double beta, SY* __restrict__ y,
              const S* __restrict__ w, double* rr, double* partials, unsigned* counter) {
  using Rg = Ar<S>;
  using V = typename Rg::T;
  __shared__ double sh[32];
  __shared__ V scc[MMAX];
  const int mm = m_dev ? min(max(*m_dev, 0), m) : m;
  if (threadIdx.x < MMAX) {
    const double ci = (int)threadIdx.x < mm ? c[threadIdx.x] : 0.0;
    scc[threadIdx.x] = Rg::from_d(sign == 1.0 ? ci : sign == -1.0 ? -ci : sign * ci);
  }
  __syncthreads();
  const V bb = Rg::from_d(beta);
  auto start = [&](long long k) -> V {
    if (beta == 0.0) return Rg::zero();
    V yk;
    if constexpr (std::is_same<SY, S>::value) yk = Rg::ld(y, k);
    else yk = Rg::from_d((double)y[k]);
    return (beta == 1.0) ? yk : Rg::fma3(bb, yk, Rg::zero());
  };
  auto resid = [&](V s, long long k, V& acc) {
    V d = s;
    if (w) d = Rg::add(s, Rg::fma3(Rg::ld(w, k), Rg::from_d(-1.0), Rg::zero()));
    acc = Rg::fma3(d, d, acc);
  };
  V v = Rg::zero();
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + stride < n; k += 2 * stride) {
    const long long k1 = k + stride;
    V s0 = start(k), s1 = start(k1);
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < mm) {
        const V ci = scc[i];
        const S* col = A + (size_t)i * n;
        s0 = Rg::fma3(ci, Rg::ld(col, k), s0);
        s1 = Rg::fma3(ci, Rg::ld(col, k1), s1);
      }
    st_any(y, k, s0);
    st_any(y, k1, s1);
    if (rr) {
      resid(s0, k, v);
      resid(s1, k1, v);
    }
  }
  if (k < n) {
    V s0 = start(k);
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < mm) s0 = Rg::fma3(scc[i], Rg::ld(A + (size_t)i * n, k), s0);
    st_any(y, k, s0);
    if (rr) resid(s0, k, v);
  }
  if (!rr) return;
  reduce_to<S>(v, rr, partials, counter, sh);
}

// One classical Gram-Schmidt pass fused with the next pass's projections:
// y <- y - sum_{i<m} c[i] A[:, i], then h[i] = A[:, i] . y for the new y
// (m = *m_dev when given).  The columns are read once for both; the dots
// are double-float, summed per block and then over blocks in order.
template <typename S, int MMAX>
__global__ void __launch_bounds__(RED_THREADS, 2)
    k_combine_dots(long long n, const S* __restrict__ A, int m, const int* m_dev,
                   const double* __restrict__ c, S* __restrict__ y, double* h,
                   double* partials, unsigned* counter) {
  using Rg = Ar<S>;
  using V = typename Rg::T;
  __shared__ double sh[MMAX * 32];
  __shared__ V scc[MMAX];
  pdl_wait();
  const int mm = m_dev ? min(max(*m_dev, 0), m) : m;
  if (threadIdx.x < MMAX)
    scc[threadIdx.x] = Rg::from_d((int)threadIdx.x < mm ? -c[threadIdx.x] : 0.0);
  __syncthreads();
  V hacc[MMAX];
#pragma unroll
  for (int i = 0; i < MMAX; ++i) hacc[i] = Rg::zero();
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    V a[MMAX];
    V sv = Rg::ld(y, k);
#pragma unroll
    for (int i = 0; i < MMAX; ++i) a[i] = i < mm ? Rg::ld(A + (size_t)i * n, k) : Rg::zero();
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < mm) sv = Rg::fma3(scc[i], a[i], sv);
    Rg::st(y, k, sv);
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < mm) Rg::dacc(hacc[i], a[i], sv);
  }
#pragma unroll
  for (int i = 0; i < MMAX; ++i) hacc[i] = Rg::dfin(hacc[i]);
  double o1[MMAX];
  block_sum_v<S, MMAX>(hacc, o1, sh);
  if (publish_partials<MMAX>(o1, partials, counter)) {
    double o[MMAX];
    finish_sum<MMAX>(partials, counter, o, sh);
    // the block sums are complete in thread 0 only
    if (threadIdx.x == 0)
      for (int q = 0; q < mm; ++q) h[q] = o[q];
  }
  pdl_launch_dependents();
}

// Gram-Schmidt acceptance: if |r_src|^2 after orthogonalisation exceeds
// tol^2 times its value before, R[:, k] = r_src / |r_src| with k the
// current count (the count itself is advanced by k_gs_count afterwards)
template <typename S>
__global__ void __launch_bounds__(256)
    k_gs_accept(long long n, S* R, int src, const double* scal, int n0, int n1, double tol,
                const int* ints) {
  using Rg = Ar<S>;
  __shared__ double s_scale;
  const double before = scal[n0], after = scal[n1];
  const bool keep = after > tol * tol * before && after > 0.0;
  if (!keep) return;
  const int k = ints[I_KCOUNT];
  if (threadIdx.x == 0) s_scale = 1.0 / sqrt(after);   // once per block
  __syncthreads();
  const typename Rg::T sc = Rg::from_d(s_scale);
  const S* a = R + (size_t)src * n;
  S* b = R + (size_t)k * n;
  GRID_LOOP(i, n) Rg::st(b, i, Rg::fma3(Rg::ld(a, i), sc, Rg::zero()));
}

// Records column src of the QR factor of the basis, Rt[:, src] (ld MAXB):
// its projections h1 + h2 on the k columns accepted before it and, when it
// is accepted, its remaining norm at row k; then advances the count.  Also
// stores the column's norm before orthogonalisation in rn[src].
__global__ void k_gs_record(const double* scal, int n0, int n1, double tol, int src,
                            const double* h1, const double* h2, double* Rt, double* rn,
                            int* ints) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double before = scal[n0], after = scal[n1];
  const bool keep = after > tol * tol * before && after > 0.0;
  const int k = ints[I_KCOUNT];
  double* col = Rt + (size_t)MAXB * src;
  for (int j = 0; j < MAXB; ++j) col[j] = j < k ? h1[j] + h2[j] : 0.0;
  if (keep) col[k] = sqrt(after);
  rn[src] = sqrt(fmax(before, 0.0));
  if (keep) ints[I_KCOUNT] = k + 1;
}

// ---------------------------------------------------------------------------
// CG recursion of the mixed path: x, r, p in the pair format; the operator
// works on the float32 shadow p32 -> q32 and the V-cycle returns z32.
// alpha and beta are formed once per block from the float64 scalars.
// ---------------------------------------------------------------------------
// The three passes below keep four indices per thread in flight (their
// loads are issued before any of them is used), enough outstanding bytes to
// stream at the copy bandwidth with one resident grid.
constexpr int CG_U = 4;

// out = sum_k a[k] b[k], a pairs, b float32.  Twelve bytes per index, so
// eight indices per thread are kept in flight.
constexpr int DOT_U = 8;
__global__ void __launch_bounds__(RED_THREADS)
    k_dot_d2f(long long n, const float2* __restrict__ a, const float* __restrict__ b,
              double* partials, unsigned* counter, double* out) {
  using Rg = Ar<float2>;
  __shared__ double sh[32];
  pdl_wait();
  dfl v[2] = {Rg::zero(), Rg::zero()};
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + (DOT_U - 1) * stride < n; k += DOT_U * stride) {
    dfl av[DOT_U];
    float bv[DOT_U];
#pragma unroll
    for (int u = 0; u < DOT_U; ++u) {
      av[u] = Rg::ld(a, k + u * stride);
      bv[u] = b[k + u * stride];
    }
#pragma unroll
    for (int u = 0; u < DOT_U; ++u) df_dot_acc(v[u & 1], av[u], dfl{bv[u], 0.f});
  }
  for (; k < n; k += stride) df_dot_acc(v[0], Rg::ld(a, k), dfl{b[k], 0.f});
  reduce_to<float2>(df_add(df_norm(v[0]), df_norm(v[1])), out, partials, counter, sh);
  pdl_launch_dependents();
}

// alpha = scal[num] / scal[den]; x += alpha p; r -= alpha q; scal[rr] = |r|^2.
// With b non-null it also starts the next V-cycle: b = r rounded to float32
// and zpre = omega dinv b (its pre-smoothing from a zero guess), the values
// the V-cycle's first kernel would compute.
// With host_rr set, |r|^2 is also written there (pinned host memory mapped
// into the device's address space), so the host reads it after an event on
// the stream without a copy between this kernel and the next.
template <bool PRE>
__global__ void __launch_bounds__(RED_THREADS)
    k_cg_xr_d2(long long n, float2* __restrict__ x, float2* __restrict__ r,
               const float2* __restrict__ p, const float* __restrict__ q, double* scal, int num,
               int den, int rr, double* partials, unsigned* counter, float* __restrict__ b,
               float* __restrict__ zpre, const float* __restrict__ dinv, float omega,
               double* host_rr) {
  using Rg = Ar<float2>;
  __shared__ double sh[32];
  __shared__ double s_alpha;
  pdl_wait();
  if (threadIdx.x == 0) s_alpha = scal[num] / scal[den];
  __syncthreads();
  const dfl al = split_d(s_alpha), mal = {-al.h, -al.l};
  dfl v[2] = {Rg::zero(), Rg::zero()};
  auto step = [&](long long kk, dfl xk, dfl pk, dfl rk0, float qk, float dk, dfl& acc) {
    Rg::st(x, kk, df_fma(al, pk, xk));
    const dfl rk = df_add(Rg::mulf(mal, qk), rk0);
    Rg::st(r, kk, rk);
    df_dot_acc(acc, rk, rk);
    if (PRE) {
      const float bv = __fadd_rn(rk.h, rk.l);
      b[kk] = bv;
      zpre[kk] = omega * dk * bv;
    }
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + (CG_U - 1) * stride < n; k += CG_U * stride) {
    dfl xv[CG_U], pv[CG_U], rv[CG_U];
    float qv[CG_U], dv[CG_U];
#pragma unroll
    for (int u = 0; u < CG_U; ++u) {
      const long long kk = k + u * stride;
      xv[u] = Rg::ld(x, kk);
      pv[u] = Rg::ld(p, kk);
      rv[u] = Rg::ld(r, kk);
      qv[u] = q[kk];
      dv[u] = PRE ? dinv[kk] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < CG_U; ++u)
      step(k + u * stride, xv[u], pv[u], rv[u], qv[u], dv[u], v[u & 1]);
  }
  for (; k < n; k += stride)
    step(k, Rg::ld(x, k), Rg::ld(p, k), Rg::ld(r, k), q[k], PRE ? dinv[k] : 0.f, v[0]);
  {
    // reduce_to's sum, with the second destination
    typename Ar<float2>::T vv[1] = {df_add(df_norm(v[0]), df_norm(v[1]))};
    double o1[1];
    block_sum_v<float2, 1>(vv, o1, sh);
    if (publish_partials<1>(o1, partials, counter)) {
      double o[1];
      finish_sum<1>(partials, counter, o, sh);
      if (threadIdx.x == 0) {
        scal[rr] = o[0];
        if (host_rr) {
          *reinterpret_cast<volatile double*>(host_rr) = o[0];
          __threadfence_system();
        }
      }
    }
  }
  pdl_launch_dependents();
}

// p = z + beta p (beta = scal[num]/scal[den], or p = z when num < 0);
// p32 = p rounded to float32
__global__ void __launch_bounds__(256)
    k_cg_p_d2(long long n, float2* __restrict__ p, float* __restrict__ p32,
              const float* __restrict__ z, const double* __restrict__ scal, int num, int den) {
  using Rg = Ar<float2>;
  __shared__ double s_beta;
  pdl_wait();
  if (threadIdx.x == 0) s_beta = num >= 0 ? scal[num] / scal[den] : 0.0;
  __syncthreads();
  const dfl be = split_d(s_beta);
  auto step = [&](long long kk, float zv, dfl pold) {
    const dfl zk = {zv, 0.f};
    const dfl pk = num >= 0 ? df_add(df_mul(be, pold), zk) : zk;
    Rg::st(p, kk, pk);
    p32[kk] = __fadd_rn(pk.h, pk.l);
  };
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + (CG_U - 1) * stride < n; k += CG_U * stride) {
    float zv[CG_U];
    dfl pv[CG_U];
#pragma unroll
    for (int u = 0; u < CG_U; ++u) {
      zv[u] = z[k + u * stride];
      pv[u] = num >= 0 ? Rg::ld(p, k + u * stride) : Rg::zero();
    }
#pragma unroll
    for (int u = 0; u < CG_U; ++u) step(k + u * stride, zv[u], pv[u]);
  }
  for (; k < n; k += stride) step(k, z[k], num >= 0 ? Rg::ld(p, k) : Rg::zero());
  pdl_launch_dependents();
}

#undef GRID_LOOP

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline int vgrid(long long n) {
  long long b = (n + 255) / 256;
  if (b > RED_BLOCKS) b = RED_BLOCKS;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_vdot(long long n, int vt, const void* a, const void* b, double* partials,
                        unsigned* counter, double* out, cudaStream_t s) {
  if (vt == V_DF2)
    k_vdot<float2><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, (const float2*)a, (const float2*)b,
                                                      partials, counter, out);
  else
    k_vdot<double><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, (const double*)a, (const double*)b,
                                                      partials, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_vconvert(long long n, int tin, const void* in, int tout, void* out,
                            cudaStream_t s) {
  if (tin == tout) {
    if (in == out) return cudaSuccess;
    if (tin == V_DF2)
      k_vcopy<float2><<<vgrid(n), 256, 0, s>>>(n, (const float2*)in, (float2*)out);
    else
      k_vcopy<double><<<vgrid(n), 256, 0, s>>>(n, (const double*)in, (double*)out);
  } else if (tin == V_F64) {
    k_split<<<vgrid(n), 256, 0, s>>>(n, (const double*)in, (float2*)out);
  } else {
    k_join<<<vgrid(n), 256, 0, s>>>(n, (const float2*)in, (double*)out);
  }
  return cudaGetLastError();
}

// x[dim node + c] = 0 where DOF c of the node is fixed; one thread per node
template <typename S>
__global__ void __launch_bounds__(256)
    k_zero_fixed(long long nn, int dim, const uint8_t* __restrict__ mask, S* __restrict__ x) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= nn) return;
  const unsigned m = mask[node];
  if (!m) return;
  for (int c = 0; c < dim; ++c)
    if ((m >> c) & 1u) x[dim * node + c] = S{};
}

cudaError_t launch_zero_fixed(long long nn, int dim, const uint8_t* mask, int vt, void* x,
                              cudaStream_t s) {
  if (nn <= 0) return cudaSuccess;
  if (vt == V_DF2)
    k_zero_fixed<float2><<<nblocks(nn, 256), 256, 0, s>>>(nn, dim, mask, (float2*)x);
  else
    k_zero_fixed<double><<<nblocks(nn, 256), 256, 0, s>>>(nn, dim, mask, (double*)x);
  return cudaGetLastError();
}

cudaError_t launch_vscale_inv_sqrt(long long n, int vt, void* a, const double* s2,
                                   cudaStream_t s) {
  if (vt == V_DF2)
    k_vscale_inv_sqrt<float2><<<vgrid(n), 256, 0, s>>>(n, (float2*)a, s2);
  else
    k_vscale_inv_sqrt<double><<<vgrid(n), 256, 0, s>>>(n, (double*)a, s2);
  return cudaGetLastError();
}

template <typename S>
static void gram_t(long long n, const void* A, int na, const int* na_dev, const void* B, int nb,
                   const int* nb_dev, double* G, int ldg, double* partials, unsigned* counter,
                   cudaStream_t s, bool sym = false) {
  // up to 2 stages x 2*MAXB columns x MD_CH values; set once, before any
  // launch of any host thread
  static std::once_flag smem_once;
  std::call_once(smem_once, [] {
    cudaFuncSetAttribute(k_gram<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(2 * 2 * MAXB * MD_CH * sizeof(S)));
  });
  if (nb == 1 && nb_dev == nullptr && !sym) {
    const int wpc = na >= 8 ? 1 : 8 / na;   // warps per column
    k_gram_col<S><<<RED_BLOCKS, 32 * na * wpc, 0, s>>>(n, (const S*)A, na, na_dev,
                                                       (const S*)B, G, partials, counter);
  } else
    k_gram<S><<<RED_BLOCKS, MD_CH, (size_t)2 * (na + nb) * MD_CH * sizeof(S), s>>>(
        n, (const S*)A, na, na_dev, (const S*)B, nb, nb_dev, G, ldg, partials, counter, sym);
}

cudaError_t launch_gram_sym(long long n, int vt, const void* A, const void* B, int m, double* G,
                            int ldg, double* partials, unsigned* counter, cudaStream_t s) {
  if (m > MAXB || m < 1) return cudaErrorInvalidValue;
  if (vt == V_DF2)
    gram_t<float2>(n, A, m, nullptr, B, m, nullptr, G, ldg, partials, counter, s, true);
  else
    gram_t<double>(n, A, m, nullptr, B, m, nullptr, G, ldg, partials, counter, s, true);
  return cudaGetLastError();
}

cudaError_t launch_gram(long long n, int vt, const void* A, int na, const int* na_dev,
                        const void* B, int nb, const int* nb_dev, double* G, int ldg,
                        double* partials, unsigned* counter, cudaStream_t s) {
  if (na > MAXB || nb > MAXB || na < 1 || nb < 1) return cudaErrorInvalidValue;
  if (vt == V_DF2)
    gram_t<float2>(n, A, na, na_dev, B, nb, nb_dev, G, ldg, partials, counter, s);
  else
    gram_t<double>(n, A, na, na_dev, B, nb, nb_dev, G, ldg, partials, counter, s);
  return cudaGetLastError();
}

template <typename S, typename SY>
static void combine_t(long long n, const void* A, int m, const int* m_dev, const double* c,
                      double sign, double beta, void* y, const void* w, double* rr,
                      double* partials, unsigned* counter, cudaStream_t s) {
  const S* a = (const S*)A;
  const S* ww = (const S*)w;
  SY* yy = (SY*)y;
  if (m <= 4)
    k_combine<S, SY, 4><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, m, m_dev, c, sign, beta, yy, ww,
                                                           rr, partials, counter);
  else if (m <= 8)
    k_combine<S, SY, 8><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, m, m_dev, c, sign, beta, yy, ww,
                                                           rr, partials, counter);
  else if (m <= 12)
    k_combine<S, SY, 12><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, m, m_dev, c, sign, beta, yy,
                                                            ww, rr, partials, counter);
  else
    k_combine<S, SY, MAXB><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, m, m_dev, c, sign, beta, yy,
                                                              ww, rr, partials, counter);
}

cudaError_t launch_combine_dots(long long n, int vt, const void* A, int m, const int* m_dev,
                                const double* c, void* y, double* h, double* partials,
                                unsigned* counter, cudaStream_t s) {
  if (m > 12 || m < 0) return cudaErrorInvalidValue;
  if (vt == V_DF2) {
    if (m <= 4)
      return launch_pdl(k_combine_dots<float2, 4>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n,
                        (const float2*)A, m, m_dev, c, (float2*)y, h, partials, counter);
    return launch_pdl(k_combine_dots<float2, 12>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n,
                      (const float2*)A, m, m_dev, c, (float2*)y, h, partials, counter);
  }
  if (m <= 4)
    return launch_pdl(k_combine_dots<double, 4>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n,
                      (const double*)A, m, m_dev, c, (double*)y, h, partials, counter);
  return launch_pdl(k_combine_dots<double, 12>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n,
                    (const double*)A, m, m_dev, c, (double*)y, h, partials, counter);
}

cudaError_t launch_combine(long long n, int vt, const void* A, int m, const int* m_dev,
                           const double* c, double sign, double beta, void* y, int yt,
                           const void* w, double* rr, double* partials, unsigned* counter,
                           cudaStream_t s) {
  if (m > MAXB || m < 0) return cudaErrorInvalidValue;
  if (vt == V_DF2 && yt == V_DF2)
    combine_t<float2, float2>(n, A, m, m_dev, c, sign, beta, y, w, rr, partials, counter, s);
  else if (vt == V_DF2 && yt == V_F64)
    combine_t<float2, double>(n, A, m, m_dev, c, sign, beta, y, w, rr, partials, counter, s);
  else if (vt == V_F64 && yt == V_F64)
    combine_t<double, double>(n, A, m, m_dev, c, sign, beta, y, w, rr, partials, counter, s);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_gs_accept(long long n, int vt, void* R, int src, const double* scal, int n0,
                             int n1, double tol, const double* h1, const double* h2, double* Rt,
                             double* rn, int* ints, cudaStream_t s) {
  if (src < 0 || src >= MAXB) return cudaErrorInvalidValue;
  if (vt == V_DF2)
    k_gs_accept<float2><<<vgrid(n), 256, 0, s>>>(n, (float2*)R, src, scal, n0, n1, tol, ints);
  else
    k_gs_accept<double><<<vgrid(n), 256, 0, s>>>(n, (double*)R, src, scal, n0, n1, tol, ints);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gs_record<<<1, 32, 0, s>>>(scal, n0, n1, tol, src, h1, h2, Rt, rn, ints);
  return cudaGetLastError();
}

// Y[:, j] = sum_{i < kq} U[i + MAXB j] Q[:, i] for j < k: the kept left
// singular directions of the basis expressed in its orthonormal QR factor.
// Each thread loads the kq entries of one index once and forms all k
// outputs; U sits in shared memory.
template <typename S, int KQ>
__global__ void __launch_bounds__(256)
    k_combine_multi(long long n, const S* __restrict__ Q, int kq, const double* __restrict__ U,
                    int k, S* __restrict__ Y) {
  using Rg = Ar<S>;
  using V = typename Rg::T;
  __shared__ V su[KQ * MAXB];
  for (int e = threadIdx.x; e < KQ * MAXB; e += blockDim.x) {
    const int i = e % KQ, j = e / KQ;
    su[e] = Rg::from_d(i < kq && j < k ? U[i + (size_t)MAXB * j] : 0.0);
  }
  __syncthreads();
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    V q[KQ];
#pragma unroll
    for (int i = 0; i < KQ; ++i) q[i] = i < kq ? Rg::ld(Q + (size_t)i * n, idx) : Rg::zero();
    for (int j = 0; j < k; ++j) {
      V acc = Rg::zero();
#pragma unroll
      for (int i = 0; i < KQ; ++i)
        if (i < kq) acc = Rg::fma3(su[i + KQ * j], q[i], acc);
      Rg::st(Y + (size_t)j * n, idx, acc);
    }
  }
}

template <typename S>
static void combine_multi_t(long long n, const void* Q, int kq, const double* U, int k, void* Y,
                            cudaStream_t s) {
  const int g = vgrid(n);
  if (kq <= 4)
    k_combine_multi<S, 4><<<g, 256, 0, s>>>(n, (const S*)Q, kq, U, k, (S*)Y);
  else if (kq <= 8)
    k_combine_multi<S, 8><<<g, 256, 0, s>>>(n, (const S*)Q, kq, U, k, (S*)Y);
  else if (kq <= 12)
    k_combine_multi<S, 12><<<g, 256, 0, s>>>(n, (const S*)Q, kq, U, k, (S*)Y);
  else
    k_combine_multi<S, MAXB><<<g, 256, 0, s>>>(n, (const S*)Q, kq, U, k, (S*)Y);
}

cudaError_t launch_combine_multi(long long n, int vt, const void* Q, int kq, const double* U,
                                 int k, void* Y, cudaStream_t s) {
  if (kq < 1 || kq > MAXB || k < 0 || k > kq || Q == Y) return cudaErrorInvalidValue;
  if (k == 0) return cudaSuccess;
  if (vt == V_DF2)
    combine_multi_t<float2>(n, Q, kq, U, k, Y, s);
  else
    combine_multi_t<double>(n, Q, kq, U, k, Y, s);
  return cudaGetLastError();
}

cudaError_t launch_dot_d2f(long long n, const void* a, const float* b, double* partials,
                           unsigned* counter, double* out, cudaStream_t s) {
  return launch_pdl(k_dot_d2f, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n, (const float2*)a, b,
                    partials, counter, out);
}

cudaError_t launch_cg_xr_d2(long long n, void* x, void* r, const void* p, const float* q,
                            double* scal, int num, int den, int rr, double* partials,
                            unsigned* counter, float* b, float* zpre, const float* dinv,
                            double omega, cudaStream_t s, double* host_rr) {
  if (b)
    return launch_pdl(k_cg_xr_d2<true>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n, (float2*)x,
                      (float2*)r, (const float2*)p, q, scal, num, den, rr, partials, counter, b,
                      zpre, dinv, (float)omega, host_rr);
  return launch_pdl(k_cg_xr_d2<false>, dim3(RED_BLOCKS), dim3(RED_THREADS), 0, s, n, (float2*)x,
                    (float2*)r, (const float2*)p, q, scal, num, den, rr, partials, counter,
                    (float*)nullptr, (float*)nullptr, (const float*)nullptr, 0.f, host_rr);
}

cudaError_t launch_cg_p_d2(long long n, void* p, float* p32, const float* z, const double* scal,
                           int num, int den, cudaStream_t s) {
  return launch_pdl(k_cg_p_d2, dim3(vgrid(n)), dim3(256), 0, s, n, (float2*)p, p32, z, scal, num,
                    den);
}

}  // namespace topo
