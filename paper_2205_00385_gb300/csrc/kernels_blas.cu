// Float64 vector kernels of the CG recursion, the CARM/PARM multi-vector
// products and Gram-Schmidt, and small dense solves run on one block.
// All reductions use a fixed grid of RED_BLOCKS blocks and a fixed summation
// tree, so results do not depend on timing or on other work on the GPU.
#include <math.h>

#include "dfmath.cuh"
#include "kernels.h"

namespace topo {

__global__ void __launch_bounds__(RED_THREADS)
    k_dot(long long n, const double* __restrict__ a, const double* __restrict__ b,
          double* partials, unsigned* counter, double* out) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    v[0] = fma(a[q], b[q], v[0]);
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *out = o[0];
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_cg_xr(long long n, double* __restrict__ x, double* __restrict__ r,
            const double* __restrict__ p, const double* __restrict__ q, double* scal, int num,
            int den, int rr, double* partials, unsigned* counter) {
  __shared__ double sh[32];
  const double alpha = scal[num] / scal[den];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, q[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
  }
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) scal[rr] = o[0];
  }
}

__global__ void __launch_bounds__(256)
    k_cg_p(long long n, double* __restrict__ p, const double* __restrict__ z,
           const double* __restrict__ scal, int num, int den) {
  const double beta = scal[num] / scal[den];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    p[i] = fma(beta, p[i], z[i]);
}

// Mixed-precision CG kernels: p, x, r stay float64; the operator works on the
// float32 shadows p32 -> q32 and the V-cycle returns z32.  Each float32
// value is widened once per pass here, not inside the operator.
__global__ void __launch_bounds__(RED_THREADS)
    k_dot_df(long long n, const double* __restrict__ a, const float* __restrict__ b,
             double* partials, unsigned* counter, double* out) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    v[0] = fma(a[q], (double)b[q], v[0]);
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *out = o[0];
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_cg_xr_f(long long n, double* __restrict__ x, double* __restrict__ r,
              const double* __restrict__ p, const float* __restrict__ q, double* scal, int num,
              int den, int rr, double* partials, unsigned* counter) {
  __shared__ double sh[32];
  const double alpha = scal[num] / scal[den];
  double v[1] = {0.0};
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    x[i] = fma(alpha, p[i], x[i]);
    const double ri = fma(-alpha, (double)q[i], r[i]);
    r[i] = ri;
    v[0] = fma(ri, ri, v[0]);
  }
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) scal[rr] = o[0];
  }
}

// p = z + beta p (beta = scal[num]/scal[den], or 0 when num < 0); p32 = p
__global__ void __launch_bounds__(256)
    k_cg_p_f(long long n, double* __restrict__ p, float* __restrict__ p32,
             const float* __restrict__ z, const double* __restrict__ scal, int num, int den) {
  const double beta = num >= 0 ? scal[num] / scal[den] : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double pi = num >= 0 ? fma(beta, p[i], (double)z[i]) : (double)z[i];
    p[i] = pi;
    p32[i] = (float)pi;
  }
}

__global__ void __launch_bounds__(256) k_copy(long long n, const double* __restrict__ a,
                                              double* __restrict__ b) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

__global__ void __launch_bounds__(256) k_scale_inv_sqrt(long long n, double* __restrict__ a,
                                                        const double* __restrict__ s2) {
  const double s = (*s2 > 0.0) ? 1.0 / sqrt(*s2) : 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    a[i] *= s;
}

// ---------------------------------------------------------------------------
// Gram matrix G[i + ldg*j] = sum_k A[k + i*n] B[k + j*n] (i < na, j < nb,
// both <= MAXB) in one pass over the data: a block stages a chunk of MD_CH
// indices of every column in shared memory (split into double-float once in
// the DF variant), then its threads accumulate 2 x 2 tiles of G over
// interleaved index subsets.  Per-block partials are summed by the last
// block in block order, so the result does not depend on scheduling.
// DF = false: float64 arithmetic (the FP64 path); true: double-float on the
// FP32 pipe (products and sums accurate to ~2^-48 relative).
// ---------------------------------------------------------------------------
constexpr int MD_CH = 128;   // indices per chunk = threads per block

template <bool DF>
struct MdVal {
  using T = double;
  __device__ static T load(double x) { return x; }
  __device__ static T zero() { return 0.0; }
  __device__ static T fma3(T a, T b, T c) { return fma(a, b, c); }
  __device__ static double to_d(T a) { return a; }
};
template <>
struct MdVal<true> {
  using T = dfl;
  __device__ static T load(double x) { return split_d(x); }
  __device__ static T zero() { return {0.f, 0.f}; }
  __device__ static T fma3(T a, T b, T c) { return df_fma(a, b, c); }
  __device__ static double to_d(T a) { return df_to_d(a); }
};

template <bool DF>
__global__ void __launch_bounds__(MD_CH)
    k_multidot(long long n, const double* __restrict__ A, int na, const int* na_dev,
               const double* __restrict__ B, int nb, const int* nb_dev, double* G, int ldg,
               double* partials, unsigned* counter) {
  using M = MdVal<DF>;
  using V = typename M::T;
  __shared__ V sv[2 * MAXB * MD_CH];
  __shared__ bool s_last;
  const int ma = na_dev ? min(max(*na_dev, 0), na) : na;
  const int mb = nb_dev ? min(max(*nb_dev, 0), nb) : nb;
  const int nv = ma + mb;
  const int tr = (ma + 1) / 2, tc = (mb + 1) / 2;
  const int ntile = tr * tc > 0 ? tr * tc : 1;
  const int S = MD_CH / ntile;   // index subsets per tile (>= 2)
  const int t = threadIdx.x;
  const int tile = t % ntile, sub = t / ntile;
  const bool active = tr * tc > 0 && sub < S;
  const int i0 = active ? 2 * (tile % tr) : 0, j0 = active ? 2 * (tile / tr) : 0;
  V acc[2][2];
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int q = 0; q < 2; ++q) acc[p][q] = M::zero();
  for (long long k0 = (long long)blockIdx.x * MD_CH; k0 < n; k0 += (long long)gridDim.x * MD_CH) {
    const long long k = k0 + t;
    for (int v = 0; v < nv; ++v) {
      const double* col = v < ma ? A + (size_t)v * n : B + (size_t)(v - ma) * n;
      sv[v * MD_CH + t] = M::load(k < n ? col[k] : 0.0);
    }
    __syncthreads();
    if (active) {
      const V* a0 = sv + i0 * MD_CH;
      const V* a1 = sv + (i0 + 1 < ma ? i0 + 1 : i0) * MD_CH;
      const V* b0 = sv + (ma + j0) * MD_CH;
      const V* b1 = sv + (ma + (j0 + 1 < mb ? j0 + 1 : j0)) * MD_CH;
      for (int idx = sub; idx < MD_CH; idx += S) {
        const V x0 = a0[idx], x1 = a1[idx], y0 = b0[idx], y1 = b1[idx];
        acc[0][0] = M::fma3(x0, y0, acc[0][0]);
        acc[1][0] = M::fma3(x1, y0, acc[1][0]);
        acc[0][1] = M::fma3(x0, y1, acc[0][1]);
        acc[1][1] = M::fma3(x1, y1, acc[1][1]);
      }
    }
    __syncthreads();
  }
  // block partials: entry (i, j) = sum over the S subsets of its tile, in order
  double* red = reinterpret_cast<double*>(sv);   // ntile * 4 * S <= 4 * MD_CH doubles
  if (active) {
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
      for (int q = 0; q < 2; ++q) red[(tile * 4 + p + 2 * q) * S + sub] = M::to_d(acc[p][q]);
  }
  __syncthreads();
  const int np = ma * mb;
  double* part = partials + (size_t)blockIdx.x * (MAXB * MAXB);
  for (int e = t; e < np; e += MD_CH) {
    const int i = e % ma, j = e / ma;
    const int tl = (i / 2) + tr * (j / 2), qq = (i & 1) + 2 * (j & 1);
    double sum = 0.0;
    for (int u = 0; u < S; ++u) sum += red[(tl * 4 + qq) * S + u];
    part[e] = sum;
  }
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int e = t; e < np; e += MD_CH) {
    double sum = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) sum += partials[(size_t)bl * (MAXB * MAXB) + e];
    G[(e % ma) + (size_t)ldg * (e / ma)] = sum;
  }
  if (t == 0) *counter = 0u;
}

// Block sum of NV per-thread values in the arithmetic of MdVal<DF>: warps
// reduce in that arithmetic (double-float shuffles on the FP32 pipe for
// DF), lane 0 widens once, and warp 0 adds the warp results in float64 in
// warp order.  The result is valid in thread 0.
template <bool DF, int NV>
__device__ __forceinline__ void block_sum_md(typename MdVal<DF>::T (&v)[NV], double (&out)[NV],
                                             double* sh /* >= NV*32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    typename MdVal<DF>::T x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if constexpr (DF) {
        const dfl y = {__shfl_down_sync(0xffffffffu, x.h, o), __shfl_down_sync(0xffffffffu, x.l, o)};
        x = df_add(x, y);
      } else {
        x += __shfl_down_sync(0xffffffffu, x, o);
      }
    }
    if (lane == 0) sh[q * 32 + warp] = MdVal<DF>::to_d(x);
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

// Column case (nb = 1): g[i] = sum_k A[k + i*n] b[k].  Warp i of a block
// accumulates column i over the block's indices (one accumulator per lane,
// so occupancy stays high and many loads are in flight); lanes and then
// blocks are summed in a fixed order.
constexpr int MC_WARPS = MAXB;

template <bool DF>
__global__ void __launch_bounds__(32 * MC_WARPS)
    k_multidot_col(long long n, const double* __restrict__ A, int na, const int* na_dev,
                   const double* __restrict__ b, double* g, double* partials,
                   unsigned* counter) {
  using M = MdVal<DF>;
  using V = typename M::T;
  __shared__ double sh[MC_WARPS];
  __shared__ bool s_last;
  const int ma = na_dev ? min(max(*na_dev, 0), na) : na;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  V acc = M::zero(), acc2 = M::zero();
  if (wi < ma) {
    const double* col = A + (size_t)wi * n;
    const long long stride = (long long)gridDim.x * 32;
    long long k = (long long)blockIdx.x * 32 + lane;
    for (; k + stride < n; k += 2 * stride) {
      const double a0 = col[k], b0 = b[k], a1 = col[k + stride], b1 = b[k + stride];
      acc = M::fma3(M::load(a0), M::load(b0), acc);
      acc2 = M::fma3(M::load(a1), M::load(b1), acc2);
    }
    if (k < n) acc = M::fma3(M::load(col[k]), M::load(b[k]), acc);
    if constexpr (DF) acc = df_add(acc, acc2);
    else acc += acc2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      if constexpr (DF) {
        const dfl y = {__shfl_down_sync(0xffffffffu, acc.h, o),
                       __shfl_down_sync(0xffffffffu, acc.l, o)};
        acc = df_add(acc, y);
      } else {
        acc += __shfl_down_sync(0xffffffffu, acc, o);
      }
    }
  }
  if (lane == 0) sh[wi] = wi < ma ? M::to_d(acc) : 0.0;
  __syncthreads();
  if (threadIdx.x < MC_WARPS) partials[(size_t)blockIdx.x * MC_WARPS + threadIdx.x] = sh[threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if ((int)threadIdx.x < ma) {
    double sum = 0.0;
    for (int bl = 0; bl < (int)gridDim.x; ++bl) sum += partials[(size_t)bl * MC_WARPS + threadIdx.x];
    g[threadIdx.x] = sum;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// y = beta*y + sign*sum_i c[i] A[:, i] (i < m <= MMAX); optional
// |y - w|^2 -> *rr.  DF: double-float accumulation, one float64 add per
// stored value.
template <bool DF, int MMAX>
__global__ void __launch_bounds__(RED_THREADS)
    k_combine(long long n, const double* __restrict__ A, int m, const int* m_dev,
              const double* __restrict__ c, double sign, double beta, double* __restrict__ y,
              const double* __restrict__ w, double* rr, double* partials, unsigned* counter) {
  using M = MdVal<DF>;
  using V = typename M::T;
  __shared__ double sh[32];
  const int mm = m_dev ? min(max(*m_dev, 0), m) : m;
  V cc[MMAX];
#pragma unroll
  for (int i = 0; i < MMAX; ++i) {
    const double ci = i < mm ? c[i] : 0.0;
    cc[i] = M::load(sign == 1.0 ? ci : sign == -1.0 ? -ci : sign * ci);
  }
  const V bb = M::load(beta);
  V v = M::zero();
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    double ca[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i) ca[i] = i < mm ? A[k + (size_t)i * n] : 0.0;
    const double cy = beta != 0.0 ? y[k] : 0.0;
    const double cw = (rr && w) ? w[k] : 0.0;
    V s = M::zero();
    if (beta != 0.0) s = (beta == 1.0) ? M::load(cy) : M::fma3(bb, M::load(cy), M::zero());
#pragma unroll
    for (int i = 0; i < MMAX; ++i)
      if (i < mm) s = M::fma3(cc[i], M::load(ca[i]), s);
    y[k] = M::to_d(s);
    if (rr) {
      V d = s;
      if (w) {
        if constexpr (DF) d = df_add(s, df_neg(split_d(cw)));
        else d = s - cw;
      }
      v = M::fma3(d, d, v);
    }
  }
  if (!rr) return;
  V vv[1] = {v};
  double o1[1];
  block_sum_md<DF, 1>(vv, o1, sh);
  if (publish_partials<1>(o1, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *rr = o[0];
  }
}

// ---------------------------------------------------------------------------
// Small dense float64 kernels (m <= 16), one thread does the work.
// ---------------------------------------------------------------------------
__device__ bool chol_small(int m, const double* A, double* L) {
  for (int i = 0; i < m * m; ++i) L[i] = 0.0;
  for (int j = 0; j < m; ++j) {
    double d = 0.5 * (A[j + m * j] + A[j + m * j]);
    for (int k = 0; k < j; ++k) d -= L[j + m * k] * L[j + m * k];
    if (!(d > 0.0)) return false;
    const double ljj = sqrt(d);
    L[j + m * j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double s = 0.5 * (A[i + m * j] + A[j + m * i]);
      for (int k = 0; k < j; ++k) s -= L[i + m * k] * L[j + m * k];
      L[i + m * j] = s / ljj;
    }
  }
  return true;
}

__device__ void chol_solve_small(int m, const double* L, const double* b, double* x) {
  double y[MAXB];
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[i + m * k] * y[k];
    y[i] = s / L[i + m * i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < m; ++k) s -= L[k + m * i] * x[k];
    x[i] = s / L[i + m * i];
  }
}

// Symmetric Jacobi eigen-decomposition (cyclic sweeps) of the m x m matrix
// A (column-major); eigenvalues in w, eigenvectors in the columns of V.
__device__ void jacobi_eigen(int m, double* A, double* w, double* V) {
  for (int i = 0; i < m * m; ++i) V[i] = 0.0;
  for (int i = 0; i < m; ++i) V[i + m * i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < m; ++p)
      for (int q = 0; q < m; ++q) {
        const double a = A[p + m * q] * A[p + m * q];
        tot += a;
        if (p != q) off += a;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = A[p + m * q];
        if (apq == 0.0) continue;
        const double theta = (A[q + m * q] - A[p + m * p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = A[k + m * p], akq = A[k + m * q];
          A[k + m * p] = c * akp - s * akq;
          A[k + m * q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = A[p + m * k], aqk = A[q + m * k];
          A[p + m * k] = c * apk - s * aqk;
          A[q + m * k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double vkp = V[k + m * p], vkq = V[k + m * q];
          V[k + m * p] = c * vkp - s * vkq;
          V[k + m * q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < m; ++i) w[i] = A[i + m * i];
}

// Ainv = A^{-1} for the small SPD K_Phi: Cholesky, else symmetric
// eigen-pseudo-inverse with relative cutoff 1e-14.
__global__ void k_small_spd_inverse(int mmax, const int* m_dev, const double* A, double* Ainv,
                                    int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = m_dev ? min(*m_dev, mmax) : mmax;
  double L[MAXB * MAXB];
  if (chol_small(m, A, L)) {
    double e[MAXB], col[MAXB];
    for (int j = 0; j < m; ++j) {
      for (int i = 0; i < m; ++i) e[i] = (i == j) ? 1.0 : 0.0;
      chol_solve_small(m, L, e, col);
      for (int i = 0; i < m; ++i) Ainv[i + m * j] = col[i];
    }
    return;
  }
  double S[MAXB * MAXB], V[MAXB * MAXB], w[MAXB];
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < m; ++i) S[i + m * j] = 0.5 * (A[i + m * j] + A[j + m * i]);
  jacobi_eigen(m, S, w, V);
  double wmax = 0.0;
  for (int i = 0; i < m; ++i) wmax = fmax(wmax, fabs(w[i]));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k)
        if (w[k] > 1e-14 * wmax) s += V[i + m * k] * V[j + m * k] / w[k];
      Ainv[i + m * j] = s;
    }
  (void)status;
}

// y = sign * A x (A column-major m x m)
__global__ void k_small_matvec(int mmax, const int* m_dev, const double* A, const double* x,
                               double* y, double sign) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = m_dev ? min(*m_dev, mmax) : mmax;
  for (int i = 0; i < m; ++i) {
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += A[i + m * k] * x[k];
    y[i] = sign * s;
  }
}

__global__ void k_small_chol_solve(int mmax, const int* m_dev, const double* A, const double* b,
                                   double* x, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = m_dev ? min(*m_dev, mmax) : mmax;
  double L[MAXB * MAXB];
  if (!chol_small(m, A, L)) {
    // fall back to the pseudo-inverse so that a result is still produced
    double S[MAXB * MAXB], V[MAXB * MAXB], w[MAXB];
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) S[i + m * j] = 0.5 * (A[i + m * j] + A[j + m * i]);
    jacobi_eigen(m, S, w, V);
    double wmax = 0.0;
    for (int i = 0; i < m; ++i) wmax = fmax(wmax, fabs(w[i]));
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) {
        if (!(w[k] > 1e-14 * wmax)) continue;
        double vb = 0.0;
        for (int q = 0; q < m; ++q) vb += V[q + m * k] * b[q];
        s += V[i + m * k] * vb / w[k];
      }
      x[i] = s;
    }
    if (status) *status = TO_E_SINGULAR;
    return;
  }
  chol_solve_small(m, L, b, x);
}

// Gram-Schmidt acceptance: column src (already orthogonalised twice) is
// kept if |r|^2 after > tol^2 |r|^2 before; it is then normalised into
// column k = ints[I_KCOUNT] and k is incremented.  Runs as a grid.
__global__ void __launch_bounds__(256)
    k_gs_accept(long long n, double* R, int src, const double* scal, int n0, int n1,
                double tol, int* ints) {
  __shared__ double s_scale;
  const double before = scal[n0], after = scal[n1];
  const bool keep = after > tol * tol * before && after > 0.0;
  const int k = ints[I_KCOUNT];
  if (keep) {
    if (threadIdx.x == 0) s_scale = 1.0 / sqrt(after);   // once per block
    __syncthreads();
    const double s = s_scale;
    const double* a = R + (size_t)src * n;
    double* b = R + (size_t)k * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
      b[i] = a[i] * s;
  }
}

__global__ void k_gs_count(const double* scal, int n0, int n1, double tol, int* ints) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double before = scal[n0], after = scal[n1];
  if (after > tol * tol * before && after > 0.0) ints[I_KCOUNT] += 1;
}

__global__ void k_eps(const double* scal, int rr, int f2, double* eps_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *eps_dev = sqrt(scal[rr] / scal[f2]);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline int vgrid(long long n) {
  long long b = (n + 255) / 256;
  if (b > RED_BLOCKS) b = RED_BLOCKS;
  return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_dot(long long n, const double* a, const double* b, double* partials,
                       unsigned* counter, double* out, cudaStream_t s) {
  k_dot<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, b, partials, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_xr(long long n, double* x, double* r, const double* p, const double* q,
                         double* scal, int num, int den, int rr, double* partials,
                         unsigned* counter, cudaStream_t s) {
  k_cg_xr<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, r, p, q, scal, num, den, rr, partials,
                                             counter);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(long long n, double* p, const double* z, const double* scal, int num,
                        int den, cudaStream_t s) {
  k_cg_p<<<vgrid(n), 256, 0, s>>>(n, p, z, scal, num, den);
  return cudaGetLastError();
}

cudaError_t launch_dot_df(long long n, const double* a, const float* b, double* partials,
                          unsigned* counter, double* out, cudaStream_t s) {
  k_dot_df<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, a, b, partials, counter, out);
  return cudaGetLastError();
}

cudaError_t launch_cg_xr_f(long long n, double* x, double* r, const double* p, const float* q,
                           double* scal, int num, int den, int rr, double* partials,
                           unsigned* counter, cudaStream_t s) {
  k_cg_xr_f<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, r, p, q, scal, num, den, rr, partials,
                                               counter);
  return cudaGetLastError();
}

cudaError_t launch_cg_p_f(long long n, double* p, float* p32, const float* z, const double* scal,
                          int num, int den, cudaStream_t s) {
  k_cg_p_f<<<vgrid(n), 256, 0, s>>>(n, p, p32, z, scal, num, den);
  return cudaGetLastError();
}

cudaError_t launch_copy(long long n, const double* a, double* b, cudaStream_t s) {
  k_copy<<<vgrid(n), 256, 0, s>>>(n, a, b);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_inv_sqrt(long long n, double* a, const double* s2, cudaStream_t s) {
  k_scale_inv_sqrt<<<vgrid(n), 256, 0, s>>>(n, a, s2);
  return cudaGetLastError();
}

cudaError_t launch_multidot(long long n, const double* A, int na, const int* na_dev,
                            const double* B, int nb, const int* nb_dev, double* G, int ldg,
                            double* partials, unsigned* counters, bool df, cudaStream_t s) {
  if (na > MAXB || nb > MAXB || na < 1 || nb < 1) return cudaErrorInvalidValue;
  if (nb == 1 && nb_dev == nullptr) {
    if (df)
      k_multidot_col<true><<<RED_BLOCKS, 32 * MC_WARPS, 0, s>>>(n, A, na, na_dev, B, G, partials,
                                                                counters);
    else
      k_multidot_col<false><<<RED_BLOCKS, 32 * MC_WARPS, 0, s>>>(n, A, na, na_dev, B, G,
                                                                 partials, counters);
    return cudaGetLastError();
  }
  if (df)
    k_multidot<true><<<RED_BLOCKS, MD_CH, 0, s>>>(n, A, na, na_dev, B, nb, nb_dev, G, ldg,
                                                  partials, counters);
  else
    k_multidot<false><<<RED_BLOCKS, MD_CH, 0, s>>>(n, A, na, na_dev, B, nb, nb_dev, G, ldg,
                                                   partials, counters);
  return cudaGetLastError();
}

template <bool DF>
static void combine_t(long long n, const double* A, int m, const int* m_dev, const double* c,
                      double sign, double beta, double* y, const double* w, double* rr,
                      double* partials, unsigned* counter, cudaStream_t s) {
  if (m <= 4)
    k_combine<DF, 4><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, A, m, m_dev, c, sign, beta, y, w, rr,
                                                        partials, counter);
  else if (m <= 8)
    k_combine<DF, 8><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, A, m, m_dev, c, sign, beta, y, w, rr,
                                                        partials, counter);
  else
    k_combine<DF, MAXB><<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, A, m, m_dev, c, sign, beta, y, w,
                                                           rr, partials, counter);
}

cudaError_t launch_combine(long long n, const double* A, int m, const int* m_dev,
                           const double* c, double sign, double beta, double* y,
                           const double* w, double* rr, double* partials, unsigned* counter,
                           bool df, cudaStream_t s) {
  if (m > MAXB || m < 0) return cudaErrorInvalidValue;
  if (df)
    combine_t<true>(n, A, m, m_dev, c, sign, beta, y, w, rr, partials, counter, s);
  else
    combine_t<false>(n, A, m, m_dev, c, sign, beta, y, w, rr, partials, counter, s);
  return cudaGetLastError();
}

cudaError_t launch_small_spd_inverse(int m, const int* m_dev, const double* A, double* Ainv,
                                     int* status, cudaStream_t s) {
  k_small_spd_inverse<<<1, 32, 0, s>>>(m, m_dev, A, Ainv, status);
  return cudaGetLastError();
}

cudaError_t launch_small_matvec(int m, const int* m_dev, const double* A, const double* x,
                                double* y, double sign, cudaStream_t s) {
  k_small_matvec<<<1, 32, 0, s>>>(m, m_dev, A, x, y, sign);
  return cudaGetLastError();
}

cudaError_t launch_small_chol_solve(int m, const int* m_dev, const double* A, const double* b,
                                    double* x, int* status, cudaStream_t s) {
  k_small_chol_solve<<<1, 32, 0, s>>>(m, m_dev, A, b, x, status);
  return cudaGetLastError();
}

cudaError_t launch_gs_accept(long long n, double* R, int src, const double* scal, int n0,
                             int n1, double tol, int* ints, cudaStream_t s) {
  k_gs_accept<<<vgrid(n), 256, 0, s>>>(n, R, src, scal, n0, n1, tol, ints);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gs_count<<<1, 32, 0, s>>>(scal, n0, n1, tol, ints);
  return cudaGetLastError();
}

cudaError_t launch_eps(const double* scal, int rr, int f2, double* eps_dev, cudaStream_t s) {
  k_eps<<<1, 32, 0, s>>>(scal, rr, f2, eps_dev);
  return cudaGetLastError();
}

}  // namespace topo
