// Float64 vector kernels of the CG recursion, the CARM/PARM multi-vector
// products and Gram-Schmidt, and small dense solves run on one block.
// All reductions use a fixed grid of RED_BLOCKS blocks and a fixed summation
// tree, so results do not depend on timing or on other work on the GPU.
#include <math.h>

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

// host_rr (may be null): pinned host memory mapped into the device's
// address space that also receives |r|^2
__global__ void __launch_bounds__(RED_THREADS)
    k_cg_xr(long long n, double* __restrict__ x, double* __restrict__ r,
            const double* __restrict__ p, const double* __restrict__ q, double* scal, int num,
            int den, int rr, double* partials, unsigned* counter, double* host_rr) {
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
    if (threadIdx.x == 0) {
      scal[rr] = o[0];
      if (host_rr) {
        *reinterpret_cast<volatile double*>(host_rr) = o[0];
        __threadfence_system();
      }
    }
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

// Truncated SVD of Eq. 21 from the QR factor of the CARM basis.  The
// basis R (m columns) equals Q Rt with Q orthonormal (kq columns) and Rt
// kq x m; with D the column norms of R, the unit-column basis R D^-1 has the
// singular values of A = Rt D^-1, and its left singular vectors are Q U with
// U those of A.  One-sided (Hestenes) Jacobi on the columns of A, lane r of
// a warp holding row r: each rotation makes a pair of columns orthogonal,
// until every pair is orthogonal to 1e-15 of the product of their norms;
// the column norms are then the singular values.  Directions
// with sigma <= tau sigma_1 are dropped; the kept ones, in descending order,
// are written to U (ld MAXB), their count to ints[I_KRED] and every
// singular value, descending, to sig.  A column of R that is zero (norm 0)
// contributes nothing.
__global__ void __launch_bounds__(32 * MAXB / 2)
    k_small_svd_trunc(int m, const int* kq_dev, const double* Rt, const double* rn, double tau,
                      double* U, double* sig, int* ints) {
  __shared__ double sA[MAXB * 32];   // column j, row r at sA[32 j + r]
  __shared__ double snrm[MAXB];
  __shared__ int sord[MAXB];
  __shared__ int s_rot;
  if (blockIdx.x != 0) return;
  const int r = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int kq = min(max(*kq_dev, 0), MAXB);
  m = min(max(m, 0), MAXB);
  for (int idx = threadIdx.x; idx < MAXB * 32; idx += blockDim.x) {
    const int j = idx >> 5, rr = idx & 31;
    double v = 0.0;
    if (j < m && rr < kq && rn[j] > 0.0) v = Rt[rr + (size_t)MAXB * j] / rn[j];
    sA[idx] = v;
  }
  __syncthreads();
  auto wsum = [](double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  };
  // One-sided (Hestenes) Jacobi in parallel order: the columns are paired by
  // the round-robin tournament (position 0 fixed, the others rotating), so
  // each of the mm - 1 steps of a sweep rotates mm / 2 disjoint pairs at once,
  // one warp per pair, and every pair meets once per sweep.
  const int mm = m + (m & 1);   // an odd count gets an empty partner
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int step = 0; step + 1 < mm; ++step) {
      if (w < mm / 2) {
        auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + step) % (mm - 1); };
        const int a = player(w), b = player(mm - 1 - w);
        const int p = min(a, b), q = max(a, b);
        if (q < m) {
          const double ap = sA[32 * p + r], aq = sA[32 * q + r];
          const double alpha = wsum(ap * ap), beta = wsum(aq * aq), gamma = wsum(ap * aq);
          if (fabs(gamma) > 1e-15 * sqrt(alpha * beta)) {
            const double zeta = (beta - alpha) / (2.0 * gamma);
            const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
            sA[32 * p + r] = c * ap - sn * aq;
            sA[32 * q + r] = sn * ap + c * aq;
            if (r == 0) s_rot = 1;
          }
        }
      }
      __syncthreads();
    }
    if (!s_rot) break;
    __syncthreads();
  }
  if (w != 0) return;
  for (int j = 0; j < MAXB; ++j) {
    const double a = sA[32 * j + r];
    const double nj = sqrt(wsum(a * a));
    if (r == 0) snrm[j] = j < m ? nj : -1.0;
  }
  __syncwarp();
  if (r == 0) {
    // descending order of the column norms (ties keep column order)
    bool used[MAXB];
    for (int j = 0; j < MAXB; ++j) used[j] = false;
    for (int t = 0; t < m; ++t) {
      int best = -1;
      for (int j = 0; j < m; ++j)
        if (!used[j] && (best < 0 || snrm[j] > snrm[best])) best = j;
      used[best] = true;
      sord[t] = best;
    }
  }
  __syncwarp();
  const double s1 = m > 0 ? snrm[sord[0]] : 0.0;
  int k = 0;
  for (int t = 0; t < m; ++t) {
    const int j = sord[t];
    const double sj = snrm[j];
    if (r == 0) sig[t] = sj;
    if (!(s1 > 0.0) || !(sj > tau * s1)) continue;
    if (r < kq) U[r + (size_t)MAXB * k] = sA[32 * j + r] / sj;
    ++k;
  }
  if (r == 0) ints[I_KRED] = k;
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
                         unsigned* counter, cudaStream_t s, double* host_rr) {
  k_cg_xr<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, r, p, q, scal, num, den, rr, partials,
                                             counter, host_rr);
  return cudaGetLastError();
}

cudaError_t launch_cg_p(long long n, double* p, const double* z, const double* scal, int num,
                        int den, cudaStream_t s) {
  k_cg_p<<<vgrid(n), 256, 0, s>>>(n, p, z, scal, num, den);
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


cudaError_t launch_small_svd_trunc(int m, const int* kq_dev, const double* Rt, const double* rn,
                                   double tau, double* U, double* sig, int* ints,
                                   cudaStream_t s) {
  if (m < 1 || m > MAXB) return cudaErrorInvalidValue;
  k_small_svd_trunc<<<1, 32 * MAXB / 2, 0, s>>>(m, kq_dev, Rt, rn, tau, U, sig, ints);
  return cudaGetLastError();
}

cudaError_t launch_eps(const double* scal, int rr, int f2, double* eps_dev, cudaStream_t s) {
  k_eps<<<1, 32, 0, s>>>(scal, rr, f2, eps_dev);
  return cudaGetLastError();
}

}  // namespace topo
