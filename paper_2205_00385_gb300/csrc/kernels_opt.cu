// Design-side kernels: SIMP modulus (Eq. 1), density filter and its
// transpose (Eq. 31-33), compliance and sensitivity (Eq. 3, 6, 34) and the
// optimality-criteria update with a device-side bisection for the volume
// multiplier.  All float64.
#include <math.h>

#include "dfmath.cuh"
#include "kernels.h"

namespace topo {

__device__ __forceinline__ double ipow(double x, double p) {
  if (p == 3.0) return x * x * x;
  if (p == 2.0) return x * x;
  if (p == 1.0) return x;
  if (p == 4.0) return (x * x) * (x * x);
  return pow(x, p);
}

__global__ void __launch_bounds__(256)
    k_simp(long long nel, const double* __restrict__ rho, double E0, double Emin, double penal,
           double* __restrict__ E64, float* __restrict__ E32) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const double E = Emin + (E0 - Emin) * ipow(rho[e], penal);
  E64[e] = E;
  E32[e] = (float)E;
}

__global__ void __launch_bounds__(256)
    k_delta(long long nel, const double* __restrict__ E, const double* __restrict__ Ep,
            double* __restrict__ dE64, float* __restrict__ dE32, float* __restrict__ Ep32) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nel) return;
  const double d = E[e] - Ep[e];
  dE64[e] = d;
  dE32[e] = (float)d;
  Ep32[e] = (float)Ep[e];
}

// invHs_i = 1 / sum_j w_ij (precomputed, so no float64 division per term)
// mode 0: out_i = invHs_i sum_j w_ij in_j ; mode 1: out_e = sum_i w_ie in_i invHs_i
// mode 2: out_i = invHs_i (in ignored)
template <int DIM>
__global__ void __launch_bounds__(256)
    k_filter(GridP g, StencilP st, int mode, const double* __restrict__ invHs,
             const double* __restrict__ in, double* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.nel) return;
  const int ex = (int)(e % g.nx);
  const long long rest = e / g.nx;
  const int ey = (int)(rest % g.ny);
  const int ez = DIM == 3 ? (int)(rest / g.ny) : 0;
  double acc = 0.0;
  for (int q = 0; q < st.count; ++q) {
    const int jx = ex + st.d[q][0], jy = ey + st.d[q][1], jz = ez + st.d[q][2];
    bool in_range = jx >= 0 && jx < g.nx && jy >= 0 && jy < g.ny;
    if (DIM == 3) in_range = in_range && jz >= 0 && jz < g.nz;
    if (!in_range) continue;
    const long long j = jx + (long long)g.nx * (jy + (long long)g.ny * (DIM == 3 ? jz : 0));
    const double w = st.w[q];
    if (mode == 0)
      acc = fma(w, in[j], acc);
    else if (mode == 1)
      acc = fma(w, in[j] * invHs[j], acc);
    else
      acc += w;
  }
  if (mode == 0)
    out[e] = acc * invHs[e];
  else if (mode == 1)
    out[e] = acc;
  else
    out[e] = 1.0 / acc;
}

// Double-float Walsh blocks of KE (hi and lo parts of each float64 entry)
struct WhtDf {
  float h[8][3][3], l[8][3][3];
};

// 3D compliance and sensitivity of k_sensitivity3_wht in double-float
// arithmetic (mixed path), for an integer penalisation exponent:
// dc_e = pfac rho_e^ipen ce_e with pfac = -penal (E0 - Emin), ipen = penal - 1.
__global__ void __launch_bounds__(RED_THREADS)
    k_sensitivity3_df(GridP g, const uint8_t* __restrict__ mask, WhtDf kb,
                      const double* __restrict__ u, const double* __restrict__ E,
                      const double* __restrict__ rho, double pfac, int ipen,
                      double* __restrict__ dc, double* compliance, double* partials,
                      unsigned* counter) {
  __shared__ double sh[32];
  const dfl pf = split_d(pfac);
  dfl v[1] = {{0.f, 0.f}};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.nel;
       e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.nx);
    const long long rest = e / g.nx;
    const int ey = (int)(rest % g.ny);
    const int ez = (int)(rest / g.ny);
    dfl X[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = ex + (a & 1), j = ey + ((a >> 1) & 1), k = ez + ((a >> 2) & 1);
      const long long nd = i + (long long)g.nnx * (j + (long long)g.nny * k);
      const unsigned m = mask[nd];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        X[c][a] = ((m >> c) & 1u) ? dfl{0.f, 0.f} : split_d(u[3 * nd + c]);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int h = 1; h < 8; h <<= 1)
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (!(a & h)) {
            const dfl p = X[c][a], q = X[c][a + h];
            X[c][a] = df_add(p, q);
            X[c][a + h] = df_add(p, df_neg(q));
          }
    dfl ce = {0.f, 0.f};
#pragma unroll
    for (int tau = 0; tau < 8; ++tau) {
      dfl z[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = X[c][tau ^ (1 << c)];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dfl s = df_mul(dfl{kb.h[tau][c][0], kb.l[tau][c][0]}, z[0]);
        s = df_add(df_mul(dfl{kb.h[tau][c][1], kb.l[tau][c][1]}, z[1]), s);
        s = df_add(df_mul(dfl{kb.h[tau][c][2], kb.l[tau][c][2]}, z[2]), s);
        ce = df_add(df_mul(z[c], s), ce);
      }
    }
    const dfl re = split_d(rho[e]);
    dfl f = pf;
    for (int q = 0; q < ipen; ++q) f = df_mul(f, re);
    dc[e] = df_to_d(df_mul(f, ce));
    v[0] = df_add(df_mul(split_d(E[e]), ce), v[0]);
  }
  double o1[1];
  block_sum_df<1>(v, o1, sh);
  if (publish_partials<1>(o1, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *compliance = o[0];
  }
}

// ce_e = u_e^T KE u_e; dc_e = -penal (E0-Emin) rho_e^(penal-1) ce_e;
// compliance = sum_e E_e ce_e (deterministic reduction).
// 3D: u_e^T KE u_e = X^T B X with X the Walsh transform of u_e (KE = T B T),
// ~170 float64 operations per element instead of ~600.
__global__ void __launch_bounds__(RED_THREADS)
    k_sensitivity3_wht(GridP g, const uint8_t* __restrict__ mask, WhtBlocks<double> kb,
                       const double* __restrict__ u, const double* __restrict__ E,
                       const double* __restrict__ rho, double penal, double E0, double Emin,
                       double* __restrict__ dc, double* compliance, double* partials,
                       unsigned* counter) {
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.nel;
       e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.nx);
    const long long rest = e / g.nx;
    const int ey = (int)(rest % g.ny);
    const int ez = (int)(rest / g.ny);
    double X[3][8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = ex + (a & 1), j = ey + ((a >> 1) & 1), k = ez + ((a >> 2) & 1);
      const long long nd = i + (long long)g.nnx * (j + (long long)g.nny * k);
      const unsigned m = mask[nd];
#pragma unroll
      for (int c = 0; c < 3; ++c) X[c][a] = ((m >> c) & 1u) ? 0.0 : u[3 * nd + c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) fwht8<double>(X[c]);
    double ce = 0.0;
#pragma unroll
    for (int tau = 0; tau < 8; ++tau) {
      double z[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) z[c] = X[c][tau ^ (1 << c)];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s = kb.b[tau][c][0] * z[0];
        s = fma(kb.b[tau][c][1], z[1], s);
        s = fma(kb.b[tau][c][2], z[2], s);
        ce = fma(z[c], s, ce);
      }
    }
    const double re = rho[e];
    dc[e] = -penal * (E0 - Emin) * ipow(re, penal - 1.0) * ce;
    v[0] = fma(E[e], ce, v[0]);
  }
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *compliance = o[0];
  }
}

template <int DIM>
__global__ void __launch_bounds__(RED_THREADS)
    k_sensitivity(GridP g, const uint8_t* __restrict__ mask, KEP<double, Geo<DIM>::ND> ke,
                  const double* __restrict__ u, const double* __restrict__ E,
                  const double* __restrict__ rho, double penal, double E0, double Emin,
                  double* __restrict__ dc, double* compliance, double* partials,
                  unsigned* counter, const double* __restrict__ adj) {
  constexpr int ND = Geo<DIM>::ND, NPE = Geo<DIM>::NPE;
  __shared__ double sh[32];
  double v[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < g.nel;
       e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % g.nx);
    const long long rest = e / g.nx;
    const int ey = (int)(rest % g.ny);
    const int ez = DIM == 3 ? (int)(rest / g.ny) : 0;
    // ue: the field; ve: the adjoint field (the field itself for compliance)
    double ue[ND], ve[ND];
#pragma unroll
    for (int a = 0; a < NPE; ++a) {
      const int i = ex + (a & 1), j = ey + ((a >> 1) & 1), k = ez + ((a >> 2) & 1);
      const long long nd = i + (long long)g.nnx * (j + (long long)g.nny * (DIM == 3 ? k : 0));
      const unsigned m = mask[nd];
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const bool fx = (m >> c) & 1u;
        ue[DIM * a + c] = fx ? 0.0 : u[DIM * nd + c];
        ve[DIM * a + c] = fx ? 0.0 : (adj ? adj[DIM * nd + c] : u[DIM * nd + c]);
      }
    }
    double ce = 0.0;
#pragma unroll
    for (int r = 0; r < ND; ++r) {
      double s = 0.0;
#pragma unroll
      for (int c = 0; c < ND; ++c) s = fma(ke.v[r * ND + c], ue[c], s);
      ce = fma(ve[r], s, ce);
    }
    const double re = rho[e];
    dc[e] = -penal * (E0 - Emin) * ipow(re, penal - 1.0) * ce;
    v[0] = fma(E[e], ce, v[0]);
  }
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) *compliance = o[0];
  }
}

// a_e = rho_e sqrt(max(0, -dc_e / dv_e)); bracket [0, 1e9]
__global__ void __launch_bounds__(256)
    k_oc_prep(long long nel, const double* __restrict__ rho, const double* __restrict__ dc,
              const double* __restrict__ dv, double* __restrict__ a, double* scal) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    scal[S_OC_L1] = 0.0;
    scal[S_OC_L2] = 1e9;
  }
  if (e >= nel) return;
  a[e] = rho[e] * sqrt(fmax(0.0, -dc[e] / dv[e]));
}

__device__ __forceinline__ double oc_new(double a, double s, double r, double move) {
  const double lo = fmax(0.0, r - move), hi = fmin(1.0, r + move);
  return fmin(hi, fmax(lo, a * s));
}

// One bisection step: lmid = (l1+l2)/2; the filtered volume of rho_new(lmid)
// decides which half is kept (as in the oracle).  No-op once the bracket is
// within a relative 1e-13.
__global__ void __launch_bounds__(RED_THREADS)
    k_oc_step(long long nel, const double* __restrict__ rho, const double* __restrict__ a,
              const double* __restrict__ dv, double move, double target, double* scal,
              double* partials, unsigned* counter) {
  __shared__ double sh[32];
  const double l1 = scal[S_OC_L1], l2 = scal[S_OC_L2];
  if (!((l2 - l1) > 1e-13 * (l1 + l2))) return;
  const double lmid = 0.5 * (l1 + l2);
  const double s = 1.0 / sqrt(lmid);
  double v[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nel;
       e += (long long)gridDim.x * blockDim.x)
    v[0] = fma(dv[e], oc_new(a[e], s, rho[e], move), v[0]);
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) {
      if (o[0] > target)
        scal[S_OC_L1] = lmid;
      else
        scal[S_OC_L2] = lmid;
      scal[S_OC_VOL] = o[0];
    }
  }
}

// Context path: the move-limit bounds are stored once, so a bisection step
// costs one multiply, two clamps and one multiply-add in float64 per element
// (same values as k_oc_step, which recomputes them).
__global__ void __launch_bounds__(256)
    k_oc_prep_b(long long nel, const double* __restrict__ rho, const double* __restrict__ dc,
                const double* __restrict__ dv, double move, double* __restrict__ a,
                double* __restrict__ lo, double* __restrict__ hi, double* scal) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    scal[S_OC_L1] = 0.0;
    scal[S_OC_L2] = 1e9;
  }
  if (e >= nel) return;
  const double r = rho[e];
  a[e] = r * sqrt(fmax(0.0, -dc[e] / dv[e]));
  lo[e] = fmax(0.0, r - move);
  hi[e] = fmin(1.0, r + move);
}

__global__ void __launch_bounds__(RED_THREADS)
    k_oc_step_b(long long nel, const double* __restrict__ a, const double* __restrict__ lo,
                const double* __restrict__ hi, const double* __restrict__ dv, double target,
                double* scal, double* partials, unsigned* counter) {
  __shared__ double sh[32];
  const double l1 = scal[S_OC_L1], l2 = scal[S_OC_L2];
  if (!((l2 - l1) > 1e-13 * (l1 + l2))) return;
  const double lmid = 0.5 * (l1 + l2);
  const double s = 1.0 / sqrt(lmid);
  double v[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nel;
       e += (long long)gridDim.x * blockDim.x)
    v[0] = fma(dv[e], fmin(hi[e], fmax(lo[e], a[e] * s)), v[0]);
  block_sum<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_sum<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) {
      if (o[0] > target)
        scal[S_OC_L1] = lmid;
      else
        scal[S_OC_L2] = lmid;
      scal[S_OC_VOL] = o[0];
    }
  }
}

// Context path of the mixed and float64 solvers alike: the lambda search
// runs as an OC_SPLIT-way section per pass in double-float on the FP32 pipe
// (the volume at OC_SPLIT - 1 interior points of [l1, l2] is summed for
// every element in one sweep, and the sub-interval holding the root is
// kept), 3 bits of bracket per sweep against 1 for a float64 bisection
// step.  It stops at the same relative bracket of 1e-13.
constexpr int OC_SPLIT = 8;

// x^eta of the OC rule (sqrt for the compliance rule's eta = 1/2) and the
// multiplier's factor lambda^-eta
__device__ __forceinline__ double oc_damp(double x, double eta) {
  return eta == 0.5 ? sqrt(x) : pow(x, eta);
}
__device__ __forceinline__ double oc_lam_factor(double lam, double eta) {
  return eta == 0.5 ? 1.0 / sqrt(lam) : pow(lam, -eta);
}

__global__ void __launch_bounds__(256)
    k_oc_prep_d(long long nel, const double* __restrict__ rho, const double* __restrict__ dc,
                const double* __restrict__ dv, double move, double* __restrict__ a64,
                float2* __restrict__ a, float2* __restrict__ lo, float2* __restrict__ hi,
                float2* __restrict__ dvd, double* scal, double eta) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e == 0) {
    scal[S_OC_L1] = 0.0;
    scal[S_OC_L2] = 1e9;
  }
  if (e >= nel) return;
  const double r = rho[e];
  const double ae = r * oc_damp(fmax(0.0, -dc[e] / dv[e]), eta);
  a64[e] = ae;
  const dfl av = split_d(ae);
  const dfl lv = split_d(fmax(0.0, r - move)), hv = split_d(fmin(1.0, r + move));
  const dfl dd = split_d(dv[e]);
  a[e] = make_float2(av.h, av.l);
  lo[e] = make_float2(lv.h, lv.l);
  hi[e] = make_float2(hv.h, hv.l);
  dvd[e] = make_float2(dd.h, dd.l);
}

// Section point j (1 .. OC_SPLIT-1) of the bracket [l1, l2]: evenly spaced,
// or, while the lower end is still 0, geometric (l2 / 8^(OC_SPLIT - j)), which
// brings an upper end far above lambda down by up to 8^7 per sweep; point
// OC_SPLIT is l2 itself.
__device__ __forceinline__ double oc_point(double l1, double l2, int j) {
  if (j >= OC_SPLIT) return l2;
  if (l1 == 0.0) return ldexp(l2, -3 * (OC_SPLIT - j));
  return l1 + (double)j * ((l2 - l1) / OC_SPLIT);
}

__global__ void __launch_bounds__(RED_THREADS)
    k_oc_section(long long nel, const float2* __restrict__ a, const float2* __restrict__ lo,
                 const float2* __restrict__ hi, const float2* __restrict__ dvd, double target,
                 double* scal, double* partials, unsigned* counter, double eta) {
  constexpr int NP = OC_SPLIT - 1;
  __shared__ double sh[NP * 32];
  __shared__ dfl s_s[NP];
  const double l1 = scal[S_OC_L1], l2 = scal[S_OC_L2];
  if (!((l2 - l1) > 1e-13 * (l1 + l2))) return;
  if (threadIdx.x < NP) {
    const double lam = oc_point(l1, l2, threadIdx.x + 1);
    s_s[threadIdx.x] = split_d(oc_lam_factor(lam, eta));
  }
  __syncthreads();
  dfl sv[NP], v[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    sv[j] = s_s[j];
    v[j] = {0.f, 0.f};
  }
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nel;
       e += (long long)gridDim.x * blockDim.x) {
    const float2 a2 = a[e], l2v = lo[e], h2 = hi[e], d2 = dvd[e];
    const dfl av = {a2.x, a2.y}, lv = {l2v.x, l2v.y}, hv = {h2.x, h2.y}, dd = {d2.x, d2.y};
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      dfl x = df_mul(av, sv[j]);
      x = df_gt(x, hv) ? hv : (df_gt(lv, x) ? lv : x);
      df_dot_acc(v[j], dd, x);
    }
  }
#pragma unroll
  for (int j = 0; j < NP; ++j) v[j] = df_norm(v[j]);
  double o1[NP];
  block_sum_df<NP>(v, o1, sh);
  if (publish_partials<NP>(o1, partials, counter)) {
    double o[NP];
    finish_sum<NP>(partials, counter, o, sh);
    if (threadIdx.x == 0) {
      // the volume decreases with lambda: keep the last point above target
      // and the first at or below it
      int k = 0;
      while (k < NP && o[k] > target) ++k;
      const double nl1 = k > 0 ? oc_point(l1, l2, k) : l1;
      const double nl2 = oc_point(l1, l2, k + 1);
      scal[S_OC_L1] = nl1;
      scal[S_OC_L2] = nl2;
      scal[S_OC_VOL] = k > 0 ? o[k - 1] : o[0];
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS)
    k_oc_final(long long nel, double* __restrict__ rho, const double* __restrict__ a,
               double move, double* scal, double* change_dev, double* partials,
               unsigned* counter, double eta) {
  __shared__ double sh[32];
  const double lam = 0.5 * (scal[S_OC_L1] + scal[S_OC_L2]);
  const double s = oc_lam_factor(lam, eta);
  double v[1] = {0.0};
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nel;
       e += (long long)gridDim.x * blockDim.x) {
    const double r = rho[e];
    const double rn = oc_new(a[e], s, r, move);
    rho[e] = rn;
    v[0] = fmax(v[0], fabs(rn - r));
  }
  block_max<1>(v, sh);
  if (publish_partials<1>(v, partials, counter)) {
    double o[1];
    finish_max<1>(partials, counter, o, sh);
    if (threadIdx.x == 0) {
      scal[S_CHANGE] = o[0];
      if (change_dev) *change_dev = o[0];
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_simp(long long nel, const double* rho, double E0, double Emin, double penal,
                        double* E64, float* E32, cudaStream_t s) {
  k_simp<<<nblocks(nel, 256), 256, 0, s>>>(nel, rho, E0, Emin, penal, E64, E32);
  return cudaGetLastError();
}

cudaError_t launch_delta(long long nel, const double* E, const double* Eprev, double* dE64,
                         float* dE32, float* Eprev32, cudaStream_t s) {
  k_delta<<<nblocks(nel, 256), 256, 0, s>>>(nel, E, Eprev, dE64, dE32, Eprev32);
  return cudaGetLastError();
}

cudaError_t launch_filter(int dim, const GridP& g, const StencilP& st, int mode,
                          const double* Hs, const double* in, double* out, cudaStream_t s) {
  if (dim == 2)
    k_filter<2><<<nblocks(g.nel, 256), 256, 0, s>>>(g, st, mode, Hs, in, out);
  else
    k_filter<3><<<nblocks(g.nel, 256), 256, 0, s>>>(g, st, mode, Hs, in, out);
  return cudaGetLastError();
}

bool sensitivity_df_ok(int dim, double penal) {
  return dim == 3 && penal >= 1.0 && penal <= 9.0 && penal == (double)(int)penal;
}

cudaError_t launch_sensitivity_df(const GridP& g, const uint8_t* mask, const double* wht,
                                  const double* u, const double* E, const double* rho,
                                  double penal, double E0, double Emin, double* dc,
                                  double* compliance, double* partials, unsigned* counter,
                                  cudaStream_t s) {
  if (!wht || !sensitivity_df_ok(3, penal)) return cudaErrorInvalidValue;
  WhtDf kb;
  for (int q = 0; q < 72; ++q) {
    const float h = (float)wht[q];
    (&kb.h[0][0][0])[q] = h;
    (&kb.l[0][0][0])[q] = (float)(wht[q] - (double)h);
  }
  k_sensitivity3_df<<<RED_BLOCKS, RED_THREADS, 0, s>>>(g, mask, kb, u, E, rho,
                                                       -penal * (E0 - Emin), (int)penal - 1, dc,
                                                       compliance, partials, counter);
  return cudaGetLastError();
}

cudaError_t launch_filter_norm(int dim, const GridP& g, const StencilP& st, double* Hs,
                               cudaStream_t s) {
  return launch_filter(dim, g, st, 2, nullptr, nullptr, Hs, s);
}

template <int DIM>
static cudaError_t sens_t(const GridP& g, const uint8_t* mask, const double* kev, const double* u,
                          const double* E, const double* rho, double penal, double E0,
                          double Emin, double* dc, double* compliance, double* partials,
                          unsigned* counter, cudaStream_t s, const double* v) {
  constexpr int ND = Geo<DIM>::ND;
  KEP<double, ND> ke;
  for (int q = 0; q < ND * ND; ++q) ke.v[q] = kev[q];
  k_sensitivity<DIM><<<RED_BLOCKS, RED_THREADS, 0, s>>>(g, mask, ke, u, E, rho, penal, E0, Emin,
                                                        dc, compliance, partials, counter, v);
  return cudaGetLastError();
}

cudaError_t launch_sensitivity(int dim, const GridP& g, const uint8_t* mask, const double* ke,
                               const double* wht, const double* u, const double* E,
                               const double* rho, double penal, double E0, double Emin,
                               double* dc, double* compliance, double* partials,
                               unsigned* counter, cudaStream_t s, const double* v) {
  if (dim == 2)
    return sens_t<2>(g, mask, ke, u, E, rho, penal, E0, Emin, dc, compliance, partials, counter, s,
                     v);
  if (wht && !v) {
    WhtBlocks<double> kb;
    for (int q = 0; q < 72; ++q) (&kb.b[0][0][0])[q] = wht[q];
    k_sensitivity3_wht<<<RED_BLOCKS, RED_THREADS, 0, s>>>(g, mask, kb, u, E, rho, penal, E0, Emin,
                                                          dc, compliance, partials, counter);
    return cudaGetLastError();
  }
  return sens_t<3>(g, mask, ke, u, E, rho, penal, E0, Emin, dc, compliance, partials, counter, s,
                   v);
}

cudaError_t launch_oc_prep(long long nel, const double* rho, const double* dc,
                           const double* dv, double* a, double* scal, cudaStream_t s) {
  k_oc_prep<<<nblocks(nel, 256), 256, 0, s>>>(nel, rho, dc, dv, a, scal);
  return cudaGetLastError();
}

cudaError_t launch_oc_step(long long nel, const double* rho, const double* a,
                           const double* dv, double move, double target, double* scal,
                           double* partials, unsigned* counter, cudaStream_t s) {
  k_oc_step<<<RED_BLOCKS, RED_THREADS, 0, s>>>(nel, rho, a, dv, move, target, scal, partials,
                                               counter);
  return cudaGetLastError();
}

cudaError_t launch_oc_prep_b(long long nel, const double* rho, const double* dc,
                             const double* dv, double move, double* a, double* lo, double* hi,
                             double* scal, cudaStream_t s) {
  k_oc_prep_b<<<nblocks(nel, 256), 256, 0, s>>>(nel, rho, dc, dv, move, a, lo, hi, scal);
  return cudaGetLastError();
}

cudaError_t launch_oc_step_b(long long nel, const double* a, const double* lo, const double* hi,
                             const double* dv, double target, double* scal, double* partials,
                             unsigned* counter, cudaStream_t s) {
  k_oc_step_b<<<RED_BLOCKS, RED_THREADS, 0, s>>>(nel, a, lo, hi, dv, target, scal, partials,
                                                 counter);
  return cudaGetLastError();
}

cudaError_t launch_oc_prep_d(long long nel, const double* rho, const double* dc,
                             const double* dv, double move, double* a64, void* a2, void* lo2,
                             void* hi2, void* dv2, double* scal, cudaStream_t s, double eta) {
  k_oc_prep_d<<<nblocks(nel, 256), 256, 0, s>>>(nel, rho, dc, dv, move, a64, (float2*)a2,
                                                (float2*)lo2, (float2*)hi2, (float2*)dv2, scal,
                                                eta);
  return cudaGetLastError();
}

cudaError_t launch_oc_section(long long nel, const void* a2, const void* lo2, const void* hi2,
                              const void* dv2, double target, double* scal, double* partials,
                              unsigned* counter, cudaStream_t s, double eta) {
  k_oc_section<<<RED_BLOCKS, RED_THREADS, 0, s>>>(nel, (const float2*)a2, (const float2*)lo2,
                                                  (const float2*)hi2, (const float2*)dv2, target,
                                                  scal, partials, counter, eta);
  return cudaGetLastError();
}

cudaError_t launch_oc_final(long long nel, double* rho, const double* a, double move,
                            double* scal, double* change_dev, double* partials,
                            unsigned* counter, cudaStream_t s, double eta) {
  k_oc_final<<<RED_BLOCKS, RED_THREADS, 0, s>>>(nel, rho, a, move, scal, change_dev, partials,
                                                counter, eta);
  return cudaGetLastError();
}

}  // namespace topo
