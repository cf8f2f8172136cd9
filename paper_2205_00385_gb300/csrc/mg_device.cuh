// Per-item bodies of the multigrid transfer and stored-level stencil kernels
// (Algorithm 2: restriction P^T, interpolation P, the level operator with
// its residual / damped-Jacobi epilogues).  The fused coarse V-cycle
// (kernels_vfuse.cu) calls all of them, the one-kernel-per-step
// interpolation and stencil apply (kernels_mg.cu, kernels_fe.cu) call
// theirs, and the one-kernel restriction (kernels_mg.cu, one thread per
// value) repeats restrict_finish's per-term arithmetic in the same order,
// so the two paths compute the same values bit for bit.
//
// CG selects how vectors that the calling kernel may itself have written are
// loaded: false, a plain load (one kernel per step: the data come from
// earlier kernels); true, ld.global.cg (cached in L2 only), for the fused
// kernel whose CTAs exchange those vectors between phases of one launch.
#pragma once

#include "kernels.h"

namespace topo {

template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// ---------------------------------------------------------------------------
// Assembled stencil of a stored level: per DOF row, the coefficients of the
// 3^DIM neighbouring nodes' DIM components (81 in 3D).  Boundary conditions
// are folded in at assembly (fixed columns are zero, a fixed row is the
// identity row), so the apply is a plain stencil product
//   y_r = sum_q S_r[q] x[col(r, q)].
// Coefficient qq of neighbour plane pz couples row r = DIM n + c with
// component qq % DIM of the neighbour n + (dx, dy, dz), qq / DIM =
// (dx+1) + 3 (dy+1), pz = dz + 1.  Layout: each plane's 9 DIM coefficients
// are padded to a multiple of W = 16 / sizeof(T) and stored in W-wide groups
// group-major, S[((pz GP + qq / W) rows + r) W + qq % W], so that a row's
// coefficients are GP 16-byte loads per plane and a warp's load of one group
// is 512 contiguous bytes.
// ---------------------------------------------------------------------------
template <int DIM, typename T>
struct StencilLayout {
  static constexpr int NP = DIM == 3 ? 3 : 1;          // neighbour planes
  static constexpr int NQP = 9 * DIM;                  // coefficients per plane
  static constexpr int W = 16 / (int)sizeof(T);        // values per group
  static constexpr int GP = (NQP + W - 1) / W;         // groups per plane
  __host__ __device__ static long long index(long long rows, long long r, int pz, int qq) {
    return ((long long)(pz * GP + qq / W) * rows + r) * W + qq % W;
  }
  __host__ __device__ static long long values(long long rows) { return rows * NP * GP * W; }
};

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using V = float4;
  __device__ static float get(const float4& v, int l) {
    return l == 0 ? v.x : l == 1 ? v.y : l == 2 ? v.z : v.w;
  }
};
template <>
struct Vec16<double> {
  using V = double2;
  __device__ static double get(const double2& v, int l) { return l == 0 ? v.x : v.y; }
};

// Row r of y = S x with the epilogue (K x, b - K x, or the damped Jacobi
// sweep); each plane's coefficient groups and neighbour values are all
// loaded before its sums, which run in a fixed order.
template <int DIM, typename T, int EPI, bool CG>
__device__ __forceinline__ void stencil_row(const GridP& g, const T* __restrict__ S,
                                            const T* __restrict__ x, T* __restrict__ y,
                                            const T* __restrict__ b, const T* __restrict__ dinv,
                                            T omega, long long r) {
  using SL = StencilLayout<DIM, T>;
  using VV = typename Vec16<T>::V;
  const long long rows = DIM * g.nn;
  const long long n = r / DIM;
  const int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny);
  const int k = DIM == 3 ? (int)(n / ((long long)g.nnx * g.nny)) : 0;
  // clamped neighbour indices (their coefficients are zero outside the grid)
  int ix[3], jy[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    ix[d] = min(max(i + d - 1, 0), g.nnx - 1);
    jy[d] = min(max(j + d - 1, 0), g.nny - 1);
  }
  const VV* Sv = reinterpret_cast<const VV*>(S);
  T acc = T(0);
#pragma unroll
  for (int pz = 0; pz < SL::NP; ++pz) {
    const int kz = DIM == 3 ? min(max(k + pz - 1, 0), g.nnz - 1) : 0;
    VV sv[SL::GP];
    T xv[SL::NQP];
#pragma unroll
    for (int q = 0; q < SL::GP; ++q) sv[q] = __ldg(Sv + (long long)(pz * SL::GP + q) * rows + r);
#pragma unroll
    for (int qq = 0; qq < SL::NQP; ++qq) {
      const int o = qq / DIM, cp = qq % DIM;
      const long long m = ix[o % 3] + (long long)g.nnx * (jy[o / 3] + (long long)g.nny * kz);
      xv[qq] = ldv<CG>(x + DIM * m + cp);
    }
#pragma unroll
    for (int qq = 0; qq < SL::NQP; ++qq)
      acc = fma(Vec16<T>::get(sv[qq / SL::W], qq % SL::W), xv[qq], acc);
  }
  if (EPI == EPI_APPLY)
    y[r] = acc;
  else if (EPI == EPI_RESID)
    y[r] = ldv<CG>(b + r) - acc;
  else
    y[r] = ldv<CG>(x + r) + omega * __ldg(dinv + r) * (ldv<CG>(b + r) - acc);
}

// Products and sums rounded one by one (no contraction into FMAs), so that
// every kernel calling these bodies computes the same bits whatever the
// compiler does around them.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// The weighted sum of a coarse node's 3^DIM fine neighbours (masks m and
// values v as loaded, index (a, b, q) = (dz, dy, dx) + 1), in a fixed order,
// and the coarse node's outputs.
template <int DIM, typename T>
__device__ __forceinline__ void restrict_finish(const GridP& gf, const GridP& gc,
                                                const uint8_t* __restrict__ maskc,
                                                const unsigned (&m)[DIM == 3 ? 3 : 1][3][3],
                                                const T (&v)[DIM == 3 ? 3 : 1][3][3][DIM],
                                                T* __restrict__ bc, const T* __restrict__ dinvc,
                                                T omega, T* __restrict__ zc, int I, int J, int K) {
  constexpr int NZ = DIM == 3 ? 3 : 1;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int a = 0; a < NZ; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int dx = q - 1, dy = b - 1, dz = DIM == 3 ? a - 1 : 0;
        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        bool in = i >= 0 && i < gf.nnx && j >= 0 && j < gf.nny;
        if (DIM == 3) in = in && k >= 0 && k < gf.nnz;
        const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
        const unsigned mm = in ? m[a][b][q] : 7u;
#pragma unroll
        for (int c = 0; c < DIM; ++c)
          acc[c] = add_rn(acc[c], ((mm >> c) & 1u) ? T(0) : mul_rn(w, v[a][b][q][c]));
      }
  const long long node = I + (long long)gc.nnx * (J + (long long)gc.nny * K);
  const unsigned mc = maskc[node];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long d = DIM * node + c;
    const T bv = ((mc >> c) & 1u) ? T(0) : acc[c];
    bc[d] = bv;
    if (zc) zc[d] = mul_rn(mul_rn(omega, dinvc[d]), bv);
  }
}

// ---------------------------------------------------------------------------
// Restriction b_c = Pm^T r_f (Pm = M_f P M_c) at coarse node (I, J, K): it
// gathers the fine nodes around (2I, 2J, 2K) with weights prod(1 - |d|/2).
// Every fine load is issued before any is used: indices are clamped into the
// grid and the out-of-range and fixed terms are dropped by selects after the
// loads, so the 3^DIM masks and values take one memory round trip; the terms
// are then summed in a fixed order.  With zc set, the coarse level is also
// pre-smoothed from a zero guess, z = omega D^-1 b.
// ---------------------------------------------------------------------------
template <int DIM, typename T, bool CG>
__device__ __forceinline__ void restrict_node(const GridP& gf, const uint8_t* __restrict__ maskf,
                                              const GridP& gc, const uint8_t* __restrict__ maskc,
                                              const T* __restrict__ rf, T* __restrict__ bc,
                                              const T* __restrict__ dinvc, T omega,
                                              T* __restrict__ zc, int I, int J, int K) {
  constexpr int NZ = DIM == 3 ? 3 : 1;
  unsigned m[NZ][3][3];
  T v[NZ][3][3][DIM];
#pragma unroll
  for (int a = 0; a < NZ; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int i = min(max(2 * I + q - 1, 0), gf.nnx - 1);
        const int j = min(max(2 * J + b - 1, 0), gf.nny - 1);
        const int k = DIM == 3 ? min(max(2 * K + a - 1, 0), gf.nnz - 1) : 0;
        const long long fn = i + (long long)gf.nnx * (j + (long long)gf.nny * k);
        m[a][b][q] = maskf[fn];
#pragma unroll
        for (int c = 0; c < DIM; ++c) v[a][b][q][c] = ldv<CG>(rf + DIM * fn + c);
      }
  restrict_finish<DIM, T>(gf, gc, maskc, m, v, bc, dinvc, omega, zc, I, J, K);
}

// ---------------------------------------------------------------------------
// z_f += Pm z_c for the fine nodes (i, j, 2q) and (i, j, 2q + 1) (3D; one
// node in 2D): each interpolates from coarse nodes floor(./2) .. ceil(./2)
// per axis, i.e. from 2 parents along an axis where its index is odd and 1
// where it is even.  Only the parents that exist are loaded (the y parity
// and the z position are uniform over a warp of the one-kernel path, the x
// parity is per lane), all before any sum, together with the fine values;
// each fine node then sums its parents' terms in a fixed order.
// ---------------------------------------------------------------------------
// The interpolated value at fine node (i, j, k), one component: its own
// value zv plus the weighted coarse values cv[a][bb][cc] at coarse nodes
// (i/2 + cc, j/2 + bb, k/2 + a), summed over the parents the node
// interpolates from with a (z) outermost and cc (x) innermost; the entries
// of other positions are not read.
template <int DIM, typename T>
__device__ __forceinline__ T prolong_one(T zv, const T (&cv)[DIM == 3 ? 2 : 1][2][2], int i, int j,
                                         int k) {
  constexpr int NK = DIM == 3 ? 2 : 1;
  const bool xo = i & 1, yo = j & 1, zo = DIM == 3 && (k & 1);
  const T w = mul_rn(mul_rn(xo ? T(0.5) : T(1), yo ? T(0.5) : T(1)), zo ? T(0.5) : T(1));
  T acc = T(0);
#pragma unroll
  for (int a = 0; a < NK; ++a) {
    if (a == 1 && !zo) break;
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      if (bb == 1 && !yo) break;
      acc = add_rn(acc, mul_rn(w, cv[a][bb][0]));
      if (xo) acc = add_rn(acc, mul_rn(w, cv[a][bb][1]));
    }
  }
  return add_rn(zv, acc);
}

template <int DIM, typename T, bool CG>
__device__ __forceinline__ void prolong_pair(const GridP& gf, const uint8_t* __restrict__ maskf,
                                             const GridP& gc, const T* __restrict__ zc,
                                             T* __restrict__ zf, int i, int j, int q) {
  constexpr int NK = DIM == 3 ? 2 : 1;   // fine nodes per item along z
  const int i0 = i >> 1, j0 = j >> 1;
  const bool xo = i & 1, yo = j & 1;
  const bool second = DIM == 3 && 2 * q + 1 < gf.nnz;   // node (i, j, 2q + 1) exists
  T cv[DIM][NK][2][2];
#pragma unroll
  for (int a = 0; a < NK; ++a)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const bool need = (a == 0 || second) && (bb == 0 || yo) && (cc == 0 || xo);
        const long long cn = (i0 + cc) + (long long)gc.nnx * ((j0 + bb) + (long long)gc.nny * (q + a));
#pragma unroll
        for (int c = 0; c < DIM; ++c) cv[c][a][bb][cc] = need ? ldv<CG>(zc + DIM * cn + c) : T(0);
      }
  unsigned m[NK];
  T zv[NK][DIM];
#pragma unroll
  for (int s = 0; s < NK; ++s) {
    if (s == 1 && !second) break;
    const long long node = i + (long long)gf.nnx * (j + (long long)gf.nny * (2 * q + s));
    m[s] = maskf[node];
#pragma unroll
    for (int c = 0; c < DIM; ++c) zv[s][c] = ldv<CG>(zf + DIM * node + c);
  }
#pragma unroll
  for (int s = 0; s < NK; ++s) {
    if (s == 1 && !second) break;
    const int k = DIM == 3 ? 2 * q + s : 0;
    const long long node = i + (long long)gf.nnx * (j + (long long)gf.nny * k);
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (!((m[s] >> c) & 1u)) zf[DIM * node + c] = prolong_one<DIM, T>(zv[s][c], cv[c], i, j, k);
  }
}

}  // namespace topo
