// Per-item bodies of the multigrid kernels below the finest grid (Algorithm
// 2): restriction with the coarse level's zero-guess smoothing,
// interpolation, the stored-level element operator (one warp per element)
// and its node gather, and one row of the coarsest-grid product.  The
// standalone kernels and the persistent coarse-cycle kernel both call them,
// so the two paths compute the same values in the same order.  The
// pointers carry no restrict qualifier: in the persistent kernel the same
// arrays are written in one phase and read in the next, so their loads must
// stay coherent ones (the kernels' own restrict-qualified parameters decide
// the cache path of the standalone launches).
#pragma once
#include "kernels.h"

namespace topo {

// b_c = Pm^T r_f at coarse node (I,J,K): the fine nodes around (2I,2J,2K)
// with weights prod(1 - |d|/2); fixed DOFs on either side contribute
// nothing.  When zc is not null, zc = omega * dinvc * b_c as well.
template <int DIM, typename T>
__device__ __forceinline__ void restrict_at(const GridP& gf, const uint8_t* maskf,
                                            const GridP& gc, const uint8_t* maskc,
                                            const T* rf, T* bc,
                                            const T* dinvc, T omega,
                                            T* zc, int I, int J, int K) {
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
        bool in = i >= 0 && i < gf.nnx && j >= 0 && j < gf.nny;
        if (DIM == 3) in = in && k >= 0 && k < gf.nnz;
        const T w = T((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
        const long long fn = i + (long long)gf.nnx * (j + (long long)gf.nny * (DIM == 3 ? k : 0));
        const unsigned m = in ? (unsigned)maskf[fn] : 7u;
#pragma unroll
        for (int c = 0; c < DIM; ++c)
          if (!((m >> c) & 1u)) acc[c] += w * rf[DIM * fn + c];
      }
  const long long node = I + (long long)gc.nnx * (J + (long long)gc.nny * K);
  const unsigned mc = maskc[node];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long d = DIM * node + c;
    const T bv = ((mc >> c) & 1u) ? T(0) : acc[c];
    bc[d] = bv;
    // the coarse level's pre-smoothing from a zero guess, z = omega D^-1 b
    if (zc) zc[d] = omega * dinvc[d] * bv;
  }
}

// z_f += Pm z_c at fine node (i,j,k): coarse nodes floor(i/2) .. ceil(i/2)
// per axis
template <int DIM, typename T>
__device__ __forceinline__ void prolong_at(const GridP& gf, const uint8_t* maskf,
                                           const GridP& gc, const T* zc,
                                           T* zf, int i, int j, int k) {
  const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
  const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (DIM == 3 && (k & 1)) ? 2 : 1;
  const T wx = (i & 1) ? T(0.5) : T(1), wy = (j & 1) ? T(0.5) : T(1),
          wz = (DIM == 3 && (k & 1)) ? T(0.5) : T(1);
  const T w = wx * wy * wz;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        if (a >= nk || bb >= nj || cc >= ni) continue;
        const long long cn = (i0 + cc) + (long long)gc.nnx * ((j0 + bb) + (long long)gc.nny * (k0 + a));
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += w * zc[DIM * cn + c];
      }
  const long long node = i + (long long)gf.nnx * (j + (long long)gf.nny * k);
  const unsigned m = maskf[node];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
    if (!((m >> c) & 1u)) zf[DIM * node + c] += acc[c];
}

// eo_e = K_e x_e for element e by one warp: the element's packed upper
// triangle is staged in the warp's shared slice tk (tri_len(ND) values,
// 16-byte aligned) with 16-byte loads, then lane r forms row r reading
// K(r, c) symmetrically with a running packed index.
template <int DIM, typename T>
__device__ __forceinline__ void gemv_elem(const GridP& g, const uint8_t* mask,
                                          const T* Kc, const T* x,
                                          T* eo, long long e, int lane, T* tk) {
  constexpr int ND = Geo<DIM>::ND, NT = tri_len(ND);
  constexpr int VW = 16 / sizeof(T);   // values per 16-byte load
  static_assert((NT * sizeof(T)) % 16 == 0, "packed triangle must be a multiple of 16 bytes");
  const int ex = (int)(e % g.nx);
  const long long rest = e / g.nx;
  const int ey = (int)(rest % g.ny);
  const int ez = DIM == 3 ? (int)(rest / g.ny) : 0;
  T xv = T(0);
  if (lane < ND) {
    const int a = lane / DIM, c = lane % DIM;
    const long long nd = (ex + (a & 1)) +
                         (long long)g.nnx * ((ey + ((a >> 1) & 1)) +
                                             (long long)g.nny * (DIM == 3 ? ez + ((a >> 2) & 1) : 0));
    xv = ((mask[nd] >> c) & 1u) ? T(0) : x[DIM * nd + c];
  }
  const T* src = Kc + (size_t)e * NT;
  for (int q = lane; q < NT / VW; q += 32) {
    if constexpr (sizeof(T) == 4)
      reinterpret_cast<float4*>(tk)[q] = __ldg(reinterpret_cast<const float4*>(src) + q);
    else
      reinterpret_cast<double2*>(tk)[q] = __ldg(reinterpret_cast<const double2*>(src) + q);
  }
  __syncwarp();
  // K(lane, c): tri_idx(c, lane) below the diagonal, whose step from c to
  // c + 1 is ND - 1 - c, then consecutive entries of row lane
  T acc = T(0);
  int idx = lane;
#pragma unroll
  for (int c = 0; c < ND; ++c) {
    const T xc = __shfl_sync(0xffffffffu, xv, c);
    if (lane < ND) acc = fma(tk[idx], xc, acc);
    idx += (c < lane) ? (ND - 1 - c) : 1;
  }
  if (lane < ND) eo[(size_t)e * ND + lane] = acc;
  __syncwarp();
}

// node (i,j,k) of a stored level: sum of the element rows of its elements
// in a fixed order, then the epilogue (K x, b - K x, or the damped Jacobi
// sweep); fixed DOFs take dfix * x
template <int DIM, typename T, int EPI>
__device__ __forceinline__ void gather_at(const GridP& g, const uint8_t* mask,
                                          const T* eo, const T* x,
                                          T* y, const T* b,
                                          const T* dinv, T omega, T dfix, int i,
                                          int j, int k) {
  constexpr int ND = Geo<DIM>::ND;
  constexpr int NZ = DIM == 3 ? 2 : 1;
  const long long node = i + (long long)g.nnx * (j + (long long)g.nny * k);
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int ez = 0; ez < NZ; ++ez)
#pragma unroll
    for (int ey = 0; ey < 2; ++ey)
#pragma unroll
      for (int ex = 0; ex < 2; ++ex) {
        const int ei = i - 1 + ex, ej = j - 1 + ey, ek = k - 1 + ez;
        bool in = ei >= 0 && ei < g.nx && ej >= 0 && ej < g.ny;
        if (DIM == 3) in = in && ek >= 0 && ek < g.nz;
        if (!in) continue;
        const long long e = ei + (long long)g.nx * (ej + (long long)g.ny * (DIM == 3 ? ek : 0));
        const int a = (1 - ex) + 2 * (1 - ey) + (DIM == 3 ? 4 * (1 - ez) : 0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += eo[(size_t)e * ND + DIM * a + c];
      }
  const unsigned m = mask[node];
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const long long d = DIM * node + c;
    const T Ax = ((m >> c) & 1u) ? dfix * x[d] : acc[c];
    if (EPI == EPI_APPLY)
      y[d] = Ax;
    else if (EPI == EPI_RESID)
      y[d] = b[d] - Ax;
    else
      y[d] = x[d] + omega * dinv[d] * (b[d] - Ax);
  }
}

// y[row] = A[row, :] x by one warp (strided lane sums, then a fixed
// shuffle tree)
template <typename T>
__device__ __forceinline__ void dense_row(int n, const T* A, const T* x,
                                          T* y, int row, int lane) {
  T s = T(0);
  for (int m = lane; m < n; m += 32) s += A[(size_t)row * n + m] * x[m];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

}  // namespace topo
