// Element-by-element stiffness operator K(E) x of Eq. 7 on a regular grid of
// unit Q4 / hex8 elements (matrix-free), and its diagonal.
//
// Design: owner-computes gather.  One thread owns one node; it loads the
// 3^DIM neighbourhood of nodal values once into registers and sums, over the
// 2^DIM elements around the node, the rows of (coef_e KE) or of the stored
// Galerkin matrix that belong to it.  No atomics, deterministic, and every
// nodal value / element coefficient is read from DRAM once per launch (the
// 27-fold reuse is served by L1/L2).  Boundary conditions are applied as
// M K M + dfix (I - M) with M the mask of free DOFs.
#include <type_traits>

#include "kernels.h"
#include "mg_device.cuh"

namespace topo {

template <int DIM, typename TC, typename TX, typename TY, int EPI, bool EXPL>
__global__ void __launch_bounds__(128)
    k_apply(GridP g, const uint8_t* __restrict__ mask, KEP<TC, Geo<DIM>::ND> ke,
            const TC* __restrict__ coef, const TC* __restrict__ Kc,
            const TX* __restrict__ x, TY* __restrict__ y, const TX* __restrict__ b,
            const TC* __restrict__ dinv, TC omega, TC dfix, Springs sp) {
  constexpr int ND = Geo<DIM>::ND;
  constexpr int NPE = Geo<DIM>::NPE;
  constexpr int NB = Geo<DIM>::NB;
  constexpr int NZ = DIM == 3 ? 2 : 1;
  using TE = typename std::conditional<(sizeof(TY) > sizeof(TC)), double, TC>::type;

  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nn) return;
  const int i = (int)(node % g.nnx);
  const long long rest = node / g.nnx;
  const int j = (int)(rest % g.nny);
  const int k = DIM == 3 ? (int)(rest / g.nny) : 0;

  TC xn[NB][DIM];
#pragma unroll
  for (int dz = 0; dz < (DIM == 3 ? 3 : 1); ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int s = dx + 3 * dy + 9 * dz;
        const int ii = i + dx - 1, jj = j + dy - 1, kk = k + dz - 1;
        bool in = ii >= 0 && ii < g.nnx && jj >= 0 && jj < g.nny;
        if (DIM == 3) in = in && kk >= 0 && kk < g.nnz;
        if (in) {
          const long long nb = ii + (long long)g.nnx * (jj + (long long)g.nny * (DIM == 3 ? kk : 0));
          const unsigned m = mask[nb];
#pragma unroll
          for (int c = 0; c < DIM; ++c) xn[s][c] = ((m >> c) & 1u) ? TC(0) : TC(x[DIM * nb + c]);
        } else {
#pragma unroll
          for (int c = 0; c < DIM; ++c) xn[s][c] = TC(0);
        }
      }

  TC acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = TC(0);

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
        const TC ce = EXPL ? TC(1) : coef[e];
#pragma unroll
        for (int ci = 0; ci < DIM; ++ci) {
          const int row = DIM * a + ci;
          TC s = TC(0);
#pragma unroll
          for (int bc = 0; bc < NPE; ++bc) {
            const int bx = bc & 1, by = (bc >> 1) & 1, bz = (bc >> 2) & 1;
            const int sidx = (ex + bx) + 3 * (ey + by) + (DIM == 3 ? 9 * (ez + bz) : 0);
#pragma unroll
            for (int cj = 0; cj < DIM; ++cj) {
              const int col = DIM * bc + cj;
              const TC kv = EXPL ? Kc[(size_t)e * tri_len(ND) + sym_idx(row, col, ND)]
                                 : ke.v[row * ND + col];
              s = fma(kv, xn[sidx][cj], s);
            }
          }
          acc[ci] = fma(ce, s, acc[ci]);
        }
      }

  const unsigned mself = mask[node];
#pragma unroll
  for (int ci = 0; ci < DIM; ++ci) {
    const long long d = DIM * node + ci;
    TE Ax = ((mself >> ci) & 1u) ? TE(dfix) * TE(x[d]) : TE(acc[ci]);
    if (!((mself >> ci) & 1u))
      for (int q = 0; q < sp.n; ++q)
        if (sp.dof[q] == d) Ax += TE(sp.k[q]) * TE(x[d]);
    if (EPI == EPI_APPLY) {
      y[d] = TY(Ax);
    } else if (EPI == EPI_RESID) {
      y[d] = TY(TE(b[d]) - Ax);
    } else {
      y[d] = TY(TE(x[d]) + TE(omega) * TE(dinv[d]) * (TE(b[d]) - Ax));
    }
  }
}

// ---------------------------------------------------------------------------
// Finest-grid hex8 operator, element-by-element with a Walsh-Hadamard
// factorisation of KE.
//
// KE commutes with the three coordinate reflections of the unit cube (which
// permute corners a -> a xor s and flip the reflected displacement
// component).  The Walsh-Hadamard transform over corners,
// X[t][c] = sum_a (-1)^{popcount(a & t)} x[a][c], therefore block-diagonalises
// KE: X[t][c] only couples to X[t'][c'] with t xor e_c == t' xor e_c', eight
// 3x3 blocks.  KE x = FWHT( B FWHT(x) ) with B (including the 1/64 of the
// two transforms) built on the host from KE, so one element costs
// 72 adds + 72 FMA + 72 adds instead of 576 FMA.
//
// Each thread owns one element column (ex, ey) and streams up in z, keeping
// the shared face's nodal values and partial forces in registers.  A block
// covers 16 x 8 element columns and owns the 15 x 7 nodes whose four
// surrounding columns it computes (owner-computes; one column of halo);
// per z-layer the four column partials of each owned node are summed in
// shared memory in a fixed order (deterministic, no atomics).
// ---------------------------------------------------------------------------
constexpr int WX = 16, WY = 8, WOX = WX - 1, WOY = WY - 1, WZC = 16;

// Level-1 Galerkin operator in the Walsh basis.  With 2x coarsening, the
// fine element at child position ch of a coarse element sees the nodal
// vector W_ch x (multilinear interpolation), so the coarse element operator is
// sum_ch E_ch W_ch^T KE W_ch = T (sum_ch E_ch M_ch^T B M_ch) T with
// M_ch = T W_ch T / 8.  M_ch is the tensor product over the axes of the 2x2
// factor [[1, +-1/2], [0, 1/2]] (Walsh index 0 = sum, 1 = difference; the
// sign is + for the lower child position and - for the upper), so it only
// couples X[t] with X[t'] for t a subset of t'.
__host__ __device__ constexpr float wmix(int ch, int t, int tp) {
  return ((t & 1) ? ((tp & 1) ? 0.5f : 0.0f) : ((tp & 1) ? ((ch & 1) ? -0.5f : 0.5f) : 1.0f)) *
         ((t & 2) ? ((tp & 2) ? 0.5f : 0.0f) : ((tp & 2) ? ((ch & 2) ? -0.5f : 0.5f) : 1.0f)) *
         ((t & 4) ? ((tp & 4) ? 0.5f : 0.0f) : ((tp & 4) ? ((ch & 4) ? -0.5f : 0.5f) : 1.0f));
}

// Row c of Walsh block tau times zt, skipping the block's structural zeros
// (27 of the 72 entries; their indices are compile-time after unrolling).
template <typename TC>
__device__ __forceinline__ TC wht_row(const WhtBlocks<TC>& kb, int tau, int c, const TC (&zt)[3]) {
  TC s = TC(0);
  bool first = true;
#pragma unroll
  for (int cp = 0; cp < 3; ++cp) {
    if (wht_zero(tau, c, cp)) continue;
    s = first ? kb.b[tau][c][cp] * zt[cp] : fma(kb.b[tau][c][cp], zt[cp], s);
    first = false;
  }
  return s;
}

// ye = element operator applied to the element's nodal values (bottom face
// xb = corners 0..3, top face xt = corners 4..7).  GAL1 = false: E_e KE; true:
// the level-1 Galerkin composite with the eight child moduli ce[].
template <typename TC, bool GAL1>
__device__ __forceinline__ void wht_element(const WhtBlocks<TC>& kb, const TC (&ce)[GAL1 ? 8 : 1],
                                            const TC (&xb)[4][3], const TC (&xt)[4][3],
                                            TC (&ye)[8][3]) {
  TC X[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      X[c][q] = xb[q][c];
      X[c][q + 4] = xt[q][c];
    }
    fwht8<TC>(X[c]);
  }
  TC Y[3][8];
  if (!GAL1) {
#pragma unroll
    for (int tau = 0; tau < 8; ++tau) {
      TC zt[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) zt[c] = ce[0] * X[c][tau ^ (1 << c)];
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[c][tau ^ (1 << c)] = wht_row(kb, tau, c, zt);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int t = 0; t < 8; ++t) Y[c][t] = TC(0);
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      TC Xf[3][8], Zf[3][8];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          TC s = TC(0);
#pragma unroll
          for (int tp = 0; tp < 8; ++tp)
            if ((t & ~tp) == 0) s = fma(TC(wmix(ch, t, tp)), X[c][tp], s);
          Xf[c][t] = s;
        }
#pragma unroll
      for (int tau = 0; tau < 8; ++tau) {
        TC zt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) zt[c] = ce[ch] * Xf[c][tau ^ (1 << c)];
#pragma unroll
        for (int c = 0; c < 3; ++c) Zf[c][tau ^ (1 << c)] = wht_row(kb, tau, c, zt);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int tp = 0; tp < 8; ++tp)
#pragma unroll
          for (int t = 0; t < 8; ++t)
            if ((t & ~tp) == 0) Y[c][tp] = fma(TC(wmix(ch, t, tp)), Zf[c][t], Y[c][tp]);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    fwht8<TC>(Y[c]);
#pragma unroll
    for (int a = 0; a < 8; ++a) ye[a][c] = Y[c][a];
  }
}

// ---------------------------------------------------------------------------
// Coarse levels with stored Galerkin element matrices are applied from their
// assembled stencil (StencilLayout in mg_device.cuh).
// ---------------------------------------------------------------------------
// one thread per (row, padded slot): the sum over the elements containing
// node n and its neighbour of the packed element matrix entry
// (DIM a_n + c, DIM a_m + c'), elements in a fixed order; padding slots are 0
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
    k_stencil_assemble(GridP g, const uint8_t* __restrict__ mask, const T* __restrict__ Kc,
                       T* __restrict__ S) {
  using SL = StencilLayout<DIM, T>;
  constexpr int ND = Geo<DIM>::ND, NSLOT = SL::NP * SL::GP * SL::W;
  const long long rows = DIM * g.nn;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * NSLOT) return;
  const int slot = (int)(t / rows);
  const long long r = t % rows;
  const int pz = slot / (SL::GP * SL::W), qq = slot % (SL::GP * SL::W);
  T s = T(0);
  if (qq < SL::NQP) {
    const long long n = r / DIM;
    const int c = (int)(r % DIM), cp = qq % DIM, o = qq / DIM;
    const int dx = o % 3 - 1, dy = o / 3 - 1, dz = DIM == 3 ? pz - 1 : 0;
    const int i = (int)(n % g.nnx), j = (int)((n / g.nnx) % g.nny);
    const int k = DIM == 3 ? (int)(n / ((long long)g.nnx * g.nny)) : 0;
    const int im = i + dx, jm = j + dy, km = k + dz;
    bool in = im >= 0 && im < g.nnx && jm >= 0 && jm < g.nny;
    if (DIM == 3) in = in && km >= 0 && km < g.nnz;
    if (in) {
      const long long m = im + (long long)g.nnx * (jm + (long long)g.nny * km);
      if ((mask[n] >> c) & 1u) {
        s = (m == n && cp == c) ? T(1) : T(0);     // fixed row: identity
      } else if (!((mask[m] >> cp) & 1u)) {        // fixed column: zero
        const int exlo = max(max(i, im) - 1, 0), exhi = min(min(i, im), g.nx - 1);
        const int eylo = max(max(j, jm) - 1, 0), eyhi = min(min(j, jm), g.ny - 1);
        const int ezlo = DIM == 3 ? max(max(k, km) - 1, 0) : 0;
        const int ezhi = DIM == 3 ? min(min(k, km), g.nz - 1) : 0;
        for (int ez = ezlo; ez <= ezhi; ++ez)
          for (int ey = eylo; ey <= eyhi; ++ey)
            for (int ex = exlo; ex <= exhi; ++ex) {
              const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
              const int ar = (i - ex) + 2 * (j - ey) + (DIM == 3 ? 4 * (k - ez) : 0);
              const int ac = (im - ex) + 2 * (jm - ey) + (DIM == 3 ? 4 * (km - ez) : 0);
              s += Kc[(size_t)e * tri_len(ND) + sym_idx(DIM * ar + c, DIM * ac + cp, ND)];
            }
      }
    }
  }
  S[SL::index(rows, r, pz, qq)] = s;
}

// y = S x with the epilogue (K x, b - K x, or the damped Jacobi sweep); one
// thread per row (body in mg_device.cuh).
template <int DIM, typename T, int EPI>
__global__ void __launch_bounds__(256, 2)
    k_stencil_apply(GridP g, const T* __restrict__ S, const T* __restrict__ x, T* __restrict__ y,
                    const T* __restrict__ b, const T* __restrict__ dinv, T omega) {
  const long long rows = DIM * g.nn;
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  if (r >= rows) return;
  stencil_row<DIM, T, EPI, false>(g, S, x, y, b, dinv, omega, r);
  pdl_launch_dependents();
}

template <int DIM, typename T, int EPI>
static cudaError_t run_stencil(const ApplyArgs& a, cudaStream_t s) {
  const long long rows = DIM * a.g.nn;
  return launch_pdl(k_stencil_apply<DIM, T, EPI>, dim3(nblocks(rows, 256)), dim3(256), 0, s, a.g,
                    static_cast<const T*>(a.S), static_cast<const T*>(a.x), static_cast<T*>(a.y),
                    static_cast<const T*>(a.b), static_cast<const T*>(a.dinv), T(a.omega));
}

template <int DIM, typename T>
static cudaError_t run_stencil_epi(const ApplyArgs& a, cudaStream_t s) {
  switch (a.epi) {
    case EPI_APPLY: return run_stencil<DIM, T, EPI_APPLY>(a, s);
    case EPI_RESID: return run_stencil<DIM, T, EPI_RESID>(a, s);
    default: return run_stencil<DIM, T, EPI_SMOOTH>(a, s);
  }
}

// the assembled form carries the identity rows of fixed DOFs, so only
// dfix = 1 is representable
static cudaError_t run_expl_any(const ApplyArgs& a, cudaStream_t s) {
  if (a.tx != a.tc || a.ty != a.tc || a.S == nullptr || a.dfix != 1.0) return cudaErrorInvalidValue;
  if (a.dim == 2)
    return a.tc == T_F64 ? run_stencil_epi<2, double>(a, s) : run_stencil_epi<2, float>(a, s);
  return a.tc == T_F64 ? run_stencil_epi<3, double>(a, s) : run_stencil_epi<3, float>(a, s);
}

template <int DIM, typename T>
static cudaError_t stencil_t(const GridP& g, const uint8_t* mask, const void* Kc, void* S,
                             cudaStream_t s) {
  const long long tot = StencilLayout<DIM, T>::values((long long)DIM * g.nn);
  k_stencil_assemble<DIM, T><<<nblocks(tot, 256), 256, 0, s>>>(g, mask, (const T*)Kc, (T*)S);
  return cudaGetLastError();
}

cudaError_t launch_stencil_assemble(int dim, int t, const GridP& g, const uint8_t* mask,
                                    const void* Kc, void* S, cudaStream_t s) {
  if (dim == 2) return t == T_F64 ? stencil_t<2, double>(g, mask, Kc, S, s)
                                  : stencil_t<2, float>(g, mask, Kc, S, s);
  return t == T_F64 ? stencil_t<3, double>(g, mask, Kc, S, s) : stencil_t<3, float>(g, mask, Kc, S, s);
}

long long stencil_values(int dim, int t, const GridP& g) {
  const long long rows = (long long)dim * g.nn;
  if (dim == 2)
    return t == T_F64 ? StencilLayout<2, double>::values(rows) : StencilLayout<2, float>::values(rows);
  return t == T_F64 ? StencilLayout<3, double>::values(rows) : StencilLayout<3, float>::values(rows);
}

// Element operator of the column-streaming kernel
enum { OPK_FINE = 0, OPK_GAL1 = 1 };

template <typename TC, typename TX, typename TY, int EPI, int OP>
__global__ void __launch_bounds__(WX * WY, (OP == OPK_GAL1 && sizeof(TC) == 4) ? 4 : 1)
    k_apply3_col(GridP g, GridP gf, const uint8_t* __restrict__ mask, WhtBlocks<TC> kb,
                 const TC* __restrict__ coef, int zc, const TX* __restrict__ x,
                 TY* __restrict__ y, const TX* __restrict__ b, const TC* __restrict__ dinv,
                 TC omega, TC dfix, bool clean) {
  // clean: x is zero on every fixed DOF, so the input masks are not loaded
  // (the fixed rows' outputs are still set from the node masks)
  using TE = typename std::conditional<(sizeof(TY) > sizeof(TC)), double, TC>::type;
  constexpr bool GAL1 = OP == OPK_GAL1;
  __shared__ TC part[2][4][WY][WX][3];
  pdl_wait();
  const int tx = threadIdx.x % WX, ty = threadIdx.x / WX;
  const int x0 = blockIdx.x * WOX, y0 = blockIdx.y * WOY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nnz);
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const bool col_ok = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
  const long long plane = (long long)g.nnx * g.nny;

  // nodal values of the current bottom face (corners 0..3) and top face
  TC xb[4][3], xt[4][3];
  TC acc[4][3];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[q][c] = TC(0);

  // Face loads are software-pipelined: the raw values and masks of the next
  // top face are requested before the current element is computed, so their
  // latency overlaps the arithmetic.
  TX raw[4][3];
  unsigned rmask = 0u;   // 3 bits per corner; all set = out of range
  auto issue_face = [&](int kz) {
    rmask = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ex + (q & 1), j = ey + (q >> 1);
      if (col_ok && kz >= 0 && kz < g.nnz) {
        const long long nd = i + (long long)g.nnx * j + plane * kz;
        if (!clean) rmask |= ((unsigned)mask[nd] & 7u) << (3 * q);
#pragma unroll
        for (int c = 0; c < 3; ++c) raw[q][c] = x[3 * nd + c];
      } else {
        rmask |= 7u << (3 * q);
#pragma unroll
        for (int c = 0; c < 3; ++c) raw[q][c] = TX(0);
      }
    }
  };
  auto consume_face = [&](TC (&f)[4][3]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) f[q][c] = ((rmask >> (3 * q + c)) & 1u) ? TC(0) : TC(raw[q][c]);
  };

  issue_face(z0 - 1);
  consume_face(xb);
  issue_face(z0);
  const bool own = tx < WOX && ty < WOY && (x0 + tx) < g.nnx && (y0 + ty) < g.nny;
  int buf = 0;
  for (int ez = z0 - 1; ez < z1; ++ez) {
    consume_face(xt);
    if (ez + 2 <= z1) issue_face(ez + 2);
    TC ye[8][3];
    const bool el_ok = col_ok && ez >= 0 && ez < g.nz;
    if (el_ok) {
      TC ce[GAL1 ? 8 : 1];
      if (!GAL1) {
        ce[0] = coef[ex + (long long)g.nx * (ey + (long long)g.ny * ez)];
      } else {
#pragma unroll
        for (int ch = 0; ch < (GAL1 ? 8 : 1); ++ch)
          ce[ch] = coef[(2 * ex + (ch & 1)) +
                        (long long)gf.nx * ((2 * ey + ((ch >> 1) & 1)) +
                                            (long long)gf.ny * (2 * ez + ((ch >> 2) & 1)))];
      }
      wht_element<TC, GAL1>(kb, ce, xb, xt, ye);
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) ye[a][c] = TC(0);
    }
    // bottom face of this element completes this column's share of layer ez
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        part[buf][q][ty][tx][c] = acc[q][c] + ye[q][c];
        acc[q][c] = ye[q + 4][c];
        xb[q][c] = xt[q][c];
      }
    __syncthreads();
    if (own && ez >= z0) {
      // node (x0+tx, y0+ty, ez): corner 3 of column (tx,ty), corner 2 of
      // (tx+1,ty), corner 1 of (tx,ty+1), corner 0 of (tx+1,ty+1)
      const long long nd = (x0 + tx) + (long long)g.nnx * (y0 + ty) + plane * ez;
      const unsigned m = mask[nd];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const TC s = ((part[buf][3][ty][tx][c] + part[buf][2][ty][tx + 1][c]) +
                      part[buf][1][ty + 1][tx][c]) + part[buf][0][ty + 1][tx + 1][c];
        const long long d = 3 * nd + c;
        const TE Ax = ((m >> c) & 1u) ? TE(dfix) * TE(x[d]) : TE(s);
        if (EPI == EPI_APPLY) {
          y[d] = TY(Ax);
        } else if (EPI == EPI_RESID) {
          y[d] = TY(TE(b[d]) - Ax);
        } else {
          y[d] = TY(TE(x[d]) + TE(omega) * TE(dinv[d]) * (TE(b[d]) - Ax));
        }
      }
    }
    buf ^= 1;
  }
  pdl_launch_dependents();
}

template <int DIM, typename TC, bool EXPL>
__global__ void __launch_bounds__(256)
    k_diag(GridP g, const uint8_t* __restrict__ mask, KEP<TC, Geo<DIM>::ND> ke,
           const TC* __restrict__ coef, const TC* __restrict__ Kc, TC* __restrict__ dinv,
           Springs sp) {
  constexpr int ND = Geo<DIM>::ND;
  constexpr int NZ = DIM == 3 ? 2 : 1;
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nn) return;
  const int i = (int)(node % g.nnx);
  const long long rest = node / g.nnx;
  const int j = (int)(rest % g.nny);
  const int k = DIM == 3 ? (int)(rest / g.nny) : 0;
  TC d[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) d[c] = TC(0);
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
        for (int c = 0; c < DIM; ++c) {
          const int row = DIM * a + c;
          d[c] += EXPL ? Kc[(size_t)e * tri_len(ND) + tri_idx(row, row, ND)]
                       : coef[e] * ke.v[row * ND + row];
        }
      }
  for (int q = 0; q < sp.n; ++q)
#pragma unroll
    for (int c = 0; c < DIM; ++c)
      if (sp.dof[q] == DIM * node + c) d[c] += TC(sp.k[q]);
  const unsigned m = mask[node];
#pragma unroll
  for (int c = 0; c < DIM; ++c)
    dinv[DIM * node + c] = ((m >> c) & 1u) ? TC(1) : TC(1) / d[c];
}

// ---------------------------------------------------------------------------
// Host dispatch
// ---------------------------------------------------------------------------
template <int DIM, typename TC, typename TX, typename TY, int EPI, bool EXPL>
static cudaError_t run_apply(const ApplyArgs& a, cudaStream_t s) {
  constexpr int ND = Geo<DIM>::ND;
  KEP<TC, ND> ke;
  if (!EXPL) {
    const TC* src = static_cast<const TC*>(a.ke);
    for (int q = 0; q < ND * ND; ++q) ke.v[q] = src[q];
  } else {
    for (int q = 0; q < ND * ND; ++q) ke.v[q] = TC(0);
  }
  const int th = 128;
  k_apply<DIM, TC, TX, TY, EPI, EXPL><<<nblocks(a.g.nn, th), th, 0, s>>>(
      a.g, a.mask, ke, static_cast<const TC*>(a.coef), static_cast<const TC*>(a.Kc),
      static_cast<const TX*>(a.x), static_cast<TY*>(a.y), static_cast<const TX*>(a.b),
      static_cast<const TC*>(a.dinv), TC(a.omega), TC(a.dfix), a.springs);
  return cudaGetLastError();
}

template <int DIM, typename TC, typename TX, typename TY, bool EXPL>
static cudaError_t run_apply_epi(const ApplyArgs& a, cudaStream_t s) {
  switch (a.epi) {
    case EPI_APPLY: return run_apply<DIM, TC, TX, TY, EPI_APPLY, EXPL>(a, s);
    case EPI_RESID: return run_apply<DIM, TC, TX, TY, EPI_RESID, EXPL>(a, s);
    default: return run_apply<DIM, TC, TX, TY, EPI_SMOOTH, EXPL>(a, s);
  }
}

// node-centric gather kernel: finest grid in 2D (and 3D without Walsh blocks)
template <int DIM>
static cudaError_t run_apply_dim(const ApplyArgs& a, cudaStream_t s) {
  if (a.expl) return cudaErrorInvalidValue;
  if (a.tc == T_F64) {
    if (a.tx != T_F64 || a.ty != T_F64) return cudaErrorInvalidValue;
    return run_apply_epi<DIM, double, double, double, false>(a, s);
  }
  if (a.tx == T_F64 && a.ty == T_F64) return run_apply_epi<DIM, float, double, double, false>(a, s);
  if (a.tx == T_F32 && a.ty == T_F32) return run_apply_epi<DIM, float, float, float, false>(a, s);
  if (a.tx == T_F32 && a.ty == T_F64) return run_apply_epi<DIM, float, float, double, false>(a, s);
  return cudaErrorInvalidValue;
}

// resident blocks of the float32 level-1 Galerkin column kernel (cached per
// device; queried at set-up, outside any stream capture)
template <int EPI>
static long long gal1_slots() {
  static long long cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cache[dev] > 0) return cache[dev];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &per_sm, k_apply3_col<float, float, float, EPI, OPK_GAL1>, WX * WY, 0) != cudaSuccess ||
      sms <= 0 || per_sm <= 0)
    return 0;
  cache[dev] = (long long)sms * per_sm;
  return cache[dev];
}

void col_prepare() {
  gal1_slots<EPI_APPLY>();
  gal1_slots<EPI_RESID>();
  gal1_slots<EPI_SMOOTH>();
}

template <typename TC, typename TX, typename TY, int EPI, int OP>
static cudaError_t run_col(const ApplyArgs& a, cudaStream_t s) {
  WhtBlocks<TC> kb;
  const TC* src = static_cast<const TC*>(a.wht);
  for (int q = 0; q < 72; ++q) (&kb.b[0][0][0])[q] = src ? src[q] : TC(0);
  const int gx = (a.g.nnx + WOX - 1) / WOX, gy = (a.g.nny + WOY - 1) / WOY;
  // z-chunk: the standard 16 layers, shortened on small grids so that the
  // launch still covers the GPU (each chunk recomputes one element layer)
  int zc = WZC;
  while (zc > 2 && (long long)gx * gy * ((a.g.nnz + zc - 1) / zc) < 2 * 152) zc /= 2;
  // level-1 Galerkin operator (latency-bound, one block per column chunk):
  // the chunk length minimising waves x (layers + 1 recomputed)
  const long long slots =
      (OP == OPK_GAL1 && sizeof(TC) == 4 && sizeof(TX) == 4 && sizeof(TY) == 4) ? gal1_slots<EPI>() : 0;
  if (slots > 0) {
    long long best = -1;
    for (int c = 2; c <= WZC; ++c) {
      const long long blocks = (long long)gx * gy * ((a.g.nnz + c - 1) / c);
      const long long cost = ((blocks + slots - 1) / slots) * (c + 1);
      if (best < 0 || cost < best || (cost == best && c > zc)) {
        best = cost;
        zc = c;
      }
    }
  }
  if (a.zsplit > 0) zc = min(a.zsplit, (int)a.g.nnz);   // chosen by the autotuner
  dim3 grid(gx, gy, (a.g.nnz + zc - 1) / zc);
  return launch_pdl(k_apply3_col<TC, TX, TY, EPI, OP>, grid, dim3(WX * WY), 0, s, a.g, a.gf, a.mask,
                    kb, static_cast<const TC*>(a.coef), zc, static_cast<const TX*>(a.x),
                    static_cast<TY*>(a.y), static_cast<const TX*>(a.b),
                    static_cast<const TC*>(a.dinv), TC(a.omega), TC(a.dfix), a.clean_inputs);
}

template <typename TC, typename TX, typename TY, int OP>
static cudaError_t run_col_epi(const ApplyArgs& a, cudaStream_t s) {
  switch (a.epi) {
    case EPI_APPLY: return run_col<TC, TX, TY, EPI_APPLY, OP>(a, s);
    case EPI_RESID: return run_col<TC, TX, TY, EPI_RESID, OP>(a, s);
    default: return run_col<TC, TX, TY, EPI_SMOOTH, OP>(a, s);
  }
}

template <int OP>
static cudaError_t run_col_types(const ApplyArgs& a, cudaStream_t s) {
  if (a.tc == T_F64) {
    if (a.tx != T_F64 || a.ty != T_F64) return cudaErrorInvalidValue;
    return run_col_epi<double, double, double, OP>(a, s);
  }
  if (a.tx == T_F32 && a.ty == T_F32) return run_col_epi<float, float, float, OP>(a, s);
  if (OP == OPK_FINE) {
    if (a.tx == T_F64 && a.ty == T_F64) return run_col_epi<float, double, double, OPK_FINE>(a, s);
    if (a.tx == T_F32 && a.ty == T_F64) return run_col_epi<float, float, double, OPK_FINE>(a, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_apply(const ApplyArgs& a, cudaStream_t s) {
  if (a.g.nn <= 0) return cudaSuccess;
  if (a.tc == T_DF) return launch_apply_df(a, s);
  if (a.expl) return run_expl_any(a, s);
  if (a.dim == 3) {
    if (a.gal1) return run_col_types<OPK_GAL1>(a, s);
    if (a.use_tc && tc_apply_ok(a)) return launch_apply_tc(a, s);
    if (pair_apply_ok(a)) return launch_apply_pair(a, s);
    if (a.wht != nullptr) return run_col_types<OPK_FINE>(a, s);
  }
  return a.dim == 2 ? run_apply_dim<2>(a, s) : run_apply_dim<3>(a, s);
}

void wht_blocks(const double* KE, double* out64) {
  // B = T KE T / 64 with T[(t,c),(a,c)] = (-1)^{popcount(a & t)}, restricted
  // to the eight 3x3 blocks of characters tau = t xor e_c.
  auto sgn = [](int a, int t) { return (__builtin_popcount(a & t) & 1) ? -1.0 : 1.0; };
  for (int tau = 0; tau < 8; ++tau)
    for (int c = 0; c < 3; ++c)
      for (int cp = 0; cp < 3; ++cp) {
        const int t = tau ^ (1 << c), tp = tau ^ (1 << cp);
        double s = 0.0;
        for (int a = 0; a < 8; ++a)
          for (int ap = 0; ap < 8; ++ap) s += sgn(a, t) * KE[(3 * a + c) * 24 + 3 * ap + cp] * sgn(ap, tp);
        s /= 64.0;
        out64[(tau * 3 + c) * 3 + cp] = s;
      }
}

void wht_blocks_pin_zeros(double* w64, float* w32) {
  for (int tau = 0; tau < 8; ++tau)
    for (int c = 0; c < 3; ++c)
      for (int cp = 0; cp < 3; ++cp) {
        const int q = (tau * 3 + c) * 3 + cp;
        if (wht_zero(tau, c, cp)) w64[q] = 0.0;
        w32[q] = (float)w64[q];
      }
}

template <int DIM, typename TC, bool EXPL>
static cudaError_t run_diag(const GridP& g, const uint8_t* mask, const void* coef,
                            const void* Kc, const void* kev, void* dinv, cudaStream_t s,
                            const Springs& sp) {
  constexpr int ND = Geo<DIM>::ND;
  KEP<TC, ND> ke;
  for (int q = 0; q < ND * ND; ++q) ke.v[q] = EXPL ? TC(0) : static_cast<const TC*>(kev)[q];
  k_diag<DIM, TC, EXPL><<<nblocks(g.nn, 256), 256, 0, s>>>(
      g, mask, ke, static_cast<const TC*>(coef), static_cast<const TC*>(Kc),
      static_cast<TC*>(dinv), sp);
  return cudaGetLastError();
}

cudaError_t launch_diag(int dim, const GridP& g, const uint8_t* mask, int tc, bool expl,
                        const void* coef, const void* Kc, const void* ke, void* dinv,
                        cudaStream_t s, const Springs& sp) {
  if (g.nn <= 0) return cudaSuccess;
  if (dim == 2) {
    if (tc == T_F64) return expl ? run_diag<2, double, true>(g, mask, coef, Kc, ke, dinv, s, sp)
                                 : run_diag<2, double, false>(g, mask, coef, Kc, ke, dinv, s, sp);
    return expl ? run_diag<2, float, true>(g, mask, coef, Kc, ke, dinv, s, sp)
                : run_diag<2, float, false>(g, mask, coef, Kc, ke, dinv, s, sp);
  }
  if (tc == T_F64) return expl ? run_diag<3, double, true>(g, mask, coef, Kc, ke, dinv, s, sp)
                               : run_diag<3, double, false>(g, mask, coef, Kc, ke, dinv, s, sp);
  return expl ? run_diag<3, float, true>(g, mask, coef, Kc, ke, dinv, s, sp)
              : run_diag<3, float, false>(g, mask, coef, Kc, ke, dinv, s, sp);
}

}  // namespace topo
