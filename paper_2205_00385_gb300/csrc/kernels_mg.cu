// Multigrid pieces of Algorithm 2: restriction P^T, interpolation P, Jacobi
// smoothing from a zero guess, the Galerkin coarse operators P^T K P as
// per-coarse-element matrices, and the exact coarsest-grid solve.
//
// With 2x coarsening and multilinear P, the fine elements inside one coarse
// element interpolate only from that coarse element's nodes, so P^T K P is
// again element-by-element on the coarse grid with element matrices
//   Kc_E = sum_children P_c^T Ke_child P_c,
// where P_c = W_c (x) I_dim and W_c[a][A] is the product over axes of the
// linear weights of fine corner a of child c at coarse corner A.
#include <math.h>

#include "dfmath.cuh"
#include "kernels.h"
#include "mg_device.cuh"

namespace topo {

// ---------------------------------------------------------------------------
// Restriction and interpolation.  Each value sums its terms in the order of
// restrict_finish / prolong_one (mg_device.cuh), whose per-node bodies the
// fused coarse V-cycle runs, so the bits are the same.  The restriction
// runs one thread per coarse value: consecutive threads take consecutive
// values of one coarse plane (its rows flattened), so a warp's fine loads
// span few sectors and a thread holds only its 27 terms (more threads in
// flight than one per node, which pays on the small levels).
// ---------------------------------------------------------------------------
constexpr int TVAL = 256;

// CLEAN: r_f is +-0 on every fixed DOF, so the fine masks are not loaded: a
// fixed term then adds w * (+-0) where restrict_finish adds +0, and a
// running sum that starts at +0 is never -0, so the bits are the same.
template <int DIM, typename T, bool CLEAN>
__global__ void __launch_bounds__(TVAL)
    k_restrict(GridP gf, const uint8_t* __restrict__ maskf, GridP gc,
               const uint8_t* __restrict__ maskc, const T* __restrict__ rf, T* __restrict__ bc,
               const T* __restrict__ dinvc, T omega, T* __restrict__ zc) {
  constexpr int NZ = DIM == 3 ? 3 : 1;
  const int rowv = DIM * gc.nnx;
  const int pv = blockIdx.x * TVAL + threadIdx.x;
  const int K = DIM == 3 ? (int)blockIdx.y : 0;
  pdl_wait();
  if (pv >= rowv * gc.nny) return;
  const int J = pv / rowv, v = pv - J * rowv;
  const int I = v / DIM, c = v - I * DIM;
  unsigned m[NZ][3][3];
  T x[NZ][3][3];
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
        m[a][b][q] = CLEAN ? 0u : (unsigned)maskf[fn];
        x[a][b][q] = rf[DIM * fn + c];
      }
  T acc = T(0);
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
        acc = add_rn(acc, ((mm >> c) & 1u) ? T(0) : mul_rn(w, x[a][b][q]));
      }
  const long long node = I + (long long)gc.nnx * (J + (long long)gc.nny * K);
  const long long d = DIM * node + c;
  const T bv = ((maskc[node] >> c) & 1u) ? T(0) : acc;
  bc[d] = bv;
  if (zc) zc[d] = mul_rn(mul_rn(omega, dinvc[d]), bv);
  pdl_launch_dependents();
}

// z_f += Pm z_c: threads on the fine (i, j) grid, each taking the fine nodes
// k = 2q and 2q+1 (3D), which share the coarse plane q (index work shared by
// six values; one thread per value measured 2.5x slower at the finest level).
constexpr int TBX = 32, TBY = 4;

template <typename T>
__host__ __device__ constexpr int transfer_min_blocks() {
  return sizeof(T) == 4 ? 4 : 2;   // registers for all loads in flight
}

template <int DIM, typename T>
__global__ void __launch_bounds__(TBX * TBY, transfer_min_blocks<T>())
    k_prolong_add(GridP gf, const uint8_t* __restrict__ maskf, GridP gc,
                  const T* __restrict__ zc, T* __restrict__ zf) {
  const int i = blockIdx.x * TBX + threadIdx.x, j = blockIdx.y * TBY + threadIdx.y;
  const int q = DIM == 3 ? (int)blockIdx.z : 0;
  pdl_wait();
  if (i >= gf.nnx || j >= gf.nny) return;
  prolong_pair<DIM, T, false>(gf, maskf, gc, zc, zf, i, j, q);
  pdl_launch_dependents();
}

template <typename T, typename TIN>
__global__ void __launch_bounds__(256)
    k_presmooth(long long n, const TIN* __restrict__ bin, T* __restrict__ bout,
                const T* __restrict__ dinv, T omega, T* __restrict__ z) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  pdl_wait();
  if (q >= n) return;
  const T bv = cvt<T>(bin[q]);
  if (bout) bout[q] = bv;
  z[q] = omega * dinv[q] * bv;
  pdl_launch_dependents();
}

template <typename TIN, typename TOUT>
__global__ void __launch_bounds__(256)
    k_convert(long long n, const TIN* __restrict__ in, TOUT* __restrict__ out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = cvt<TOUT>(in[q]);
}

// ---------------------------------------------------------------------------
// Galerkin level 1 from the finest grid: Kc_E = sum_c coef_child(E,c) Q_c,
// Q_c = P_c^T KE P_c (precomputed).  One thread per (entry, coarse element).
// ---------------------------------------------------------------------------
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
    k_galerkin_fine(GridP gc, GridP gf, const T* __restrict__ coef, const T* __restrict__ Qc,
                    T* __restrict__ Kc) {
  constexpr int ND = Geo<DIM>::ND, NPE = Geo<DIM>::NPE, NT = tri_len(ND);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= gc.nel * NT) return;
  const long long E = t / NT;
  const int pk = (int)(t % NT);
  int r, cc;
  tri_rc(pk, ND, r, cc);
  const int entry = r * ND + cc;
  const int EX = (int)(E % gc.nx);
  const long long rest = E / gc.nx;
  const int EY = (int)(rest % gc.ny);
  const int EZ = DIM == 3 ? (int)(rest / gc.ny) : 0;
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < NPE; ++c) {
    const int fx = 2 * EX + (c & 1), fy = 2 * EY + ((c >> 1) & 1), fz = 2 * EZ + ((c >> 2) & 1);
    const long long fe = fx + (long long)gf.nx * (fy + (long long)gf.ny * (DIM == 3 ? fz : 0));
    acc += coef[fe] * Qc[c * ND * ND + entry];
  }
  Kc[(size_t)E * NT + pk] = acc;
}

// Level-1 diagonal without stored matrices (3D): node I of level 1 sums, over
// its coarse elements E and their children ch, E_child * diag(Q_ch) at I's
// corner a.  qd.v[(ch * 8 + a) * 3 + c] = Q_ch[(3a+c),(3a+c)].
template <typename T>
struct QDiagP {
  T v[8 * 8 * 3];
};

template <typename T>
__global__ void __launch_bounds__(256)
    k_diag_l1(GridP g1, GridP gf, const uint8_t* __restrict__ mask, QDiagP<T> qd,
              const T* __restrict__ coef, T* __restrict__ dinv) {
  const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g1.nn) return;
  const int i = (int)(node % g1.nnx);
  const long long rest = node / g1.nnx;
  const int j = (int)(rest % g1.nny);
  const int k = (int)(rest / g1.nny);
  T d[3] = {T(0), T(0), T(0)};
  for (int ez = 0; ez < 2; ++ez)
    for (int ey = 0; ey < 2; ++ey)
      for (int ex = 0; ex < 2; ++ex) {
        const int EX = i - 1 + ex, EY = j - 1 + ey, EZ = k - 1 + ez;
        if (EX < 0 || EX >= g1.nx || EY < 0 || EY >= g1.ny || EZ < 0 || EZ >= g1.nz) continue;
        const int a = (1 - ex) + 2 * (1 - ey) + 4 * (1 - ez);
#pragma unroll
        for (int ch = 0; ch < 8; ++ch) {
          const long long fe = (2 * EX + (ch & 1)) +
                               (long long)gf.nx * ((2 * EY + ((ch >> 1) & 1)) +
                                                   (long long)gf.ny * (2 * EZ + ((ch >> 2) & 1)));
          const T e = coef[fe];
#pragma unroll
          for (int c = 0; c < 3; ++c) d[c] += e * qd.v[(ch * 8 + a) * 3 + c];
        }
      }
  const unsigned m = mask[node];
#pragma unroll
  for (int c = 0; c < 3; ++c) dinv[3 * node + c] = ((m >> c) & 1u) ? T(1) : T(1) / d[c];
}

// Level-2 element matrices straight from the finest moduli (3D): a level-2
// element covers 4x4x4 finest elements f, and
// Kc_E = sum_f E_f R_f with R_f = W_c1^T (W_c0^T KE W_c0) W_c1 for the
// finest element's position c0 inside its level-1 parent and that parent's
// position c1 inside E (64 precomputed tables, R[f * 576 + entry]).
template <typename T>
__global__ void __launch_bounds__(256)
    k_galerkin_l2(GridP g2, GridP gf, const T* __restrict__ coef, const T* __restrict__ R,
                  T* __restrict__ Kc) {
  constexpr int NT = tri_len(24);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g2.nel * NT) return;
  const long long E = t / NT;
  const int pk = (int)(t % NT);
  int r, cc;
  tri_rc(pk, 24, r, cc);
  const int entry = r * 24 + cc;
  const int EX = (int)(E % g2.nx);
  const long long rest = E / g2.nx;
  const int EY = (int)(rest % g2.ny);
  const int EZ = (int)(rest / g2.ny);
  T acc = T(0);
#pragma unroll 8
  for (int f = 0; f < 64; ++f) {
    const int c1 = f >> 3, c0 = f & 7;
    const int fx = 4 * EX + 2 * (c1 & 1) + (c0 & 1);
    const int fy = 4 * EY + 2 * ((c1 >> 1) & 1) + ((c0 >> 1) & 1);
    const int fz = 4 * EZ + 2 * ((c1 >> 2) & 1) + ((c0 >> 2) & 1);
    acc += coef[fx + (long long)gf.nx * (fy + (long long)gf.ny * fz)] * R[f * 576 + entry];
  }
  Kc[(size_t)E * NT + pk] = acc;
}

// Galerkin level l+1 from stored level-l element matrices.  One block of
// ND*ND threads per coarse element; T = Kchild W in shared memory, then
// Kc += W^T T, summed over the 2^DIM children.  W_c[a][A], the weight of
// coarse corner A at fine corner a of child c, is the product over the axes
// of the linear weights (c + a) / 2 (A's bit set) or (2 - c - a) / 2 (per
// axis bits, positions in half coarse-element units); it is staged in shared
// memory from integer arithmetic, an integer over 2^DIM, exact in any
// floating type.
template <int DIM, typename T>
__global__ void __launch_bounds__(Geo<DIM>::ND * Geo<DIM>::ND)
    k_galerkin_coarse(GridP gc, GridP gf, const T* __restrict__ Kf, T* __restrict__ Kc) {
  constexpr int ND = Geo<DIM>::ND, NPE = Geo<DIM>::NPE, NT = tri_len(ND);
  __shared__ T sK[ND * ND];
  __shared__ T sT[ND * ND];
  __shared__ T sW[NPE * NPE * NPE];   // [child][fine corner][coarse corner]
  const long long E = blockIdx.x;
  const int tid = threadIdx.x;
  for (int q = tid; q < NPE * NPE * NPE; q += ND * ND) {
    const int c = q / (NPE * NPE), a = (q / NPE) % NPE, A = q % NPE;
    int num = 1;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int p = ((c >> d) & 1) + ((a >> d) & 1);
      num *= ((A >> d) & 1) ? p : 2 - p;
    }
    sW[q] = T(num) / T(1 << DIM);
  }
  __syncthreads();
  const int EX = (int)(E % gc.nx);
  const long long rest = E / gc.nx;
  const int EY = (int)(rest % gc.ny);
  const int EZ = DIM == 3 ? (int)(rest / gc.ny) : 0;
  const int I = tid / ND, J = tid % ND;
  const int AI = I / DIM, ci = I % DIM, AJ = J / DIM, cj = J % DIM;
  T acc = T(0);
  for (int c = 0; c < NPE; ++c) {
    const int fx = 2 * EX + (c & 1), fy = 2 * EY + ((c >> 1) & 1), fz = 2 * EZ + ((c >> 2) & 1);
    const long long fe = fx + (long long)gf.nx * (fy + (long long)gf.ny * (DIM == 3 ? fz : 0));
    sK[tid] = Kf[(size_t)fe * NT + sym_idx(I, J, ND)];
    __syncthreads();
    // T[i][J] = sum_b K[i][(b, cj)] W_c[b][AJ]   (i = I here)
    T tv = T(0);
#pragma unroll
    for (int bcn = 0; bcn < NPE; ++bcn) tv += sK[I * ND + DIM * bcn + cj] * sW[(c * NPE + bcn) * NPE + AJ];
    sT[tid] = tv;
    __syncthreads();
    // acc[I][J] += sum_a W_c[a][AI] T[(a, ci)][J]
#pragma unroll
    for (int acn = 0; acn < NPE; ++acn) acc += sW[(c * NPE + acn) * NPE + AI] * sT[(DIM * acn + ci) * ND + J];
    __syncthreads();
  }
  if (J >= I) Kc[(size_t)E * NT + tri_idx(I, J, ND)] = acc;
}

// ---------------------------------------------------------------------------
// Coarsest grid: dense matrix with identity rows/columns at fixed DOFs.
// One thread per matrix entry, summing over the elements shared by both
// nodes (deterministic).  Row-major n x n.
// ---------------------------------------------------------------------------
template <int DIM, typename T, typename TA>
__global__ void __launch_bounds__(256)
    k_dense_assemble(GridP g, const uint8_t* __restrict__ mask, const T* __restrict__ Kc,
                     TA* __restrict__ A, double shift) {
  constexpr int ND = Geo<DIM>::ND;
  const long long n = DIM * g.nn;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const long long row = t / n, col = t % n;
  const long long nr = row / DIM, nc = col / DIM;
  const int cr = (int)(row % DIM), cc = (int)(col % DIM);
  const bool fr = (mask[nr] >> cr) & 1u, fc = (mask[nc] >> cc) & 1u;
  if (fr || fc) {
    A[t] = (row == col) ? TA(1) : TA(0);
    return;
  }
  const int ir = (int)(nr % g.nnx), jr = (int)((nr / g.nnx) % g.nny), kr = DIM == 3 ? (int)(nr / ((long long)g.nnx * g.nny)) : 0;
  const int ic = (int)(nc % g.nnx), jc = (int)((nc / g.nnx) % g.nny), kc = DIM == 3 ? (int)(nc / ((long long)g.nnx * g.nny)) : 0;
  TA s = TA(0);
  if (abs(ir - ic) <= 1 && abs(jr - jc) <= 1 && abs(kr - kc) <= 1) {
    const int exlo = max(max(ir, ic) - 1, 0), exhi = min(min(ir, ic), g.nx - 1);
    const int eylo = max(max(jr, jc) - 1, 0), eyhi = min(min(jr, jc), g.ny - 1);
    const int ezlo = DIM == 3 ? max(max(kr, kc) - 1, 0) : 0;
    const int ezhi = DIM == 3 ? min(min(kr, kc), g.nz - 1) : 0;
    for (int ez = ezlo; ez <= ezhi; ++ez)
      for (int ey = eylo; ey <= eyhi; ++ey)
        for (int ex = exlo; ex <= exhi; ++ex) {
          const long long e = ex + (long long)g.nx * (ey + (long long)g.ny * ez);
          const int ar = (ir - ex) + 2 * (jr - ey) + (DIM == 3 ? 4 * (kr - ez) : 0);
          const int ac = (ic - ex) + 2 * (jc - ey) + (DIM == 3 ? 4 * (kc - ez) : 0);
          s += (TA)Kc[(size_t)e * tri_len(ND) + sym_idx(DIM * ar + cr, DIM * ac + cc, ND)];
        }
  }
  A[t] = row == col ? (TA)((double)s * (1.0 + shift)) : s;
}

// In-place Cholesky (lower) of the n x n row-major matrix A by one block,
// right-looking.  A non-positive pivot sets *status = TO_E_SINGULAR.
template <typename T>
__global__ void __launch_bounds__(1024) k_cholesky(int n, T* __restrict__ A, int* status) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      T d = A[(size_t)k * n + k];
      if (!(d > T(0))) {
        s_bad = 1;
        d = T(1);
      }
      A[(size_t)k * n + k] = sqrt(d);
    }
    __syncthreads();
    const T lkk = A[(size_t)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= lkk;
    __syncthreads();
    for (int i = k + 1 + ty; i < n; i += nty) {
      const T lik = A[(size_t)i * n + k];
      for (int j = k + 1 + tx; j <= i; j += 32) A[(size_t)i * n + j] -= lik * A[(size_t)j * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && s_bad) *status = TO_E_SINGULAR;
}

// Blocked right-looking Cholesky (lower, in place) by one block of 1024
// threads: per 32-column block, the diagonal block is factored in shared
// memory (one entry per thread in each column's update), the panel below it
// is staged in shared memory and solved row by row, and the trailing lower
// triangle is updated by all threads in 4 x 4 register tiles.
constexpr int CB = 32, CBP = 33;

__device__ __forceinline__ void tri_index(long long p, int& ii, int& jj) {
  // float estimate (GB300's FP64 pipe is slow), corrected in integers
  int r = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
  while ((long long)r * (r + 1) / 2 > p) --r;
  while ((long long)(r + 1) * (r + 2) / 2 <= p) ++r;
  ii = r;
  jj = (int)(p - (long long)r * (r + 1) / 2);
}

template <typename T>
__global__ void __launch_bounds__(1024) k_cholesky_blocked(int n, T* __restrict__ A, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Dg = reinterpret_cast<T*>(smem_raw);   // CB x CBP
  T* Pn = Dg + CB * CBP;                    // (n) x CBP panel rows
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  for (int k0 = 0; k0 < n; k0 += CB) {
    const int kb = min(CB, n - k0);
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
      const int r = idx / kb, cc = idx % kb;
      Dg[r * CBP + cc] = A[(size_t)(k0 + r) * n + k0 + cc];
    }
    __syncthreads();
    // diagonal block: per column j the pivot, the scaling of the column and
    // the rank-1 update of the block's remaining lower triangle, one entry
    // per thread (thread (r, cc) = (tid / 32, tid % 32))
    {
      const int r = tid >> 5, cc = tid & 31;
      for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
          T d = Dg[j * CBP + j];
          if (!(d > T(0))) {
            s_bad = 1;
            d = T(1);
          }
          Dg[j * CBP + j] = sqrt(d);
        }
        __syncthreads();
        if (tid > j && tid < kb) Dg[tid * CBP + j] /= Dg[j * CBP + j];
        __syncthreads();
        if (r > j && r < kb && cc > j && cc <= r) Dg[r * CBP + cc] -= Dg[r * CBP + j] * Dg[cc * CBP + j];
        __syncthreads();
      }
    }
    for (int idx = tid; idx < kb * kb; idx += blockDim.x) {
      const int r = idx / kb, cc = idx % kb;
      if (cc <= r) A[(size_t)(k0 + r) * n + k0 + cc] = Dg[r * CBP + cc];
    }
    const int m = n - k0 - kb;
    // the panel below the diagonal block, staged by all threads (coalesced
    // rows), then solved row by row in place
    for (int idx = tid; idx < m * kb; idx += blockDim.x) {
      const int r = idx / kb, cc = idx - r * kb;
      Pn[r * CBP + cc] = A[(size_t)(k0 + kb + r) * n + k0 + cc];
    }
    __syncthreads();
    for (int r = tid; r < m; r += blockDim.x) {
      const size_t row = (size_t)(k0 + kb + r) * n + k0;
      T xr[CB];
#pragma unroll
      for (int cc = 0; cc < CB; ++cc) {
        if (cc < kb) {
          T s = Pn[r * CBP + cc];
#pragma unroll
          for (int t = 0; t < CB; ++t)
            if (t < cc) s -= xr[t] * Dg[cc * CBP + t];
          xr[cc] = s / Dg[cc * CBP + cc];
          A[row + cc] = xr[cc];
          Pn[r * CBP + cc] = xr[cc];
        }
      }
    }
    __syncthreads();
    // trailing update by 4 x 4 tiles of the lower triangle, one tile per
    // thread and pass: each entry sums its kb products in the same order as
    // an entry-wise loop, the tile's panel rows are read once per t
    const int mt = (m + 3) >> 2;
    const long long tiles = (long long)mt * (mt + 1) / 2;
    for (long long p = tid; p < tiles; p += blockDim.x) {
      int ti, tj;
      tri_index(p, ti, tj);
      const int r0 = 4 * ti, c0 = 4 * tj;
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
      for (int t = 0; t < kb; ++t) {
        T pr[4], pc[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          pr[a] = r0 + a < m ? Pn[(r0 + a) * CBP + t] : T(0);
          pc[a] = c0 + a < m ? Pn[(c0 + a) * CBP + t] : T(0);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += pr[a] * pc[b];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int ii = r0 + a, jj = c0 + b;
          if (ii < m && jj <= ii) A[(size_t)(k0 + kb + ii) * n + k0 + kb + jj] -= acc[a][b];
        }
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad) *status = TO_E_SINGULAR;
}

// X = L^{-1} by forward substitution, one warp per column (stored in the
// upper triangle-free buffer Linv, row-major, zero above the diagonal).
template <typename T>
__global__ void __launch_bounds__(256)
    k_lower_inverse(int n, const T* __restrict__ L, T* __restrict__ X) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int jc = warp;
  for (int i = lane; i < jc; i += 32) X[(size_t)i * n + jc] = T(0);
  if (lane == 0) X[(size_t)jc * n + jc] = T(1) / L[(size_t)jc * n + jc];
  __syncwarp();
  for (int i = jc + 1; i < n; ++i) {
    T s = T(0);
    for (int m = jc + lane; m < i; m += 32) s += L[(size_t)i * n + m] * X[(size_t)m * n + jc];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) X[(size_t)i * n + jc] = -s / L[(size_t)i * n + i];
    __syncwarp();
  }
}

// X = L^{-1} by column blocks: CTA jb owns the 32 columns jb*32 .. jb*32+31
// of X (zero above row block jb) and walks the row blocks ib = jb, jb+1, ...
// downwards: R = I(ib, jb) - sum_{kb < ib} L(ib, kb) X(kb, jb) (32 x 32
// products, the L block staged in shared memory, the X column block kept
// there), then one warp solves L(ib, ib) X(ib, jb) = R by forward
// substitution, a column per lane.  1024 threads: (ty, tx) = (row, column)
// within a block.
template <typename T>
__global__ void __launch_bounds__(1024) k_lower_inverse_blocked(int n, const T* __restrict__ L,
                                                                T* __restrict__ X) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nbk = (n + 31) / 32;
  T* Xs = reinterpret_cast<T*>(smem_raw);   // [nbk * 32][32]
  T* Ls = Xs + (size_t)nbk * 32 * 32;       // [32][33]
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int jb = blockIdx.x;
  for (int ib = jb; ib < nbk; ++ib) {
    T r = (ib == jb && ty == tx) ? T(1) : T(0);
    const int lr = ib * 32 + ty;
    for (int kb = jb; kb < ib; ++kb) {
      const int lc = kb * 32 + tx;
      Ls[ty * 33 + tx] = (lr < n && lc < n) ? L[(size_t)lr * n + lc] : T(0);
      __syncthreads();
#pragma unroll 8
      for (int m = 0; m < 32; ++m) r -= Ls[ty * 33 + m] * Xs[(kb * 32 + m) * 32 + tx];
      __syncthreads();
    }
    // diagonal block (identity beyond n, so padded rows solve to zero)
    {
      const int dc = ib * 32 + tx;
      Ls[ty * 33 + tx] = (lr < n && dc < n) ? L[(size_t)lr * n + dc] : (ty == tx ? T(1) : T(0));
    }
    Xs[(ib * 32 + ty) * 32 + tx] = r;
    __syncthreads();
    if (ty == 0) {
      T* xb = Xs + (size_t)ib * 32 * 32;
      for (int k = 0; k < 32; ++k) {
        T v = xb[k * 32 + tx];
        for (int m = 0; m < k; ++m) v -= Ls[k * 33 + m] * xb[m * 32 + tx];
        xb[k * 32 + tx] = v / Ls[k * 33 + k];
      }
    }
    __syncthreads();
  }
  const int col = jb * 32 + tx;
  if (col < n)
    for (int row = ty; row < n; row += 32)
      X[(size_t)row * n + col] = row >= jb * 32 ? Xs[row * 32 + tx] : T(0);
}

// Ainv = X^T X (X = L^{-1} lower triangular): Ainv[i][j] = sum_{m>=max(i,j)} X[m][i] X[m][j]
template <typename T>
__global__ void __launch_bounds__(256)
    k_gram_lower(int n, const T* __restrict__ X, T* __restrict__ Ainv) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  T s = T(0);
  for (int m = max(i, j); m < n; ++m) s += X[(size_t)m * n + i] * X[(size_t)m * n + j];
  Ainv[t] = s;
}

// y = A x with the matrix (and the accumulation) in TA and the vectors in TV
template <typename TA, typename TV>
__global__ void __launch_bounds__(256)
    k_gemv(int n, const TA* __restrict__ A, const TV* __restrict__ x, TV* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  pdl_wait();
  if (warp >= n) return;
  TA s = TA(0);
  for (int m = lane; m < n; m += 32) s += A[(size_t)warp * n + m] * (TA)x[m];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) y[warp] = (TV)s;
  pdl_launch_dependents();
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
template <int DIM, typename T>
static cudaError_t restrict_t(const GridP& gf, const uint8_t* mf, const GridP& gc,
                              const uint8_t* mc, const void* rf, void* bc, const void* dinvc,
                              double omega, void* zc, bool clean, cudaStream_t s) {
  if (gc.nn <= 0) return cudaSuccess;
  const long long pv = (long long)DIM * gc.nnx * gc.nny;
  if (pv >= (1LL << 31) - TVAL || gc.nnz > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((pv + TVAL - 1) / TVAL), DIM == 3 ? gc.nnz : 1);
  auto kern = clean ? k_restrict<DIM, T, true> : k_restrict<DIM, T, false>;
  return launch_pdl(kern, grid, dim3(TVAL), 0, s, gf, mf, gc, mc, (const T*)rf, (T*)bc,
                    (const T*)dinvc, T(omega), (T*)zc);
}

cudaError_t launch_restrict(int dim, int t, const GridP& gf, const uint8_t* mf, const GridP& gc,
                            const uint8_t* mc, const void* rf, void* bc, const void* dinvc,
                            double omega, void* zc, bool clean, cudaStream_t s) {
  if (dim == 2)
    return t == T_F64 ? restrict_t<2, double>(gf, mf, gc, mc, rf, bc, dinvc, omega, zc, clean, s)
                      : restrict_t<2, float>(gf, mf, gc, mc, rf, bc, dinvc, omega, zc, clean, s);
  return t == T_F64 ? restrict_t<3, double>(gf, mf, gc, mc, rf, bc, dinvc, omega, zc, clean, s)
                    : restrict_t<3, float>(gf, mf, gc, mc, rf, bc, dinvc, omega, zc, clean, s);
}

template <int DIM, typename T>
static cudaError_t prolong_t(const GridP& gf, const uint8_t* mf, const GridP& gc, const void* zc,
                             void* zf, cudaStream_t s) {
  if (gf.nn <= 0) return cudaSuccess;
  dim3 grid((gf.nnx + TBX - 1) / TBX, (gf.nny + TBY - 1) / TBY, DIM == 3 ? (gf.nnz + 1) / 2 : 1);
  return launch_pdl(k_prolong_add<DIM, T>, grid, dim3(TBX, TBY), 0, s, gf, mf, gc, (const T*)zc,
                    (T*)zf);
}

cudaError_t launch_prolong_add(int dim, int t, const GridP& gf, const uint8_t* mf,
                               const GridP& gc, const void* zc, void* zf, cudaStream_t s) {
  if (dim == 2) return t == T_F64 ? prolong_t<2, double>(gf, mf, gc, zc, zf, s)
                                  : prolong_t<2, float>(gf, mf, gc, zc, zf, s);
  return t == T_F64 ? prolong_t<3, double>(gf, mf, gc, zc, zf, s)
                    : prolong_t<3, float>(gf, mf, gc, zc, zf, s);
}

cudaError_t launch_presmooth(int t, int tin, long long n, const void* bin, void* bout,
                             const void* dinv, double omega, void* z, cudaStream_t s) {
  const int nb = nblocks(n, 256);
  if (t == T_F64) {
    if (tin != T_F64) return cudaErrorInvalidValue;
    return launch_pdl(k_presmooth<double, double>, dim3(nb), dim3(256), 0, s, n,
                      (const double*)bin, (double*)bout, (const double*)dinv, omega, (double*)z);
  } else if (tin == T_F64) {
    return launch_pdl(k_presmooth<float, double>, dim3(nb), dim3(256), 0, s, n,
                      (const double*)bin, (float*)bout, (const float*)dinv, (float)omega, (float*)z);
  } else if (tin == T_D2) {
    return launch_pdl(k_presmooth<float, float2>, dim3(nb), dim3(256), 0, s, n,
                      (const float2*)bin, (float*)bout, (const float*)dinv, (float)omega, (float*)z);
  } else {
    return launch_pdl(k_presmooth<float, float>, dim3(nb), dim3(256), 0, s, n,
                      (const float*)bin, (float*)bout, (const float*)dinv, (float)omega, (float*)z);
  }
  return cudaGetLastError();
}

cudaError_t launch_convert(int tin, int tout, long long n, const void* in, void* out,
                           cudaStream_t s) {
  const int nb = nblocks(n, 256);
  if (tin == T_D2 && tout == T_F32)
    k_convert<float2, float><<<nb, 256, 0, s>>>(n, (const float2*)in, (float*)out);
  else if (tin == T_F32 && tout == T_D2)
    k_convert<float, float2><<<nb, 256, 0, s>>>(n, (const float*)in, (float2*)out);
  else if (tin == T_F64 && tout == T_F32)
    k_convert<double, float><<<nb, 256, 0, s>>>(n, (const double*)in, (float*)out);
  else if (tin == T_F32 && tout == T_F64)
    k_convert<float, double><<<nb, 256, 0, s>>>(n, (const float*)in, (double*)out);
  else if (tin == T_F64)
    k_convert<double, double><<<nb, 256, 0, s>>>(n, (const double*)in, (double*)out);
  else
    k_convert<float, float><<<nb, 256, 0, s>>>(n, (const float*)in, (float*)out);
  return cudaGetLastError();
}

template <int DIM, typename T>
static cudaError_t gal_fine_t(const GridP& gc, const GridP& gf, const void* coef, const void* Qc,
                              void* Kc, cudaStream_t s) {
  constexpr int ND = Geo<DIM>::ND;
  const long long tot = gc.nel * tri_len(ND);
  k_galerkin_fine<DIM, T><<<nblocks(tot, 256), 256, 0, s>>>(gc, gf, (const T*)coef,
                                                            (const T*)Qc, (T*)Kc);
  return cudaGetLastError();
}

// Springs in the level-1 Galerkin matrices: the spring at fine DOF (node n,
// component c) adds k w_A w_B to entry (DIM A + c, DIM B + c) of one coarse
// element holding n, w the 1D linear weights of n at that element's corners
// (P^T S P; any element holding n gives the same assembled operator, since
// n interpolates only from the corners of each element holding it).  One
// thread per spring, springs applied in order.
template <int DIM, typename T>
__global__ void k_spring_galerkin(GridP gc, GridP gf, Springs sp, T* __restrict__ Kc) {
  constexpr int ND = Geo<DIM>::ND, NPE = Geo<DIM>::NPE, NT = tri_len(ND);
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (int q = 0; q < sp.n; ++q) {
    const long long node = sp.dof[q] / DIM;
    const int c = (int)(sp.dof[q] % DIM);
    const int i = (int)(node % gf.nnx);
    const long long rest = node / gf.nnx;
    const int j = (int)(rest % gf.nny);
    const int k = DIM == 3 ? (int)(rest / gf.nny) : 0;
    const int EX = min(i / 2, gc.nx - 1), EY = min(j / 2, gc.ny - 1);
    const int EZ = DIM == 3 ? min(k / 2, gc.nz - 1) : 0;
    const long long E = EX + (long long)gc.nx * (EY + (long long)gc.ny * EZ);
    double w[NPE];
    for (int a = 0; a < NPE; ++a) {
      const double px = 0.5 * (i - 2 * EX), py = 0.5 * (j - 2 * EY), pz = 0.5 * (k - 2 * EZ);
      w[a] = ((a & 1) ? px : 1.0 - px) * (((a >> 1) & 1) ? py : 1.0 - py) *
             (DIM == 3 ? (((a >> 2) & 1) ? pz : 1.0 - pz) : 1.0);
    }
    for (int a = 0; a < NPE; ++a)
      for (int b = a; b < NPE; ++b) {
        const double v = sp.k[q] * w[a] * w[b];
        if (v != 0.0) Kc[(size_t)E * NT + tri_idx(DIM * a + c, DIM * b + c, ND)] += T(v);
      }
  }
}

cudaError_t launch_spring_galerkin(int dim, int t, const GridP& gc, const GridP& gf,
                                   const Springs& sp, void* Kc, cudaStream_t s) {
  if (sp.n <= 0) return cudaSuccess;
  if (dim == 2) {
    if (t == T_F64) k_spring_galerkin<2, double><<<1, 32, 0, s>>>(gc, gf, sp, (double*)Kc);
    else k_spring_galerkin<2, float><<<1, 32, 0, s>>>(gc, gf, sp, (float*)Kc);
  } else {
    if (t == T_F64) k_spring_galerkin<3, double><<<1, 32, 0, s>>>(gc, gf, sp, (double*)Kc);
    else k_spring_galerkin<3, float><<<1, 32, 0, s>>>(gc, gf, sp, (float*)Kc);
  }
  return cudaGetLastError();
}

cudaError_t launch_galerkin_fine(int dim, int t, const GridP& gc, const GridP& gf,
                                 const void* coef, const void* Qc, void* Kc, cudaStream_t s) {
  if (dim == 2) return t == T_F64 ? gal_fine_t<2, double>(gc, gf, coef, Qc, Kc, s)
                                  : gal_fine_t<2, float>(gc, gf, coef, Qc, Kc, s);
  return t == T_F64 ? gal_fine_t<3, double>(gc, gf, coef, Qc, Kc, s)
                    : gal_fine_t<3, float>(gc, gf, coef, Qc, Kc, s);
}

template <typename T>
static cudaError_t diag_l1_t(const GridP& g1, const GridP& gf, const uint8_t* mask,
                             const double* qdiag, const void* coef, void* dinv, cudaStream_t s) {
  QDiagP<T> qd;
  for (int q = 0; q < 192; ++q) qd.v[q] = T(qdiag[q]);
  k_diag_l1<T><<<nblocks(g1.nn, 256), 256, 0, s>>>(g1, gf, mask, qd, (const T*)coef, (T*)dinv);
  return cudaGetLastError();
}

cudaError_t launch_diag_l1(int t, const GridP& g1, const GridP& gf, const uint8_t* mask,
                           const double* qdiag, const void* coef, void* dinv, cudaStream_t s) {
  return t == T_F64 ? diag_l1_t<double>(g1, gf, mask, qdiag, coef, dinv, s)
                    : diag_l1_t<float>(g1, gf, mask, qdiag, coef, dinv, s);
}

cudaError_t launch_galerkin_l2(int t, const GridP& g2, const GridP& gf, const void* coef,
                               const void* R, void* Kc, cudaStream_t s) {
  const long long tot = g2.nel * tri_len(24);
  if (t == T_F64)
    k_galerkin_l2<double><<<nblocks(tot, 256), 256, 0, s>>>(g2, gf, (const double*)coef,
                                                             (const double*)R, (double*)Kc);
  else
    k_galerkin_l2<float><<<nblocks(tot, 256), 256, 0, s>>>(g2, gf, (const float*)coef,
                                                           (const float*)R, (float*)Kc);
  return cudaGetLastError();
}

template <int DIM, typename T>
static cudaError_t gal_coarse_t(const GridP& gc, const GridP& gf, const void* Kf, void* Kc,
                                cudaStream_t s) {
  constexpr int ND = Geo<DIM>::ND;
  if (gc.nel <= 0) return cudaSuccess;
  k_galerkin_coarse<DIM, T><<<(unsigned)gc.nel, ND * ND, 0, s>>>(gc, gf, (const T*)Kf, (T*)Kc);
  return cudaGetLastError();
}

cudaError_t launch_galerkin_coarse(int dim, int t, const GridP& gc, const GridP& gf,
                                   const void* Kf, void* Kc, cudaStream_t s) {
  if (dim == 2) return t == T_F64 ? gal_coarse_t<2, double>(gc, gf, Kf, Kc, s)
                                  : gal_coarse_t<2, float>(gc, gf, Kf, Kc, s);
  return t == T_F64 ? gal_coarse_t<3, double>(gc, gf, Kf, Kc, s)
                    : gal_coarse_t<3, float>(gc, gf, Kf, Kc, s);
}

template <int DIM, typename T, typename TA>
static cudaError_t dense_t(const GridP& g, const uint8_t* mask, const void* Kc, void* A,
                           double shift, cudaStream_t s) {
  const long long n = DIM * g.nn;
  k_dense_assemble<DIM, T, TA><<<nblocks(n * n, 256), 256, 0, s>>>(g, mask, (const T*)Kc,
                                                                   (TA*)A, shift);
  return cudaGetLastError();
}

cudaError_t launch_dense_assemble(int dim, int t, int ta, const GridP& g, const uint8_t* mask,
                                  const void* Kc, void* A, double shift, cudaStream_t s) {
  if (t == T_F64 && ta == T_F64)
    return dim == 2 ? dense_t<2, double, double>(g, mask, Kc, A, shift, s)
                    : dense_t<3, double, double>(g, mask, Kc, A, shift, s);
  if (t == T_F32 && ta == T_F64)
    return dim == 2 ? dense_t<2, float, double>(g, mask, Kc, A, shift, s)
                    : dense_t<3, float, double>(g, mask, Kc, A, shift, s);
  if (t == T_F32 && ta == T_F32)
    return dim == 2 ? dense_t<2, float, float>(g, mask, Kc, A, shift, s)
                    : dense_t<3, float, float>(g, mask, Kc, A, shift, s);
  return cudaErrorInvalidValue;
}

// The blocked kernels' dynamic shared memory limit is set once, to the most
// the device allows next to the kernel's static shared memory, not to each
// call's own size: contexts of different sizes run their set-up from
// different host threads, and a limit lowered by one thread between another
// thread's setting and launch would reject that launch.
template <typename K>
static int raise_dyn_smem_limit(K kernel) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, kernel) != cudaSuccess)
    return 48 * 1024;
  const int lim = optin - (int)fa.sharedSizeBytes;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) ==
                 cudaSuccess
             ? lim
             : 48 * 1024;
}

template <typename T>
static cudaError_t cholinv_t(int n, void* A, void* Ainv, int* status, cudaStream_t s) {
  const size_t smem = (size_t)(CB * CBP + (size_t)n * CBP) * sizeof(T);
  static const int chol_lim = raise_dyn_smem_limit(k_cholesky_blocked<T>);
  static const int inv_lim = raise_dyn_smem_limit(k_lower_inverse_blocked<T>);
  cudaError_t e;
  if (smem <= (size_t)chol_lim) {
    k_cholesky_blocked<T><<<1, 1024, smem, s>>>(n, (T*)A, status);
  } else {
    k_cholesky<T><<<1, 1024, 0, s>>>(n, (T*)A, status);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // Ainv is used as scratch for L^{-1} first, then A receives X^T X and
  // the buffers are swapped by copying back.
  const int nbk = (n + 31) / 32;
  const size_t ismem = ((size_t)nbk * 32 * 32 + 32 * 33) * sizeof(T);
  if (ismem <= (size_t)inv_lim) {
    k_lower_inverse_blocked<T><<<nbk, 1024, ismem, s>>>(n, (const T*)A, (T*)Ainv);
  } else {
    k_lower_inverse<T><<<nblocks((long long)n * 32, 256), 256, 0, s>>>(n, (const T*)A, (T*)Ainv);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram_lower<T><<<nblocks((long long)n * n, 256), 256, 0, s>>>(n, (const T*)Ainv, (T*)A);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(Ainv, A, sizeof(T) * (size_t)n * n, cudaMemcpyDeviceToDevice, s);
}

cudaError_t launch_cholesky_inverse(int t, int n, void* A, void* Ainv, int* status,
                                    cudaStream_t s) {
  return t == T_F64 ? cholinv_t<double>(n, A, Ainv, status, s)
                    : cholinv_t<float>(n, A, Ainv, status, s);
}

cudaError_t launch_dense_gemv(int ta, int t, int n, const void* A, const void* x, void* y,
                              cudaStream_t s) {
  const int nb = nblocks((long long)n * 32, 256);
  if (ta == T_F64 && t == T_F64)
    return launch_pdl(k_gemv<double, double>, dim3(nb), dim3(256), 0, s, n, (const double*)A,
                      (const double*)x, (double*)y);
  if (ta == T_F64)
    return launch_pdl(k_gemv<double, float>, dim3(nb), dim3(256), 0, s, n, (const double*)A,
                      (const float*)x, (float*)y);
  return launch_pdl(k_gemv<float, float>, dim3(nb), dim3(256), 0, s, n, (const float*)A,
                    (const float*)x, (float*)y);
}

}  // namespace topo
