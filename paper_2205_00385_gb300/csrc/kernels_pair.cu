// Finest-grid 3D stiffness operator in float32, two element columns per
// thread with packed f32x2 arithmetic (Sec. 2 / Eq. 1: K(rho) x assembled
// element by element from E_e KE; fixed DOFs enter as M K M + dfix (I - M)).
//
// The element operator is applied in the corner Walsh-Hadamard basis
// (KE = T B T with B eight 3x3 blocks, 45 non-zero entries).  Compared with
// the one-column kernel in kernels_fe.cu:
//  * each thread owns the element pair (i, i+1) of one x-row of columns and
//    streams it up in z; the pair's two elements are the two lanes of every
//    f32x2 add / mul / fma, so one instruction serves both elements;
//  * the transform is separable, T = T_z (x) T_xy: the xy part of each
//    horizontal face is computed once and serves the element below and the
//    element above; on the way back, the two elements' contributions to a
//    shared face are added in the xy-Walsh domain and transformed once;
//  * one face row (three nodes) is loaded per thread and row, the middle
//    node serving both elements;
//  * fixed-DOF masking runs only in warps that touch a node column holding a
//    fixed DOF (a per-column flag computed once at mesh set-up).
// A block of 16 x 8 threads covers 32 x 8 element columns and owns the
// 30 x 7 nodes whose surrounding columns it computes; per z-layer the
// column partials of each owned node are summed in shared memory in a fixed
// order (deterministic, no atomics).
#include <algorithm>

#include "kernels.h"
#include "topo_internal.cuh"

namespace topo {
namespace {

constexpr int PX = 16, POX = 2 * (PX - 1), PZC = 16;

struct WhtPair {
  float2 b[8][3][3];   // Walsh blocks with each entry in both lanes
};

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b = fma(b, -1, a), rounded once: the packed FMA keeps the operands in
// register pairs chosen by the compiler (no packed subtract intrinsic)
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// 4-point Walsh-Hadamard transform over the corners q = bx + 2 by of a face
// (self-inverse up to the factor 4, which is folded into B).
__device__ __forceinline__ void wht4(const float2 (&v)[4], float2 (&w)[4]) {
  const float2 s0 = padd(v[0], v[1]), d0 = psub(v[0], v[1]);
  const float2 s1 = padd(v[2], v[3]), d1 = psub(v[2], v[3]);
  w[0] = padd(s0, s1);
  w[1] = padd(d0, d1);
  w[2] = psub(s0, s1);
  w[3] = psub(d0, d1);
}

// true if column cp of Walsh block tau is structurally zero
__host__ __device__ constexpr bool wht_col_zero(int tau, int cp) {
  return wht_zero(tau, 0, cp) && wht_zero(tau, 1, cp) && wht_zero(tau, 2, cp);
}

// Element pair: bottom and top face transforms Wb, Wt (xy-Walsh, per
// component), moduli ce = (E_A, E_B).  Returns the xy-Walsh coefficients of
// the pair's contributions to its bottom face (Ub) and top face (Ut).
__device__ __forceinline__ void pair_element(const WhtPair& kb, float2 ce,
                                             const float2 (&Wb)[3][4], const float2 (&Wt)[3][4],
                                             float2 (&Ub)[3][4], float2 (&Ut)[3][4]) {
  float2 X[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      X[c][t] = padd(Wb[c][t], Wt[c][t]);
      X[c][t + 4] = psub(Wb[c][t], Wt[c][t]);
    }
  float2 Y[3][8];
#pragma unroll
  for (int tau = 0; tau < 8; ++tau) {
    float2 zt[3];
#pragma unroll
    for (int cp = 0; cp < 3; ++cp)
      zt[cp] = wht_col_zero(tau, cp) ? make_float2(0.f, 0.f) : pmul(ce, X[cp][tau ^ (1 << cp)]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 s = make_float2(0.f, 0.f);
      bool first = true;
#pragma unroll
      for (int cp = 0; cp < 3; ++cp) {
        if (wht_zero(tau, c, cp)) continue;
        s = first ? pmul(kb.b[tau][c][cp], zt[cp]) : pfma(kb.b[tau][c][cp], zt[cp], s);
        first = false;
      }
      Y[c][tau ^ (1 << c)] = s;
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      Ub[c][t] = padd(Y[c][t], Y[c][t + 4]);
      Ut[c][t] = psub(Y[c][t], Y[c][t + 4]);
    }
}

struct PairArgs {
  GridP g;
  const uint8_t* mask;
  const uint8_t* colfix;   // per node column (i, j): any DOF fixed at any k
  const float* coef;
  int zc;
  const float* x;
  float* y;
  const float* b;
  const float* dinv;
  float omega, dfix;
  bool clean_inputs;       // x (and, fused, b) zero on every fixed DOF
  // work-list launch (null: one block per tile and z-chunk): wl[0] hands out
  // the items (tile x fastest, z-chunk slowest), wl[1] counts the CTAs done
  unsigned* wl;
  int gx, gy, nitems;
};

// Face tile of a block of PX x PY threads: (2 PX + 1) x (PY + 1) nodes,
// three floats per node, rows of FROW floats (odd, so the two half-warps'
// rows hit disjoint banks).  PY is 8 or 16 (the taller tile computes 16
// element rows for 15 owned node rows instead of 8 for 7).
constexpr int FNX = 2 * PX + 1, FROW = 3 * FNX;
constexpr int NSTAGE = 4;                                   // faces in flight
static_assert((NSTAGE & (NSTAGE - 1)) == 0, "stage index uses a mask");
static_assert(FROW <= 128, "face copy: 4 lanes per row segment");
template <int PY>
struct PairGeo {
  static constexpr int POY = PY - 1, FNY = PY + 1, FTILE = FROW * FNY, NT = PX * PY;
  static constexpr int NWARP = NT / 32, RPW = (FNY + NWARP - 1) / NWARP;   // face rows per warp
};

__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int PY>
struct PairSmem {
  float face[NSTAGE][PairGeo<PY>::FTILE];
  float4 pub[2][4][PY][PX];
};

// MODE 0: no fixed DOF in the block's columns; 1: inputs and outputs masked
// (M K M x + dfix (I - M) x for any x); 2: outputs only, for inputs that are
// zero on the fixed DOFs (the solver's own vectors), where masking the input
// values changes nothing and only the fixed rows' outputs need setting.
template <int EPI, int MODE, int PY>
__device__ __forceinline__ void pair_loop(const PairArgs& a, const WhtPair& kb,
                                          PairSmem<PY>& sm, int bx, int by, int bz) {
  using G = PairGeo<PY>;
  constexpr int POY = G::POY, FNY = G::FNY, FTILE = G::FTILE;
  constexpr bool MASKED = MODE == 1, MASK_OUT = MODE != 0;
  const GridP& g = a.g;
  const int tid = threadIdx.x;
  const int tx = tid % PX, ty = tid / PX;
  const int X0 = bx * POX, Y0 = by * POY;
  const int z0 = bz * a.zc, z1 = min(z0 + a.zc, g.nnz);
  const int i = X0 - 1 + 2 * tx, j = Y0 - 1 + ty;   // corner 0 of element A
  const long long plane = (long long)g.nnx * g.nny;
  const bool eA = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  const bool eB = i + 1 >= 0 && i + 1 < g.nx && j >= 0 && j < g.ny;

  // Face copies: warp w copies tile rows w, w + 4, w + 8; lane l copies the
  // row's floats l + 32 j (j < 4).  Out-of-range nodes are zero-filled (copy
  // size 0) from a clamped, in-range address.
  const int lane = tid & 31, warp = tid >> 5;
  int xoff[4];             // float offset of (lane, j) within a row of node x = 0
  unsigned xok = 0u;       // bit j: column l + 32 j holds an in-range node
  {
    const int xc = min(max(X0 - 1, 0), g.nnx - 1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int col = lane + 32 * j;
      const int ni = X0 - 1 + col / 3;
      const bool ok = col < FROW && ni >= 0 && ni < g.nnx;
      xok |= (ok ? 1u : 0u) << j;
      xoff[j] = ok ? 3 * (X0 - 1) + col : 3 * xc;
    }
  }
  const int fbase = z0 - 1;   // face index of stage 0
  auto issue_face = [&](int kz) {
    const int slot = (kz - fbase) & (NSTAGE - 1);
    if (kz >= 0 && kz < g.nnz && kz <= z1) {
      float* dst = sm.face[slot];
      const float* src = a.x + 3 * plane * kz;
#pragma unroll
      for (int rr = 0; rr < G::RPW; ++rr) {
        const int row = warp + G::NWARP * rr;
        if (row < FNY) {
          const int nj = Y0 - 1 + row;
          const bool rok = nj >= 0 && nj < g.nny;
          const float* rsrc = src + 3LL * g.nnx * min(max(nj, 0), g.nny - 1);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (lane + 32 * j < FROW)
              cp_async4(dst + row * FROW + lane + 32 * j, rsrc + xoff[j],
                        rok && ((xok >> j) & 1u));
        }
      }
    } else if (kz >= z0 - 1 && kz <= z1) {
      // face outside the grid: zeros
      float* dst = sm.face[slot];
      for (int f = tid; f < FTILE; f += G::NT) dst[f] = 0.f;
    }
    cp_commit();
  };
  // node masks of a face (MASKED): 3 bits per (r, n)
  auto face_mask = [&](int kz) -> unsigned {
    unsigned m = 0u;
    if (kz < 0 || kz >= g.nnz) return m;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        const bool ok = i + n >= 0 && i + n < g.nnx && j + r >= 0 && j + r < g.nny;
        const long long nd = (long long)(i + n) + (long long)g.nnx * (j + r) + plane * kz;
        m |= (ok ? (unsigned)a.mask[nd] & 7u : 0u) << (3 * (3 * r + n));
      }
    return m;
  };
  // face -> xy-Walsh coefficients of the pair, per component
  auto face_wht = [&](int kz, unsigned fm, float2 (&W)[3][4]) {
    const float* fs = sm.face[(kz - fbase) & (NSTAGE - 1)] + ty * FROW + 6 * tx;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v[2][3];
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          const float u = fs[r * FROW + 3 * n + c];
          v[r][n] = (MASKED && ((fm >> (3 * (3 * r + n) + c)) & 1u)) ? 0.f : u;
        }
      float2 P[4];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        P[2 * r] = make_float2(v[r][0], v[r][1]);
        P[2 * r + 1] = make_float2(v[r][1], v[r][2]);
      }
      wht4(P, W[c]);
    }
  };
  auto coef_pair = [&](int ez) -> float2 {
    const bool zin = ez >= 0 && ez < g.nz;
    const long long eo = (long long)(eA ? i : i + 1) + (long long)g.nx * (j + (long long)g.ny * ez);
    return make_float2(zin && eA ? a.coef[eo] : 0.f, zin && eB ? a.coef[eo + (eA ? 1 : 0)] : 0.f);
  };

  const bool own = tx < PX - 1 && ty < PY - 1 && i + 1 < g.nnx && j + 1 < g.nny;
  const bool own2 = own && i + 2 < g.nnx;

  // prologue: faces z0-1 .. z0+NSTAGE-2 in flight, z0-1 and z0 complete
#pragma unroll
  for (int s = 0; s < NSTAGE; ++s) issue_face(z0 - 1 + s);
  cp_wait<NSTAGE - 2>();
  __syncthreads();
  float2 Wb[3][4], Wt[3][4], Up[3][4];
  unsigned mb = MASKED ? face_mask(z0 - 1) : 0u, mt = MASKED ? face_mask(z0) : 0u;
  face_wht(z0 - 1, mb, Wb);
  __syncthreads();
  issue_face(z0 - 1 + NSTAGE);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int t = 0; t < 4; ++t) Up[c][t] = make_float2(0.f, 0.f);
  float2 ce = coef_pair(z0 - 1);
  int buf = 0;
  // invariant at the top of step ez: the stages hold faces ez+1 .. ez+NSTAGE,
  // face ez+1 complete and visible to the block
  for (int ez = z0 - 1; ez < z1; ++ez) {
    // epilogue operands of the owned nodes of layer ez, requested before the
    // element compute so that their latency overlaps it
    const long long nd0 = (long long)(i + 1) + (long long)g.nnx * (j + 1) + plane * ez;
    const bool ep = own && ez >= z0;
    float eb[2][3], ex[2][3], ed[2][3];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool ok = ep && (m == 0 || own2);
        const long long d = 3 * (nd0 + m) + c;
        eb[m][c] = (EPI != EPI_APPLY && ok) ? a.b[d] : 0.f;
        ex[m][c] = (EPI == EPI_SMOOTH && ok) ? a.x[d] : 0.f;
        ed[m][c] = (EPI == EPI_SMOOTH && ok) ? a.dinv[d] : 0.f;
      }
    face_wht(ez + 1, mt, Wt);
    const float2 ce_next = coef_pair(ez + 1);
    if (MASKED) mt = face_mask(ez + 2);
    float2 Ub[3][4], Ut[3][4];
    pair_element(kb, ce, Wb, Wt, Ub, Ut);
    ce = ce_next;
    float part[2][3][3];   // nodal partials of layer ez: row r, node i+n, component
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 acc[4], o[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        acc[t] = padd(Up[c][t], Ub[c][t]);
        Up[c][t] = Ut[c][t];
        Wb[c][t] = Wt[c][t];
      }
      wht4(acc, o);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        part[r][0][c] = o[2 * r].x;
        part[r][1][c] = o[2 * r + 1].x + o[2 * r].y;
        part[r][2][c] = o[2 * r + 1].y;
      }
    }
    sm.pub[buf][0][ty][tx] = make_float4(part[0][0][0], part[0][0][1], part[0][0][2], 0.f);
    sm.pub[buf][1][ty][tx] = make_float4(part[0][1][0], part[0][1][1], part[0][1][2], 0.f);
    sm.pub[buf][2][ty][tx] = make_float4(part[0][2][0], part[0][2][1], part[0][2][2], 0.f);
    sm.pub[buf][3][ty][tx] = make_float4(part[1][0][0], part[1][0][1], part[1][0][2], 0.f);
    cp_wait<NSTAGE - 2>();   // this thread's copies of face ez+2 have landed
    __syncthreads();
    issue_face(ez + 1 + NSTAGE);   // into the stage of face ez+1, read above
    if (ep) {
      const float4 m1 = sm.pub[buf][1][ty + 1][tx];
      const float4 q3 = sm.pub[buf][3][ty][tx + 1];
      const float4 q2 = sm.pub[buf][2][ty + 1][tx];
      const float4 q0 = sm.pub[buf][0][ty + 1][tx + 1];
      float s[2][3];
      s[0][0] = part[1][1][0] + m1.x;
      s[0][1] = part[1][1][1] + m1.y;
      s[0][2] = part[1][1][2] + m1.z;
      s[1][0] = ((part[1][2][0] + q3.x) + q2.x) + q0.x;
      s[1][1] = ((part[1][2][1] + q3.y) + q2.y) + q0.y;
      s[1][2] = ((part[1][2][2] + q3.z) + q2.z) + q0.z;
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        if (m == 1 && !own2) break;
        const long long nd = nd0 + m;
        const unsigned mk = MASK_OUT ? (unsigned)a.mask[nd] : 0u;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long d = 3 * nd + c;
          const float Ax = (MASK_OUT && ((mk >> c) & 1u)) ? a.dfix * a.x[d] : s[m][c];
          if (EPI == EPI_APPLY) {
            a.y[d] = Ax;
          } else if (EPI == EPI_RESID) {
            a.y[d] = eb[m][c] - Ax;
          } else {
            a.y[d] = ex[m][c] + a.omega * ed[m][c] * (eb[m][c] - Ax);
          }
        }
      }
    }
    buf ^= 1;
  }
  cp_wait<0>();
}

// Register / tile variants, timed by the autotuner: variant 0, 128 threads
// (PY = 8) and the resident blocks per SM (MINB) the register allocation
// allows without spilling (four for K p, three for the residual and
// smoother epilogues); variant 1, 256 threads (PY = 16, less redundant
// element work at tile edges) and two blocks per SM.  Either runs one block
// per (tile, z-chunk), or as a work list (a.wl set): one CTA per resident
// slot, each taking the next item from a counter until none is left, so
// that CTAs whose items finish early take more and the SMs stay busy to the
// end; the last CTA to finish resets the counters for the next launch.
// An item computes exactly what the block of the same tile and chunk
// computes, so both forms give the same bits.
template <int EPI, int MINB, int PY>
__global__ void __launch_bounds__(PX * PY, MINB)
    k_apply3_pair(PairArgs a, WhtPair kb) {
  extern __shared__ __align__(16) unsigned char pair_smem[];
  __shared__ int s_item;
  PairSmem<PY>& sm = *reinterpret_cast<PairSmem<PY>*>(pair_smem);
  const int tx = threadIdx.x % PX, ty = threadIdx.x / PX;
  // does the tile's node-column range hold a fixed DOF (set up once)
  auto tile_flag = [&](int bx, int by) {
    const int i = bx * POX - 1 + 2 * tx, j = by * PairGeo<PY>::POY - 1 + ty;
    bool flag = a.colfix == nullptr;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int n = 0; n < 3; ++n)
        if (a.colfix && i + n >= 0 && i + n < a.g.nnx && j + r >= 0 && j + r < a.g.nny)
          flag |= a.colfix[(i + n) + (long long)a.g.nnx * (j + r)] != 0;
    return flag;
  };
  // all threads of a block must take the same branch (both contain
  // __syncthreads), so the decision is block-wide
  auto tile = [&](int bx, int by, int bz, bool flag) {
    if (!__syncthreads_or(flag))
      pair_loop<EPI, 0, PY>(a, kb, sm, bx, by, bz);
    else if (a.clean_inputs)
      pair_loop<EPI, 2, PY>(a, kb, sm, bx, by, bz);
    else
      pair_loop<EPI, 1, PY>(a, kb, sm, bx, by, bz);
  };
  if (a.wl == nullptr) {
    const bool flag = tile_flag(blockIdx.x, blockIdx.y);
    // (the column flags are set up once; everything below reads the vectors
    // of preceding kernels)
    pdl_wait();
    tile(blockIdx.x, blockIdx.y, blockIdx.z, flag);
  } else {
    pdl_wait();
    for (;;) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(a.wl, 1u);
      __syncthreads();
      const int item = s_item;
      if (item >= a.nitems) break;
      const int bx = item % a.gx, rest = item / a.gx;
      const int by = rest % a.gy, bz = rest / a.gy;
      tile(bx, by, bz, tile_flag(bx, by));
      __syncthreads();   // shared memory (and s_item) is reused by the next item
    }
    if (threadIdx.x == 0) {
      __threadfence();
      // every CTA has taken its last item before it counts itself done, so
      // the last one may reset the hand-out counter
      if (atomicAdd(a.wl + 1, 1u) == gridDim.x - 1) {
        atomicExch(a.wl, 0u);
        atomicExch(a.wl + 1, 0u);
      }
    }
  }
  pdl_launch_dependents();
}

__global__ void k_colfix(GridP g, const uint8_t* __restrict__ mask, uint8_t* __restrict__ colfix) {
  const long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncol = (long long)g.nnx * g.nny;
  if (col >= ncol) return;
  unsigned any = 0u;
  for (int k = 0; k < g.nnz; ++k) any |= mask[col + ncol * k];
  colfix[col] = any ? 1 : 0;
}

}  // namespace

cudaError_t launch_colfix(const GridP& g, const uint8_t* mask, uint8_t* colfix, cudaStream_t s) {
  const long long ncol = (long long)g.nnx * g.nny;
  if (ncol <= 0) return cudaSuccess;
  k_colfix<<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(g, mask, colfix);
  return cudaGetLastError();
}

template <int EPI, int V>
struct PairVar {
  static constexpr int PY = V ? 16 : 8;
  static constexpr int MINB = V ? 2 : (EPI == EPI_APPLY ? 4 : 3);
  static constexpr int NT = PX * PY;
  static constexpr size_t SMEM = sizeof(PairSmem<PY>);
};

template <int EPI, int V>
static auto pair_kernel() {
  return k_apply3_pair<EPI, PairVar<EPI, V>::MINB, PairVar<EPI, V>::PY>;
}

template <int EPI, int V>
static int pair_occupancy() {
  auto kern = pair_kernel<EPI, V>();
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)PairVar<EPI, V>::SMEM) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PairVar<EPI, V>::NT,
                                                    PairVar<EPI, V>::SMEM) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return per_sm;
}

// resident blocks of the pair kernel on the current device (cached per
// device, epilogue and variant)
static long long pair_slots(int epi, int variant) {
  static long long cache[3][2][64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  const int e = epi == EPI_APPLY ? 0 : epi == EPI_RESID ? 1 : 2;
  const int v = variant ? 1 : 0;
  if (cache[e][v][dev] > 0) return cache[e][v][dev];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == 0)
    per_sm = v ? pair_occupancy<EPI_APPLY, 1>() : pair_occupancy<EPI_APPLY, 0>();
  else if (e == 1)
    per_sm = v ? pair_occupancy<EPI_RESID, 1>() : pair_occupancy<EPI_RESID, 0>();
  else
    per_sm = v ? pair_occupancy<EPI_SMOOTH, 1>() : pair_occupancy<EPI_SMOOTH, 0>();
  if (sms <= 0 || per_sm <= 0) return 2 * 152;
  cache[e][v][dev] = (long long)sms * per_sm;
  return cache[e][v][dev];
}

void pair_prepare() {
  // occupancy queries happen here, outside any stream capture
  for (int v = 0; v < 2; ++v) {
    pair_slots(EPI_APPLY, v);
    pair_slots(EPI_RESID, v);
    pair_slots(EPI_SMOOTH, v);
  }
}

bool pair_apply_ok(const ApplyArgs& a) {
  return a.dim == 3 && !a.expl && !a.gal1 && a.wht != nullptr && a.tc == T_F32 &&
         a.tx == T_F32 && a.ty == T_F32 && 3LL * a.g.nn < (1LL << 40);
}

cudaError_t launch_apply_pair(const ApplyArgs& a, cudaStream_t s) {
  if (!pair_apply_ok(a)) return cudaErrorInvalidValue;
  if (a.g.nn <= 0) return cudaSuccess;
  WhtPair kb;
  const float* src = static_cast<const float*>(a.wht);
  for (int q = 0; q < 72; ++q) {
    const float v = src[q];
    (&kb.b[0][0][0])[q] = make_float2(v, v);
  }
  PairArgs p;
  p.g = a.g;
  p.mask = a.mask;
  p.colfix = a.colfix;
  p.coef = static_cast<const float*>(a.coef);
  p.x = static_cast<const float*>(a.x);
  p.y = static_cast<float*>(a.y);
  p.b = static_cast<const float*>(a.b);
  p.dinv = static_cast<const float*>(a.dinv);
  p.omega = (float)a.omega;
  p.dfix = (float)a.dfix;
  p.clean_inputs = a.clean_inputs;
  const int var = (a.variant & 1) ? 1 : 0;
  const bool wl = (a.variant & 2) && a.wl != nullptr;
  const int poy = var ? PairGeo<16>::POY : PairGeo<8>::POY;
  const int gx = (a.g.nnx + POX - 1) / POX, gy = (a.g.nny + poy - 1) / poy;
  // z-chunks: each chunk streams its layers and recomputes one element layer
  // below it; the count is chosen to minimise waves x layers per chunk for
  // the resident-block capacity of the device
  const long long slots = pair_slots(a.epi, var);
  const long long nxy = (long long)gx * gy;
  int best = 1;
  long long best_cost = -1;
  // a chunk length chosen by the autotuner replaces the search
  for (int nzc = 1; a.zsplit <= 0 && nzc <= a.g.nnz; ++nzc) {
    const int zc = (a.g.nnz + nzc - 1) / nzc;
    if ((a.g.nnz + zc - 1) / zc != nzc) continue;
    const long long waves = (nxy * nzc + slots - 1) / slots;
    const long long cost = waves * (zc + 1);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = nzc;
    }
  }
  p.zc = a.zsplit > 0 ? min(a.zsplit, (int)a.g.nnz) : (a.g.nnz + best - 1) / best;
  best = (a.g.nnz + p.zc - 1) / p.zc;
  p.gx = gx;
  p.gy = gy;
  p.nitems = gx * gy * best;
  p.wl = wl ? a.wl : nullptr;
  dim3 grid = wl ? dim3((unsigned)std::min<long long>(slots, p.nitems)) : dim3(gx, gy, best);
#define PAIR_LAUNCH(E, V)                                                                   \
  launch_pdl(pair_kernel<E, V>(), grid, dim3(PairVar<E, V>::NT), PairVar<E, V>::SMEM, s, p, kb)
  switch (a.epi) {
    case EPI_APPLY: return var ? PAIR_LAUNCH(EPI_APPLY, 1) : PAIR_LAUNCH(EPI_APPLY, 0);
    case EPI_RESID: return var ? PAIR_LAUNCH(EPI_RESID, 1) : PAIR_LAUNCH(EPI_RESID, 0);
    default: return var ? PAIR_LAUNCH(EPI_SMOOTH, 1) : PAIR_LAUNCH(EPI_SMOOTH, 0);
  }
#undef PAIR_LAUNCH
  return cudaGetLastError();
}

}  // namespace topo
