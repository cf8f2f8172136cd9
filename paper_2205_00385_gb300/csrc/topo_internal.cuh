// Internal definitions shared by the translation units of libtopo.so.
// Nothing here is part of the public ABI (include/topo.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/topo.h"

namespace topo {

constexpr int MAXL = 10;        // multigrid levels
constexpr int MAXB = 16;        // PARM / CARM columns
constexpr int RED_BLOCKS = 608; // fixed grid of deterministic reductions (4 x 152 SMs)
constexpr int RED_THREADS = 256;
constexpr int MAX_STENCIL = 128;

// ---------------------------------------------------------------------------
// Geometry of one grid level.  2D grids have nz = 0 elements and nnz = 1.
// ---------------------------------------------------------------------------
struct GridP {
  int nx, ny, nz;      // elements per axis
  int nnx, nny, nnz;   // nodes per axis
  long long nn, nel;   // node and element counts
};

// Linear springs to ground on free finest-grid DOFs (Sec. 4.3): the
// operator becomes K + S with S diagonal, k[q] at dof[q].
constexpr int MAX_SPRINGS = 4;
struct Springs {
  int n = 0;
  long long dof[MAX_SPRINGS] = {};
  double k[MAX_SPRINGS] = {};
};

// Symmetric element matrices of the stored coarse levels keep their upper
// triangle, row-major packed: entry (r, c), r <= c, at tri_idx(r, c, nd);
// tri_len(nd) = nd (nd + 1) / 2 entries per element.
__host__ __device__ constexpr int tri_len(int nd) { return nd * (nd + 1) / 2; }
__host__ __device__ constexpr int tri_idx(int r, int c, int nd) {
  return r * nd - (r * (r - 1)) / 2 + (c - r);
}
__host__ __device__ constexpr int sym_idx(int r, int c, int nd) {
  return r <= c ? tri_idx(r, c, nd) : tri_idx(c, r, nd);
}
// packed index p -> (r, c)
__host__ __device__ inline void tri_rc(int p, int nd, int& r, int& c) {
  r = 0;
  while (p >= nd - r) {
    p -= nd - r;
    ++r;
  }
  c = r + p;
}

template <int DIM>
struct Geo {
  static constexpr int NPE = 1 << DIM;            // nodes per element
  static constexpr int ND = DIM * NPE;            // DOFs per element
  static constexpr int NB = (DIM == 2) ? 9 : 27;  // nodes in a 3^DIM neighbourhood
};

template <typename T, int ND>
struct KEP {
  T v[ND * ND];
};

// The hex8 KE in the Walsh-Hadamard basis over element corners: eight 3x3
// blocks, b[tau][c][c'] couples X[tau^e_c][c] and X[tau^e_c'][c'], with
// KE = T B T and T the unnormalised transform (see kernels_fe.cu).
template <typename TC>
struct WhtBlocks {
  TC b[8][3][3];
};

// Structural zeros of the Walsh blocks of an isotropic hex8 KE: for a
// single-bit character tau = e_k the translation component k decouples
// (row and column zero); for a two-bit character the third component
// decouples from the other two.  The host verifies these entries vanish
// to rounding and stores them as exact zeros; kernels skip them.
__host__ __device__ constexpr bool wht_zero(int tau, int c, int cp) {
  return (tau == 1 || tau == 2 || tau == 4)
             ? (tau == (1 << c) || tau == (1 << cp))
             : ((tau == 3 || tau == 5 || tau == 6) && c != cp &&
                ((7 ^ tau) == (1 << c) || (7 ^ tau) == (1 << cp)));
}

// in-place unnormalised Walsh-Hadamard transform of 8 corner values
template <typename TC>
__device__ __forceinline__ void fwht8(TC (&v)[8]) {
#pragma unroll
  for (int h = 1; h < 8; h <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & h)) {
        const TC u = v[a], w = v[a + h];
        v[a] = u + w;
        v[a + h] = u - w;
      }
}

struct StencilP {
  int count;
  int d[MAX_STENCIL][3];
  double w[MAX_STENCIL];
};

// Scalar slots in ctx->scal (float64, device)
enum Slot {
  S_RR = 0, S_PQ = 1, S_RZ0 = 2, S_RZ1 = 3, S_NRM = 4, S_TMP = 5, S_COMPL = 6,
  S_OC_L1 = 7, S_OC_L2 = 8, S_OC_VOL = 9, S_OC_DONE = 10, S_CHANGE = 11, S_EPS = 12,
  S_NRM0 = 13, S_NRM1 = 14, S_FNORM2 = 15, S_FLAG = 16,
  S_NSLOTS = 64
};

// Small-matrix area layout in ctx->small (float64, device), offsets in doubles
enum SmallOff {
  SM_KPHI = 0,                      // N_s x N_s
  SM_KPHI_INV = SM_KPHI + 256,      // N_s x N_s
  SM_Z = SM_KPHI_INV + 256,         // N_s (Phi^T t)
  SM_W = SM_Z + 16,                 // N_s (K_Phi^{-1} z), negated
  SM_H = SM_W + 16,                 // GS coefficients
  SM_KR = SM_H + 16,                // m x m
  SM_FR = SM_KR + 256,              // m
  SM_Y = SM_FR + 16,                // m
  SM_H2 = SM_Y + 16,                // GS coefficients of the second pass
  SM_RT = SM_H2 + 16,               // QR factor of the CARM basis, MAXB x N_m (ld MAXB)
  SM_RN = SM_RT + 256,              // norms of the CARM basis columns before orthogonalisation
  SM_U = SM_RN + 16,                // left singular vectors kept by Eq. 21, kq x k (ld MAXB)
  SM_SIG = SM_U + 256,              // singular values of the unit-column basis, descending
  SM_TOTAL = SM_SIG + 16 + 48
};

// I_KCOUNT: columns accepted by the QR of the CARM basis; I_KRED: directions
// kept by the truncated SVD of Eq. 21
// I_TIMEOUT: a bounded device wait expired (TO_E_TIMEOUT)
enum IntSlot { I_KCOUNT = 0, I_STATUS = 1, I_KRED = 2, I_TIMEOUT = 3, I_COARSE = 4, I_NINTS = 16 };

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV float64 values, finished by the last
// block of the grid, which sums the per-block partials in block order.
// ---------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* >= NV*32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[q * 32 + warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[q] = s;  // valid in thread 0
    }
  }
  __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    if (lane == 0) sh[q * 32 + warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : -1e308;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
      v[q] = s;
    }
  }
  __syncthreads();
}

// Programmatic dependent launch.  A kernel launched by launch_pdl() may be
// scheduled while its predecessor in the stream is still running.  It calls
// pdl_wait() before touching memory a preceding kernel writes (it returns
// once every preceding grid has completed and its writes are visible; a
// no-op for an ordinary launch), and pdl_launch_dependents() when its own
// work is issued, which lets the next such kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Writes this block's partials; returns true in all threads of the last block
// to arrive (which may then read all partials).  counter is reset by it.
template <int NV>
__device__ __forceinline__ bool publish_partials(const double (&v)[NV], double* partials,
                                                 unsigned* counter) {
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partials[(size_t)blockIdx.x * NV + q] = v[q];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// In the last block: out[q] = sum over blocks (in order) of partial q.
template <int NV>
__device__ __forceinline__ void finish_sum(const double* partials, unsigned* counter,
                                           double (&out)[NV], double* sh) {
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  // each thread sums a fixed, strided subset of blocks; then a fixed tree
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += partials[(size_t)b * NV + q];
  }
  block_sum<NV>(acc, sh);
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = acc[q];
  if (threadIdx.x == 0) *counter = 0u;
}

template <int NV>
__device__ __forceinline__ void finish_max(const double* partials, unsigned* counter,
                                           double (&out)[NV], double* sh) {
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = -1e308;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = fmax(acc[q], partials[(size_t)b * NV + q]);
  }
  block_max<NV>(acc, sh);
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = acc[q];
  if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace topo

// ---------------------------------------------------------------------------
// Host-side context
// ---------------------------------------------------------------------------
struct LevelBuf {
  topo::GridP g;
  long long n;           // DOFs
  uint8_t* mask;         // per node: bit c set = DOF c fixed
  uint8_t* colfix;       // per node column (i, j): 1 if any of its DOFs is fixed
  void* dinv;            // T[n]
  void* b;               // T[n]
  void* z;               // T[n]
  void* z2;              // T[n]
  void* r;               // T[n]
  void* Kc;              // T[nel*tri_len(ND)], packed upper triangles (stored levels)
  void* S;               // T[DIM*nn * 3^DIM*DIM]: assembled stencil (stored levels)
};

struct to_ctx {
  to_mesh_desc desc;
  int dim, nd, npe, L;
  bool mixed;
  cudaStream_t stream;
  LevelBuf lv[topo::MAXL];
  long long n, nel, nn;
  int nc;                // DOFs of the coarsest level
  // fine-level coefficient arrays
  double *E64, *Eprev64, *dE64, *rho_phys;
  float *E32, *Eprev32, *dE32;
  double *f, *invHs, *oc_a;   // invHs: 1 / row sums of the filter weights
  // f as double-float pairs (mixed path; the long float64-accurate vectors
  // r, p, Phi, KPhi, R, Q, t and the CG iterate are held as pairs there)
  double* fd;
  double* w64;   // float64 scratch of the mixed path without a double-float operator (2D)
  double *oc_lo, *oc_hi;      // OC move-limit bounds of the current update (pairs)
  double *oc_a2, *oc_dv2;     // OC factors and dv as double-float pairs
  // CG
  double *r, *z, *p, *q;
  float *p32, *q32;     // float32 shadows of p and K p (mixed path)
  // PARM / CARM
  double *Phi, *KPhi, *R, *Q, *t;
  int parm_count, parm_head;
  int carm_built;   // directions of the last CARM basis R~ kept by Eq. 21 (0: none built)
  int carm_qr;      // columns of its QR factor (directions before truncation)
  // Galerkin tables (level-1 child matrices Q_c), float64 and float32
  double* Qc64;
  float* Qc32;
  // 3D, >= 3 levels: level 1 applied from the finest moduli (no stored
  // matrices); level 2 formed with the 64 grandchild tables R2
  bool l1_implicit;
  bool df_ok;          // double-float finest-grid operator available (3D)
  double* R2_64;
  float* R2_32;
  double qdiag[192];   // diag(Q_ch) per child and corner, for the level-1 diagonal
  // coarsest level
  void* Adense;
  void* Ainv;
  // reductions and scalars
  double* partials;
  unsigned* counters;
  double* scal;
  double* small;
  int* ints;
  // host state
  double fnorm;
  bool have_density, hier_stale;
  double KE64[576];
  float KE32[576];
  double wht64[72];   // Walsh-Hadamard blocks of KE (3D only)
  float wht32[72];
  topo::StencilP stencil;
  std::string last_error;
  long long launches;
  unsigned prof_mask;   // bit k: time launches of profiling kind k
  // V-cycles captured as CUDA graphs, keyed by their buffers and precision
  struct VGraph {
    const void* rin;
    const void* zout;
    const void* coef;
    int zt;
    bool pre;   // right-hand side and pre-smoothing already in place
    cudaGraphExec_t exec;
    long long launches;
    double bytes;   // algorithmic DRAM bytes of one replay
  };
  double vcycle_bytes;   // algorithmic bytes of the last V-cycle enqueued
  int coarse_t;          // storage of the coarsest matrix and its inverse
  double coarse_shift;   // relative diagonal shift of the coarsest matrix
  int tuned_zc[8];       // autotuned layers per z-chunk per TO_TUNE_* kernel (0: heuristic)
  int tuned_var[8];      // autotuned register variant per TO_TUNE_* kernel (pair kernels)
  int carm_flags;        // TO_CARM_* options of to_carm_build
  bool use_tc;           // float32 finest-grid operator on the tensor cores
  bool fuse_coarse;      // coarse end of the V-cycle as one cluster launch (option)
  bool tall_tiles;       // float32 finest-grid operator with 16-row tiles (option)
  bool work_list;        // float32 finest-grid operator launched as a work list (option)
  topo::Springs springs;  // springs to ground of the finest grid (2D)
  double oc_eta;          // damping exponent of the OC update
  int vf_l0;             // its first level (0: no level qualifies)
  float* tc_bmat;        // its B operand (device, 2 x 1024 floats)
  VGraph vgraph[4];
  int n_vgraph;
  cudaStream_t cap_stream;   // private stream used only for graph capture
  double* host_rr;           // pinned host slot for the CG residual read
  double* host_rr_dev;       // the same slot as the device addresses it (mapped)
  cudaEvent_t rr_event;      // marks that read on the context stream
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
  std::vector<double> ev_bytes;
};

// (topo_api.cu) the OC update with a fixed number of lambda sections and no
// host read, capturable into a graph; same result as to_oc_update
to_status oc_update_enqueue(to_ctx* c, double volfrac, double move, const double* dc_f,
                            const double* dv_f, double* rho, double* change_dev);
// (batch.cu) drops the cached batch graphs that reference c
void batch_forget(const to_ctx* c);

namespace topo {

// Counter slots (ctx->counters, one per reduction site in flight)
// C_PAIR: the float32 pair kernel's work-list counters, two per epilogue
enum Counter { C_DOT = 0, C_MULTI = 1 /* .. +16 */, C_UPD = 20, C_OC = 21, C_SENS = 22,
               C_MAX = 23, C_PAIR = 24 /* .. +6 */, C_NCOUNTERS = 32 };

// --- launch helpers (host) ---
void note_launch(to_ctx* c);
// message returned by to_last_error(NULL)
void set_global_error(const std::string& msg);
cudaError_t check_launch(to_ctx* c, const char* what);
void prof_begin(to_ctx* c, int kind, cudaEvent_t* e0);
void prof_end(to_ctx* c, int kind, cudaEvent_t e0);

inline int nblocks(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace topo
