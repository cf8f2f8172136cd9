// Finest-grid 3D stiffness operator on the 5th-generation tensor cores
// (tcgen05): y = M (sum_e E_e A_e^T KE A_e) M x + dfix (I - M) x and its
// residual / smoother epilogues, in float32 storage.
//
// Per element layer a CTA computes D = X KE^T for 128 elements at once
// (M = 128 rows, one element each; K = 32: the eight corners' (x, y, z, 0)
// records; N = 32: the 24 outputs, padded), then scales row e by E_e and
// sums the rows into the nodes it owns, in a fixed order.
//
// Operand layouts (canonical K-major, no swizzle, core matrices of 8 rows
// of 16 bytes):
//  * A is read in place from the staged node faces.  A face holds the
//    17 x 9 nodes of the tile as 16-byte records, y fastest, so the eight
//    elements of one x-column (rows 8 g .. 8 g + 7) find corner (dx, dy) of
//    their face at 8 consecutive records: each 8 x 16-byte core matrix is
//    contiguous.  One MMA (K = 8, two core matrices along K) covers the
//    corner pair dx = 0, 1 of one (dy, dz): the two are one x-column
//    (144 bytes) apart, and so are consecutive row groups, so LBO = SBO =
//    144 bytes; four MMAs cover (dy, dz).  Core matrices either coincide
//    exactly or are disjoint.
//  * B = KE rearranged to rows n = 3 a_out + c_out (24 used of 32) and
//    columns in the MMAs' corner order, stored with LBO = 128 bytes (next
//    four columns) and SBO = 1024 bytes (next eight rows).
//  * D (128 lanes x 32 columns, float32) lives in tensor memory; warp w
//    reads lanes 32 w .. 32 w + 31 with tcgen05.ld.
// Precision: each float32 operand is split into two TF32 parts (high: the
// leading 11 significant bits; low: the next 11 of the remainder), and
// D = X_hi K_hi + X_lo K_hi + X_hi K_lo, accumulated in float32: about
// 2^-21 relative per element product (float32 arithmetic: 2^-23 to 2^-22).
//
// Waits on the MMA completion barrier are bounded; on expiry the CTA
// records TO_E_TIMEOUT in the status word, waits once more (bounded) for
// its MMAs in flight, frees its tensor memory and returns.
#include <cstring>

#include "kernels.h"
#include "topo_internal.cuh"

namespace topo {
namespace {

constexpr int TCX = 16, TCY = 8;              // elements per tile: x, y
constexpr int TSX = TCX - 1, TSY = TCY - 1;   // owned nodes per tile: x, y
constexpr int FNX = TCX + 1, FNY = TCY + 1;   // face nodes per tile
constexpr int FREC = FNX * FNY;               // 153 records
constexpr int FBYTES = 2560;                  // one face (153 x 16 bytes), rounded to 256
constexpr int CSTR = 28;                      // floats per element row of the contribution buffer
constexpr int TMEM_COLS = 32;
constexpr long long WAIT_LIMIT = 1LL << 22;   // spins of a barrier wait (well under a second)

struct TcArgs {
  GridP g;
  const uint8_t* mask;
  const float* coef;
  const float* bmat;   // [2][32 x 32] float: K_hi, K_lo in the B operand layout
  int zc;
  const float* x;
  float* y;
  const float* b;
  const float* dinv;
  float omega, dfix;
  int* status;
};

struct __align__(1024) TcSmem {
  unsigned char face[2][2][FBYTES];   // [slot][hi, lo]
  float bop[2][32 * 32];              // B operand: K_hi, K_lo
  float contrib[128 * CSTR];          // scaled D rows
  unsigned long long mbar;
  unsigned tmem_base;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// TF32 parts of a float: the leading 11 significant bits, then the next 11
__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
  lo = __uint_as_float(__float_as_uint(v - hi) & 0xFFFFE000u);
}

// shared-memory matrix descriptor: start, leading and stride byte offsets
// (all in 16-byte units), the descriptor version of this architecture,
// no swizzle
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo,
                                                        unsigned sbo) {
  return (unsigned long long)((addr & 0x3FFFFu) >> 4) |
         ((unsigned long long)(lbo >> 4) << 16) | ((unsigned long long)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: D float32, A and B TF32, both K-major, N = 32,
// M = 128
constexpr unsigned IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((32u >> 3) << 17) |
                           ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long a,
                                         unsigned long long b, unsigned acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned phase) {
  unsigned done = 0;
  for (long long spin = 0; spin < WAIT_LIMIT; ++spin) {
    asm volatile(
        "{\n.reg .pred P1;\nmbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n"
        "selp.b32 %0, 1, 0, P1;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int EPI>
__global__ void __launch_bounds__(128) k_apply3_tc(TcArgs a) {
  extern __shared__ unsigned char tc_raw[];
  TcSmem& sm = *reinterpret_cast<TcSmem*>(
      (unsigned char*)(((size_t)tc_raw + 1023) & ~(size_t)1023));
  const GridP& g = a.g;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int X0 = blockIdx.x * TSX - 1, Y0 = blockIdx.y * TSY - 1;
  const int z0 = blockIdx.z * a.zc, z1 = min(z0 + a.zc, g.nnz);
  const long long plane = (long long)g.nnx * g.nny;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&sm.tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&sm.mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  for (int q = t; q < 2 * 32 * 32; q += 128) (&sm.bop[0][0])[q] = a.bmat[q];
  pdl_wait();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = sm.tmem_base;
  const unsigned mbar = smem_u32(&sm.mbar);
  unsigned phase = 0;
  bool failed = false;

  // stage node plane p into ring slot p & 1: hi and lo records, zero outside
  // the grid and at fixed DOFs (the operator acts on M x)
  auto stage = [&](int p) {
    unsigned char* fh = sm.face[p & 1][0];
    unsigned char* fl = sm.face[p & 1][1];
    for (int r = t; r < FREC; r += 128) {
      const int ni = r % FNX, nj = r / FNX;   // x fastest: coalesced loads
      const int gi = X0 + ni, gj = Y0 + nj;
      float v[3] = {0.f, 0.f, 0.f};
      if (p >= 0 && p < g.nnz && gi >= 0 && gi < g.nnx && gj >= 0 && gj < g.nny) {
        const long long nd = (long long)gi + (long long)g.nnx * gj + plane * p;
        const unsigned mk = a.mask[nd];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = ((mk >> c) & 1u) ? 0.f : a.x[3 * nd + c];
      }
      float h[3], l[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) tf32_split(v[c], h[c], l[c]);
      const int off = (ni * FNY + nj) * 16;   // y fastest in the face
      *reinterpret_cast<float4*>(fh + off) = make_float4(h[0], h[1], h[2], 0.f);
      *reinterpret_cast<float4*>(fl + off) = make_float4(l[0], l[1], l[2], 0.f);
    }
  };

  // owned node of this thread (threads >= 105 own none)
  const bool owner = t < TSX * TSY;
  const int oni = 1 + t % TSX, onj = 1 + t / TSX;
  const int ogi = X0 + oni, ogj = Y0 + onj;
  const bool own = owner && ogi < g.nnx && ogj < g.nny;
  // element of this thread's D row: x-column ex = t / 8, y position ey = t % 8
  const int ex = t >> 3, ey = t & 7;
  const int egi = X0 + ex, egj = Y0 + ey;
  const bool elem_in = egi >= 0 && egi < g.nx && egj >= 0 && egj < g.ny;

  float part[3] = {0.f, 0.f, 0.f};   // top-face sum of the layer below, for the owned node
  stage(z0 - 1);
  for (int ez = z0 - 1; ez < z1 && !failed; ++ez) {
    stage(ez + 1);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    const bool layer = ez >= 0 && ez < g.nz;
    float dv[32];
    if (layer) {
      if (t == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const unsigned fb = smem_u32(sm.face[ez & 1][0]), ft = smem_u32(sm.face[(ez + 1) & 1][0]);
        const unsigned bh = smem_u32(sm.bop[0]), bl = smem_u32(sm.bop[1]);
        int q = 0;
#pragma unroll
        for (int s = 0; s < 4; ++s) {   // K-step s: corners (0 / 1, dy = s & 1, dz = s >> 1)
          const unsigned fa = ((s >> 1) ? ft : fb) + (s & 1) * 16;
          const unsigned long long ah = smem_desc(fa, 144, 144);
          const unsigned long long al = smem_desc(fa + FBYTES, 144, 144);
          const unsigned long long kh = smem_desc(bh + 256 * s, 128, 1024);
          const unsigned long long kl = smem_desc(bl + 256 * s, 128, 1024);
          mma_tf32(tmem, ah, kh, q++ > 0);
          mma_tf32(tmem, al, kh, 1);
          mma_tf32(tmem, ah, kl, 1);
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                mbar)
            : "memory");
      }
      if (!mbar_wait(mbar, phase)) {
        failed = true;
        if (lane == 0) atomicExch(a.status, (int)TO_E_TIMEOUT);
      }
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned taddr = tmem + ((unsigned)(32 * warp) << 16);
      unsigned r[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
          "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
          "%28, %29, %30, %31}, [%32];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
            "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
            "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
            "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      const float e = elem_in ? a.coef[egi + (long long)g.nx * (egj + (long long)g.ny * ez)] : 0.f;
#pragma unroll
      for (int q = 0; q < 32; ++q) dv[q] = e * __uint_as_float(r[q]);
    } else {
#pragma unroll
      for (int q = 0; q < 32; ++q) dv[q] = 0.f;
    }
    float* cr = sm.contrib + t * CSTR;
#pragma unroll
    for (int q = 0; q < 24; q += 4)
      *reinterpret_cast<float4*>(cr + q) = make_float4(dv[q], dv[q + 1], dv[q + 2], dv[q + 3]);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (own) {
      // node (oni, onj): bottom corners (dz = 0) of the layer's four elements
      // around it complete plane ez; top corners (dz = 1) start plane ez + 1.
      // Element (oni - 1 + ax, onj - 1 + ay) sees the node as corner
      // (1 - ax, 1 - ay); fixed order ax, ay.
      float bot[3] = {0.f, 0.f, 0.f}, top[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int ay = 0; ay < 2; ++ay)
#pragma unroll
        for (int ax = 0; ax < 2; ++ax) {
          const int row = (oni - 1 + ax) * 8 + (onj - 1 + ay);
          const int cb = (1 - ax) + 2 * (1 - ay);   // corner index, dz = 0
          const float* src = sm.contrib + row * CSTR;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            bot[c] += src[3 * cb + c];
            top[c] += src[3 * (cb + 4) + c];
          }
        }
      if (ez >= z0) {
        const long long nd = (long long)ogi + (long long)g.nnx * ogj + plane * ez;
        const unsigned mk = a.mask[nd];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long d = 3 * nd + c;
          const float s = part[c] + bot[c];
          const float Ax = ((mk >> c) & 1u) ? a.dfix * a.x[d] : s;
          if (EPI == EPI_APPLY) {
            a.y[d] = Ax;
          } else if (EPI == EPI_RESID) {
            a.y[d] = a.b[d] - Ax;
          } else {
            a.y[d] = a.x[d] + a.omega * a.dinv[d] * (a.b[d] - Ax);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) part[c] = top[c];
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  if (failed) {
    // MMAs may still be in flight: one more bounded wait before freeing
    mbar_wait(mbar, phase);
  }
  pdl_launch_dependents();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace

// B operand (K_hi, K_lo) of the tensor-core operator from the float64
// element matrix KE (24 x 24, local DOF 3 a + c of corner a = bx + 2 by + 4 bz):
// row n = 3 a_out + c_out (rows 24..31 zero); column k = 8 s + 4 dx + c_in
// for K-step s = dy + 2 dz (c_in = 3: zero); stored as [row group n / 8]
// [column chunk k / 4][n % 8][k % 4], i.e. LBO = 128 and SBO = 1024 bytes.
void tc_pack_b(const double* KE, float* out /* 2 x 1024 */) {
  for (int q = 0; q < 2048; ++q) out[q] = 0.f;
  for (int n = 0; n < 24; ++n)
    for (int k = 0; k < 32; ++k) {
      const int s = k / 8, dx = (k / 4) & 1, cin = k % 4;
      if (cin == 3) continue;
      const int dy = s & 1, dz = s >> 1;
      const int ain = dx + 2 * dy + 4 * dz;
      const double v = KE[n * 24 + 3 * ain + cin];
      const float f = (float)v;
      unsigned u;
      memcpy(&u, &f, 4);
      u &= 0xFFFFE000u;
      float hi;
      memcpy(&hi, &u, 4);
      const float rem = (float)(v - (double)hi);
      memcpy(&u, &rem, 4);
      u &= 0xFFFFE000u;
      float lo;
      memcpy(&lo, &u, 4);
      const int off = (n / 8) * 256 + (k / 4) * 32 + (n % 8) * 4 + (k % 4);
      out[off] = hi;
      out[1024 + off] = lo;
    }
}

bool tc_apply_ok(const ApplyArgs& a) { return pair_apply_ok(a) && a.bmat != nullptr; }

static size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

cudaError_t tc_prepare() {
  const int bytes = (int)tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_apply3_tc<EPI_APPLY>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply3_tc<EPI_RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply3_tc<EPI_SMOOTH>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return e;
}

cudaError_t launch_apply_tc(const ApplyArgs& a, cudaStream_t s) {
  if (!tc_apply_ok(a) || !a.status) return cudaErrorInvalidValue;
  if (a.g.nn <= 0) return cudaSuccess;
  TcArgs p;
  p.g = a.g;
  p.mask = a.mask;
  p.coef = static_cast<const float*>(a.coef);
  p.bmat = static_cast<const float*>(a.bmat);
  p.x = static_cast<const float*>(a.x);
  p.y = static_cast<float*>(a.y);
  p.b = static_cast<const float*>(a.b);
  p.dinv = static_cast<const float*>(a.dinv);
  p.omega = (float)a.omega;
  p.dfix = (float)a.dfix;
  p.status = a.status;
  const int gx = (a.g.nnx + TSX - 1) / TSX, gy = (a.g.nny + TSY - 1) / TSY;
  // z-chunks: each recomputes one element layer below it; 16 node layers
  // per chunk unless the autotuner chose otherwise
  p.zc = a.zsplit > 0 ? min(a.zsplit, (int)a.g.nnz) : min(16, (int)a.g.nnz);
  dim3 grid(gx, gy, (a.g.nnz + p.zc - 1) / p.zc);
  const size_t smem = tc_smem_bytes();
  switch (a.epi) {
    case EPI_APPLY: return launch_pdl(k_apply3_tc<EPI_APPLY>, grid, dim3(128), smem, s, p);
    case EPI_RESID: return launch_pdl(k_apply3_tc<EPI_RESID>, grid, dim3(128), smem, s, p);
    default: return launch_pdl(k_apply3_tc<EPI_SMOOTH>, grid, dim3(128), smem, s, p);
  }
}

}  // namespace topo
