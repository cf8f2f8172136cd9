// Float64-accurate hex8 stiffness operator in double-float arithmetic.
//
// GB300 runs float64 at one FMA per clock per SM, 1/128 of the float32
// rate, so the float64 Walsh kernel (k_apply3_col<double>) is bound by the
// FP64 pipe at ~1.3 ms per 5.4M-DOF apply.  Here every value is an unevaluated sum hi + lo of two
// floats (48-bit significand) and all arithmetic runs on the FP32 pipe with
// error-free transformations (TwoSum, FMA-based TwoProduct).  float64 inputs
// are split into (hi, lo) and results widened back with integer bit
// operations, so the FP64 pipe only sees the final additions of the
// epilogue.  The structure (element columns streamed in z, owner-computes
// node sums in shared memory, Walsh blocks) is that of k_apply3_col.
#include <type_traits>

#include "dfmath.cuh"
#include "kernels.h"

namespace topo {

__device__ __forceinline__ void fwht8_df(dfl (&v)[8]) {
#pragma unroll
  for (int hh = 1; hh < 8; hh <<= 1)
#pragma unroll
    for (int a = 0; a < 8; ++a)
      if (!(a & hh)) {
        const dfl u = v[a], w = v[a + hh];
        v[a] = df_add(u, w);
        v[a + hh] = df_add(u, df_neg(w));
      }
}

struct DfBlocks {
  float h[8][3][3], l[8][3][3];
};

constexpr int DX = 16, DY = 8, DOX = DX - 1, DOY = DY - 1;

// S: storage of x, b and y -- float64 (split on load, widened on store) or
// double-float pairs float2 (used as they are)
template <int EPI, typename S>
__global__ void __launch_bounds__(DX * DY)
    k_apply3_df(GridP g, const uint8_t* __restrict__ mask, DfBlocks kb,
                const double* __restrict__ coef, int zc, const S* __restrict__ x,
                S* __restrict__ y, const S* __restrict__ b, double dfix) {
  __shared__ dfl part[2][4][DY][DX][3];
  const int tx = threadIdx.x % DX, ty = threadIdx.x / DX;
  const int x0 = blockIdx.x * DOX, y0 = blockIdx.y * DOY;
  const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.nnz);
  const int ex = x0 - 1 + tx, ey = y0 - 1 + ty;
  const bool col_ok = ex >= 0 && ex < g.nx && ey >= 0 && ey < g.ny;
  const long long plane = (long long)g.nnx * g.nny;

  dfl xb[4][3], xt[4][3], acc[4][3];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[q][c] = {0.f, 0.f};

  auto load_face = [&](int kz, dfl (&f)[4][3]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = ex + (q & 1), j = ey + (q >> 1);
      if (col_ok && kz >= 0 && kz < g.nnz) {
        const long long nd = i + (long long)g.nnx * j + plane * kz;
        const unsigned m = mask[nd];
#pragma unroll
        for (int c = 0; c < 3; ++c)
          f[q][c] = ((m >> c) & 1u) ? dfl{0.f, 0.f} : ld_df(x, 3 * nd + c);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) f[q][c] = {0.f, 0.f};
      }
    }
  };

  load_face(z0 - 1, xb);
  const bool own = tx < DOX && ty < DOY && (x0 + tx) < g.nnx && (y0 + ty) < g.nny;
  int buf = 0;
  for (int ez = z0 - 1; ez < z1; ++ez) {
    load_face(ez + 1, xt);
    dfl ye[8][3];
    if (col_ok && ez >= 0 && ez < g.nz) {
      const dfl ce = split_d(coef[ex + (long long)g.nx * (ey + (long long)g.ny * ez)]);
      dfl X[3][8];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          X[c][q] = xb[q][c];
          X[c][q + 4] = xt[q][c];
        }
        fwht8_df(X[c]);
      }
      dfl Y[3][8];
#pragma unroll
      for (int tau = 0; tau < 8; ++tau) {
        dfl zt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) zt[c] = df_mul(ce, X[c][tau ^ (1 << c)]);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dfl s = {0.f, 0.f};
          bool first = true;
#pragma unroll
          for (int cp = 0; cp < 3; ++cp) {
            if (wht_zero(tau, c, cp)) continue;
            const dfl t = df_mul(dfl{kb.h[tau][c][cp], kb.l[tau][c][cp]}, zt[cp]);
            s = first ? t : df_add(s, t);
            first = false;
          }
          Y[c][tau ^ (1 << c)] = s;
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fwht8_df(Y[c]);
#pragma unroll
        for (int a = 0; a < 8; ++a) ye[a][c] = Y[c][a];
      }
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c) ye[a][c] = {0.f, 0.f};
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        part[buf][q][ty][tx][c] = df_add(acc[q][c], ye[q][c]);
        acc[q][c] = ye[q + 4][c];
        xb[q][c] = xt[q][c];
      }
    __syncthreads();
    if (own && ez >= z0) {
      const long long nd = (x0 + tx) + (long long)g.nnx * (y0 + ty) + plane * ez;
      const unsigned m = mask[nd];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const dfl s = df_add(df_add(df_add(part[buf][3][ty][tx][c], part[buf][2][ty][tx + 1][c]),
                                    part[buf][1][ty + 1][tx][c]),
                             part[buf][0][ty + 1][tx + 1][c]);
        const long long d = 3 * nd + c;
        if constexpr (std::is_same<S, double>::value) {
          if ((m >> c) & 1u) {
            const double Ax = dfix * x[d];
            y[d] = EPI == EPI_RESID ? b[d] - Ax : Ax;
          } else if (EPI == EPI_RESID) {
            // b and K x nearly cancel near convergence: subtract the leading
            // part first (exact when close), then the trailing part
            y[d] = (b[d] - f2d(s.h)) - f2d(s.l);
          } else {
            y[d] = f2d(s.h) + f2d(s.l);
          }
        } else {
          // dfix is 0 or 1, so dfix * x is exact in the pair format
          const dfl Ax = ((m >> c) & 1u) ? (dfix != 0.0 ? ld_df(x, d) : dfl{0.f, 0.f}) : s;
          st_df(y, d, EPI == EPI_RESID ? df_add(ld_df(b, d), df_neg(Ax)) : Ax);
        }
      }
    }
    buf ^= 1;
  }
}

bool df_blocks_ok(const double* wht64) {
  double mx = 0.0;
  for (int q = 0; q < 72; ++q) mx = fmax(mx, fabs(wht64[q]));
  for (int tau = 0; tau < 8; ++tau)
    for (int c = 0; c < 3; ++c)
      for (int cp = 0; cp < 3; ++cp)
        if (wht_zero(tau, c, cp) && fabs(wht64[(tau * 3 + c) * 3 + cp]) > 1e-14 * mx) return false;
  return true;
}

// resident blocks of the pair-storage double-float kernel (cached per device;
// queried at set-up, outside any stream capture)
template <int EPI>
static long long df_slots() {
  static long long cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cache[dev] > 0) return cache[dev];
  int sms = 0, per_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_apply3_df<EPI, float2>, DX * DY, 0) !=
          cudaSuccess ||
      sms <= 0 || per_sm <= 0)
    return 0;
  cache[dev] = (long long)sms * per_sm;
  return cache[dev];
}

void df_prepare() {
  df_slots<EPI_APPLY>();
  df_slots<EPI_RESID>();
}

template <typename S>
static void run_df(const ApplyArgs& a, const DfBlocks& kb, dim3 grid, int zc, cudaStream_t s) {
  if (a.epi == EPI_RESID)
    k_apply3_df<EPI_RESID, S><<<grid, DX * DY, 0, s>>>(
        a.g, a.mask, kb, static_cast<const double*>(a.coef), zc, static_cast<const S*>(a.x),
        static_cast<S*>(a.y), static_cast<const S*>(a.b), a.dfix);
  else
    k_apply3_df<EPI_APPLY, S><<<grid, DX * DY, 0, s>>>(
        a.g, a.mask, kb, static_cast<const double*>(a.coef), zc, static_cast<const S*>(a.x),
        static_cast<S*>(a.y), static_cast<const S*>(a.b), a.dfix);
}

cudaError_t launch_apply_df(const ApplyArgs& a, cudaStream_t s) {
  if (a.dim != 3 || a.expl || a.gal1 || a.tx != a.ty || (a.tx != T_F64 && a.tx != T_D2) ||
      !a.wht || a.epi == EPI_SMOOTH || (a.tx == T_D2 && a.dfix != 0.0 && a.dfix != 1.0))
    return cudaErrorInvalidValue;
  if (a.g.nn <= 0) return cudaSuccess;
  const double* w = static_cast<const double*>(a.wht);
  DfBlocks kb;
  for (int q = 0; q < 72; ++q) {
    const float h = (float)w[q];
    (&kb.h[0][0][0])[q] = h;
    (&kb.l[0][0][0])[q] = (float)(w[q] - (double)h);
  }
  const int gx = (a.g.nnx + DOX - 1) / DOX, gy = (a.g.nny + DOY - 1) / DOY;
  int zc = 16;
  while (zc > 2 && (long long)gx * gy * ((a.g.nnz + zc - 1) / zc) < 2 * 152) zc /= 2;
  // pair storage (the mixed path's accurate products): the chunk length
  // minimising waves x (layers + 1 recomputed) for the queried occupancy
  const long long slots =
      a.tx == T_D2 ? (a.epi == EPI_RESID ? df_slots<EPI_RESID>() : df_slots<EPI_APPLY>()) : 0;
  if (slots > 0) {
    long long best = -1;
    for (int c = 2; c <= a.g.nnz; ++c) {
      const long long blocks = (long long)gx * gy * ((a.g.nnz + c - 1) / c);
      const long long cost = ((blocks + slots - 1) / slots) * (c + 1);
      if (best < 0 || cost < best) {
        best = cost;
        zc = c;
      }
    }
  }
  if (a.zsplit > 0) zc = min(a.zsplit, (int)a.g.nnz);   // chosen by the autotuner
  dim3 grid(gx, gy, (a.g.nnz + zc - 1) / zc);
  if (a.tx == T_D2)
    run_df<float2>(a, kb, grid, zc, s);
  else
    run_df<double>(a, kb, grid, zc, s);
  return cudaGetLastError();
}

}  // namespace topo
