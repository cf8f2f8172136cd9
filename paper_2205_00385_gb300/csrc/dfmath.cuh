// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// floats (48-bit significand), and every operation runs on the FP32 pipe
// with error-free transformations (TwoSum, FMA-based TwoProduct).  GB300
// executes one float64 FMA per clock per SM against 128 float32 FMAs, so
// float64-accurate arithmetic on long vectors is done this way; float64
// values are split into (hi, lo) and widened back with integer operations.
#pragma once
#include <cuda_runtime.h>

namespace topo {

struct dfl {
  float h, l;
};

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  const float s = a.h + b.h;
  const float bb = s - a.h;
  float e = (a.h - (s - bb)) + (b.h - bb);
  e += a.l + b.l;
  const float h = s + e;
  return {h, e - (h - s)};
}

__device__ __forceinline__ dfl df_neg(dfl a) { return {-a.h, -a.l}; }

__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float h = p + e;
  return {h, e - (h - p)};
}

// double -> (hi, lo) with integer operations: hi keeps the leading 24
// significant bits (truncated), lo the next 24 of the remaining 29.  Values
// outside [2^-100, 2^100] (zero, or far outside the data's range) take the
// conversion instructions instead.
__device__ __forceinline__ dfl split_d(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  if (e < 1023 - 100 || e > 1023 + 100) {
    if (e == 0) return {0.f, 0.f};
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  const unsigned s = (unsigned)(u >> 63) << 31;
  const float h = __uint_as_float(s | ((unsigned)(e - 896) << 23) | (unsigned)((u >> 29) & 0x7FFFFFu));
  const unsigned L = (unsigned)(u & 0x1FFFFFFFu);
  if (L == 0u) return {h, 0.f};
  const int sh = __clz((int)L) - 8;                  // puts the leading one at bit 23
  const unsigned m = sh >= 0 ? (L << sh) : (L >> (-sh));
  const int ef = e - 925 - sh;                       // float exponent field of lo
  if (ef <= 0) return {h, 0.f};                      // below 2^-126: negligible
  return {h, __uint_as_float(s | ((unsigned)ef << 23) | (m & 0x7FFFFFu))};
}

// exact float -> double with integer operations (zero and normal floats)
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xFFu;
  if (ef == 0u) return 0.0;
  if (ef == 0xFFu) return (double)f;
  const unsigned long long d = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(ef + 896u) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// a * b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) { return df_add(df_mul(a, b), c); }

// Dot-product accumulation acc += a * b in the manner of Ogita, Rump and
// Oishi's Dot2: the leading product is formed exactly (FMA TwoProduct) and
// added to acc.h with TwoSum; all error terms collect in acc.l without
// renormalisation (as accurate as a dot product in twice the working
// precision).  Normalise with df_norm before using acc as a pair.
__device__ __forceinline__ void df_dot_acc(dfl& acc, dfl a, dfl b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const float s = acc.h + p;
  const float bb = s - acc.h;
  const float t = (acc.h - (s - bb)) + (p - bb);
  acc.h = s;
  acc.l += t + e;
}
__device__ __forceinline__ dfl df_norm(dfl a) {
  const float h = a.h + a.l;
  return {h, a.l - (h - a.h)};
}

// (hi + lo) rounded to float64: the halves widen exactly, one float64 add
__device__ __forceinline__ double df_to_d(dfl a) { return f2d(a.h) + f2d(a.l); }

// Block sum of NV double-float values: warps reduce in double-float, lane 0
// widens once, warp 0 adds the warp results in float64 in warp order.  The
// result is valid in thread 0.  sh holds at least NV*32 doubles.
template <int NV>
__device__ __forceinline__ void block_sum_df(dfl (&v)[NV], double (&out)[NV], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    dfl x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const dfl y = {__shfl_down_sync(0xffffffffu, x.h, o), __shfl_down_sync(0xffffffffu, x.l, o)};
      x = df_add(x, y);
    }
    if (lane == 0) sh[q * 32 + warp] = df_to_d(x);
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? sh[q * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      out[q] = s;
    }
  }
  __syncthreads();
}

// a > b for normalised pairs
__device__ __forceinline__ bool df_gt(dfl a, dfl b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }

// storage access for float64-accurate values held as float64 or as pairs
__device__ __forceinline__ dfl ld_df(const double* p, long long i) { return split_d(p[i]); }
__device__ __forceinline__ dfl ld_df(const float2* p, long long i) {
  const float2 v = p[i];
  return {v.x, v.y};
}
__device__ __forceinline__ void st_df(double* p, long long i, dfl v) { p[i] = df_to_d(v); }
__device__ __forceinline__ void st_df(float2* p, long long i, dfl v) {
  p[i] = make_float2(v.h, v.l);
}

// value conversions between storage types (pairs round to float32 once)
template <typename TO, typename TI>
__device__ __forceinline__ TO cvt(TI v) {
  return TO(v);
}
template <>
__device__ __forceinline__ float cvt<float, float2>(float2 v) {
  return __fadd_rn(v.x, v.y);
}
template <>
__device__ __forceinline__ float2 cvt<float2, float>(float v) {
  return make_float2(v, 0.f);
}

}  // namespace topo
