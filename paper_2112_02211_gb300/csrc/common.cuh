// Device helpers shared by the kernels of the HPS library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hps {

// ---- complex arithmetic on double2 / float2 (x = re, y = im) --------------
__host__ __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cconjmul(double2 a, double2 b) {  // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double2 cinv(double2 a) {
  // 1/a with scaling against overflow (Smith's method)
  if (fabs(a.x) >= fabs(a.y)) {
    double r = a.y / a.x, d = a.x + a.y * r;
    return make_double2(1.0 / d, -r / d);
  } else {
    double r = a.x / a.y, d = a.y + a.x * r;
    return make_double2(r / d, -1.0 / d);
  }
}

__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cinv(float2 a) {
  if (fabsf(a.x) >= fabsf(a.y)) {
    float r = a.y / a.x, d = a.x + a.y * r;
    return make_float2(1.0f / d, -r / d);
  } else {
    float r = a.x / a.y, d = a.y + a.x * r;
    return make_float2(r / d, -1.0f / d);
  }
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Accumulate acc += a * b (complex), in the accumulator's precision.
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, acc.x);
  acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y);
  acc.y = fmaf(a.y, b.x, acc.y);
}

// ---- double-float arithmetic ---------------------------------------------------
// A value a = h + l held as two FP32 numbers with |l| <= ulp(h)/2 (about 48
// significant bits).  Error-free transformations: Knuth's TwoSum, Dekker's
// Fast2Sum (|a| >= |b|) and the FMA-based TwoProduct.  The _rn intrinsics keep
// the compiler from contracting or reassociating these sequences.
struct dfr {
  float h, l;
};
__device__ __forceinline__ dfr df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfr df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfr df_add(dfr a, dfr b) {
  dfr s = df_two_sum(a.h, b.h);
  return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfr df_neg(dfr a) { return {-a.h, -a.l}; }
__device__ __forceinline__ dfr df_mul(dfr a, dfr b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfr df_from_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(dfr a) { return (double)a.h + (double)a.l; }

// Complex double-float, stored as float4 (re.h, im.h, re.l, im.l): 16 bytes.
struct dfc {
  dfr re, im;
};
__device__ __forceinline__ dfc dfc_load(float4 v) { return {{v.x, v.z}, {v.y, v.w}}; }
__device__ __forceinline__ float4 dfc_store(dfc a) { return make_float4(a.re.h, a.im.h, a.re.l, a.im.l); }
__device__ __forceinline__ dfc dfc_zero() { return {{0.f, 0.f}, {0.f, 0.f}}; }
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_sub(dfc a, dfc b) { return {df_add(a.re, df_neg(b.re)), df_add(a.im, df_neg(b.im))}; }
__device__ __forceinline__ dfc dfc_mul(dfc a, dfc b) {
  return {df_add(df_mul(a.re, b.re), df_neg(df_mul(a.im, b.im))), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// conj(a) * b
__device__ __forceinline__ dfc dfc_conjmul(dfc a, dfc b) {
  return {df_add(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_neg(df_mul(a.im, b.re)))};
}
__device__ __forceinline__ dfc dfc_from(double2 v) { return {df_from_double(v.x), df_from_double(v.y)}; }
__device__ __forceinline__ double2 dfc_to_double2(dfc a) { return make_double2(df_to_double(a.re), df_to_double(a.im)); }

// ---- conversions ------------------------------------------------------------
template <class T> struct Real;
template <> struct Real<double2> { using type = double; };
template <> struct Real<float2> { using type = float; };

template <class TO, class FROM> __device__ __forceinline__ TO cvt(FROM v);
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 v) { return v; }
template <> __device__ __forceinline__ double2 cvt<double2, float2>(float2 v) {
  return make_double2((double)v.x, (double)v.y);
}
template <> __device__ __forceinline__ float2 cvt<float2, double2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}

template <> __device__ __forceinline__ float2 cvt<float2, float4>(float4 v) { return make_float2(v.x, v.y); }
template <> __device__ __forceinline__ double2 cvt<double2, float4>(float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
template <> __device__ __forceinline__ float4 cvt<float4, float2>(float2 v) { return make_float4(v.x, v.y, 0.f, 0.f); }
template <> __device__ __forceinline__ float4 cvt<float4, double2>(double2 v) { return dfc_store(dfc_from(v)); }

template <class T> __device__ __forceinline__ T czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

// ---- warp reductions ----------------------------------------------------------
template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Leading dimension of stored matrices: columns padded to a multiple of 4.
__host__ __device__ __forceinline__ long long rup4(long long v) { return (v + 3) / 4 * 4; }

// ---- grid geometry ------------------------------------------------------------
// Face k: axis k/2, sign -1 for even k; opposite face k^1.
struct GridDims {
  int nx, ny, nz;
  __device__ __forceinline__ int neighbor(int leaf, int face) const {
    int ix = leaf % nx, iy = (leaf / nx) % ny, iz = leaf / (nx * ny);
    int d = (face & 1) ? 1 : -1;
    switch (face >> 1) {
      case 0: ix += d; if (ix < 0 || ix >= nx) return -1; break;
      case 1: iy += d; if (iy < 0 || iy >= ny) return -1; break;
      default: iz += d; if (iz < 0 || iz >= nz) return -1; break;
    }
    return ix + nx * (iy + ny * iz);
  }
};

}  // namespace hps
