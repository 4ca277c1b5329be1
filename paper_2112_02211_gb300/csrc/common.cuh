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
