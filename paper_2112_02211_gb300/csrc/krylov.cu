// Restarted GMRES (Saad and Schultz 1986; PETSc KSP GMRES in the paper,
// Sec. 5.2) on the face system, right-preconditioned by the cluster
// block-Jacobi operator, with every Krylov step on the device in FP64:
//
//   z = M^{-1} v_j            (FP64 form: complex FP64; mixed form: complex FP32)
//   w = A z                   (same precision as z, written as FP64)
//   h = V^H w, w -= V h       (classical Gram-Schmidt, applied twice: CGS2)
//   h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j}
//   Givens rotation of the Hessenberg column, residual estimate |g_{j+1}|.
//
// At the end of each cycle x += M^{-1} (V y) and the true residual
// b - A x is recomputed with the FP64 leaf maps.  In the mixed form that
// restart residual is what restores FP64 accuracy: each cycle solves the
// correction equation with the FP32 operator and the FP64 residual drives the
// next cycle (iterative refinement with a GMRES inner solver).
//
// Dot products are formed as fixed-order block partials (1024 entries per
// block, warp shuffles, then a sequential sum over blocks), so results are
// bitwise reproducible run to run.
#include <algorithm>
#include <functional>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr int kT = 256;      // threads per block
constexpr int kE = 4;        // vector entries per thread (1024 per block)
constexpr int kChunk = kT * kE;
constexpr int kG = 4;        // vectors per register group

__device__ __forceinline__ void block_reduce_store(double2 (&acc)[kG], int ng, double2* out) {
  __shared__ double2 red[kT / 32][kG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int g = 0; g < kG; ++g) {
    acc[g].x = warp_sum(acc[g].x);
    acc[g].y = warp_sum(acc[g].y);
  }
  if (lane == 0)
#pragma unroll
    for (int g = 0; g < kG; ++g) red[warp][g] = acc[g];
  __syncthreads();
  if (threadIdx.x < ng) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < kT / 32; ++w) s = cadd(s, red[w][threadIdx.x]);
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

struct VecArgs {
  const double2* V;  // basis: vector j of rhs r at V + (j*nrhs + r)*nf
  double2* w;        // rhs r at w + r*nf
  long long nf;
  int nrhs, nvec, M1, nblk;
  double2* part;     // [rhs][nblk][M1]
  const double2* coef;  // [rhs][cstride]
  int cstride;
  const int* active;
  int self_dot;      // mdot: also w^H w (= ||w||^2) in slot nvec
};

// part = block partials of V_{0..nvec-1}^H w
__global__ void __launch_bounds__(kT) mdot_kernel(VecArgs a) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (a.active && !a.active[rhs]) return;
  const long long base = (long long)blk * kChunk + threadIdx.x;
  const double2* w = a.w + rhs * a.nf;
  double2 wv[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const long long i = base + (long long)e * kT;
    wv[e] = (i < a.nf) ? w[i] : make_double2(0.0, 0.0);
  }
  double2* out = a.part + ((long long)rhs * a.nblk + blk) * a.M1;
  const int nv = a.nvec + a.self_dot;
  for (int g0 = 0; g0 < nv; g0 += kG) {
    const int ng = min(kG, nv - g0);
    double2 acc[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) acc[g] = make_double2(0.0, 0.0);
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      if (g < ng) {
        const double2* v = (g0 + g < a.nvec) ? a.V + ((long long)(g0 + g) * a.nrhs + rhs) * a.nf : w;
#pragma unroll
        for (int e = 0; e < kE; ++e) {
          const long long i = base + (long long)e * kT;
          if (i < a.nf) {
            const double2 vv = v[i];
            acc[g].x += vv.x * wv[e].x + vv.y * wv[e].y;
            acc[g].y += vv.x * wv[e].y - vv.y * wv[e].x;
          }
        }
      }
    }
    block_reduce_store(acc, ng, out + g0);
  }
}

// w -= V coef; then (mode 1) partial dots V^H w, or (mode 2) partial ||w||^2.
__global__ void __launch_bounds__(kT) axpy_kernel(VecArgs a, int mode) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (a.active && !a.active[rhs]) return;
  __shared__ double2 cf[64];
  for (int j = threadIdx.x; j < a.nvec; j += kT) cf[j] = a.coef[(long long)rhs * a.cstride + j];
  __syncthreads();
  const long long base = (long long)blk * kChunk + threadIdx.x;
  double2* w = a.w + rhs * a.nf;
  double2 wv[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const long long i = base + (long long)e * kT;
    wv[e] = (i < a.nf) ? w[i] : make_double2(0.0, 0.0);
  }
#pragma unroll 4
  for (int j = 0; j < a.nvec; ++j) {
    const double2* v = a.V + ((long long)j * a.nrhs + rhs) * a.nf;
    const double2 c = cf[j];
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      const long long i = base + (long long)e * kT;
      if (i < a.nf) {
        const double2 vv = v[i];
        wv[e].x -= c.x * vv.x - c.y * vv.y;
        wv[e].y -= c.x * vv.y + c.y * vv.x;
      }
    }
  }
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const long long i = base + (long long)e * kT;
    if (i < a.nf) w[i] = wv[e];
  }
  double2* out = a.part + ((long long)rhs * a.nblk + blk) * a.M1;
  if (mode == 1) {
    for (int g0 = 0; g0 < a.nvec; g0 += kG) {
      const int ng = min(kG, a.nvec - g0);
      double2 acc[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) acc[g] = make_double2(0.0, 0.0);
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        if (g < ng) {
          const double2* v = a.V + ((long long)(g0 + g) * a.nrhs + rhs) * a.nf;
#pragma unroll
          for (int e = 0; e < kE; ++e) {
            const long long i = base + (long long)e * kT;
            if (i < a.nf) {
              const double2 vv = v[i];
              acc[g].x += vv.x * wv[e].x + vv.y * wv[e].y;
              acc[g].y += vv.x * wv[e].y - vv.y * wv[e].x;
            }
          }
        }
      }
      block_reduce_store(acc, ng, out + g0);
    }
  } else if (mode == 2) {
    double2 acc[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) acc[g] = make_double2(0.0, 0.0);
#pragma unroll
    for (int e = 0; e < kE; ++e) acc[0].x += wv[e].x * wv[e].x + wv[e].y * wv[e].y;
    block_reduce_store(acc, 1, out);
  }
}

// ---------------------------------------------------------------------------
// Double-float variants (mixed form).  The basis is stored as complex
// double-float (float4 per entry, 16 bytes like complex double) and every
// per-entry operation runs on the FP32 pipe; block partials leave as FP64.
// ---------------------------------------------------------------------------
struct DfArgs {
  const float4* V;  // vector j of rhs r at V + (j*nrhs + r)*nf
  float4* w;
  long long nf;
  int nrhs, nvec, M1, nblk;
  double2* part;
  const double2* coef;
  int cstride;
  const int* active;
  int self_dot;     // mdot: also w^H w (= ||w||^2) in slot nvec
};

// Compensated accumulation in the spirit of Ogita, Rump and Oishi's Dot2:
// acc = (s, c) with s the running FP32 sum and c the collected rounding errors.
// A term a*b of two double-float numbers adds its exact hi*hi product (FMA
// TwoProduct), the cross terms a.h*b.l + a.l*b.h in FP32, and the TwoSum error.
struct acc2 {
  float s, c;
};
__device__ __forceinline__ void acc2_madd(acc2& a, dfr x, dfr y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  const dfr t = df_two_sum(a.s, p);
  a.s = t.h;
  a.c = __fadd_rn(a.c, __fadd_rn(t.l, e));
}
__device__ __forceinline__ void acc2_msub(acc2& a, dfr x, dfr y) { acc2_madd(a, {-x.h, -x.l}, y); }
__device__ __forceinline__ dfr acc2_value(acc2 a) { return df_two_sum(a.s, a.c); }

// conj(v) * w accumulated into (re, im)
__device__ __forceinline__ void conjdot_acc(acc2& re, acc2& im, dfc v, dfc w) {
  acc2_madd(re, v.re, w.re);
  acc2_madd(re, v.im, w.im);
  acc2_madd(im, v.re, w.im);
  acc2_msub(im, v.im, w.re);
}

// Block sums of kG double-float complex partials per thread: the partials go
// through shared memory transposed, so each thread finishes with one warp
// reduction for the whole group.  Result per vector as complex double.
__device__ __forceinline__ void block_reduce_store_df(dfc (&part)[kG], int ng, double2* out) {
  __shared__ dfc red[kG][kT];
  __shared__ dfc red2[kG][kT / 32 / kG > 0 ? kT / 32 / kG : 1];
  static_assert(kT % (32 * kG) == 0, "block must split into kG groups of whole warps");
  constexpr int kPer = kT / kG;  // threads per vector in the transposed sum
  const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
  for (int g = 0; g < kG; ++g) red[g][tid] = part[g];
  __syncthreads();
  const int g = tid / kPer, k = tid % kPer;
  dfc a = dfc_zero();
#pragma unroll
  for (int m = 0; m < kT / kPer; ++m) a = dfc_add(a, red[g][k + kPer * m]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dfc other;
    other.re.h = __shfl_xor_sync(0xffffffffu, a.re.h, o);
    other.re.l = __shfl_xor_sync(0xffffffffu, a.re.l, o);
    other.im.h = __shfl_xor_sync(0xffffffffu, a.im.h, o);
    other.im.l = __shfl_xor_sync(0xffffffffu, a.im.l, o);
    a = dfc_add(a, other);
  }
  if (lane == 0) red2[g][k / 32] = a;
  __syncthreads();
  if (k == 0 && g < ng) {
    dfc t = red2[g][0];
    for (int w = 1; w < kPer / 32; ++w) t = dfc_add(t, red2[g][w]);
    out[g] = dfc_to_double2(t);
  }
  __syncthreads();
}

__device__ __forceinline__ dfc shfl_xor_dfc(dfc a, int o) {
  dfc r;
  r.re.h = __shfl_xor_sync(0xffffffffu, a.re.h, o);
  r.re.l = __shfl_xor_sync(0xffffffffu, a.re.l, o);
  r.im.h = __shfl_xor_sync(0xffffffffu, a.im.h, o);
  r.im.l = __shfl_xor_sync(0xffffffffu, a.im.l, o);
  return r;
}

// Warp sums of kG = 4 double-float complex partials per lane, in a fixed order and without
// block barriers: a halving exchange (offset 16: lanes 0-15 keep groups 0, 1 and lanes 16-31
// groups 2, 3; offset 8: one group per 8-lane segment) then three xor steps inside each segment.
// Every lane l returns the warp's sum of group l >> 3.
__device__ __forceinline__ dfc warp_reduce_groups(const dfc (&part)[kG]) {
  static_assert(kG == 4, "halving exchange written for 4 groups");
  const int lane = threadIdx.x & 31;
  const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
  dfc k0 = hi16 ? part[2] : part[0], k1 = hi16 ? part[3] : part[1];
  const dfc s0 = hi16 ? part[0] : part[2], s1 = hi16 ? part[1] : part[3];
  k0 = dfc_add(k0, shfl_xor_dfc(s0, 16));
  k1 = dfc_add(k1, shfl_xor_dfc(s1, 16));
  dfc k = hi8 ? k1 : k0;
  k = dfc_add(k, shfl_xor_dfc(hi8 ? k0 : k1, 8));
  k = dfc_add(k, shfl_xor_dfc(k, 4));
  k = dfc_add(k, shfl_xor_dfc(k, 2));
  k = dfc_add(k, shfl_xor_dfc(k, 1));
  return k;
}

// Partial dots V^H w of this block (one per basis vector, complex double; with nv = nvec + 1
// the last "basis vector" is w itself, giving ||w||^2): per group of kG vectors each warp
// reduces its lanes' partials on its own; one barrier at the end sums the warps in order.
// nv <= 64 (restart <= 60).
__device__ __forceinline__ void df_dots(const DfArgs& a, int rhs, long long base, const dfc (&wv)[kE], double2* out,
                                        int nv) {
  __shared__ dfc wred[kT / 32][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g0 = 0; g0 < nv; g0 += kG) {
    const int ng = min(kG, nv - g0);
    dfc part[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      acc2 re{0.f, 0.f}, im{0.f, 0.f};
      if (g < ng) {
        const float4* v = (g0 + g < a.nvec) ? a.V + ((long long)(g0 + g) * a.nrhs + rhs) * a.nf
                                            : a.w + (long long)rhs * a.nf;
        float4 vv[kE];
#pragma unroll
        for (int e = 0; e < kE; ++e) {
          const long long i = base + (long long)e * kT;
          vv[e] = (i < a.nf) ? v[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < kE; ++e) conjdot_acc(re, im, dfc_load(vv[e]), wv[e]);
      }
      part[g] = {acc2_value(re), acc2_value(im)};
    }
    const dfc sum = warp_reduce_groups(part);
    if ((lane & 7) == 0 && (lane >> 3) < ng) wred[warp][g0 + (lane >> 3)] = sum;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nv; j += kT) {
    dfc t = wred[0][j];
#pragma unroll
    for (int w = 1; w < kT / 32; ++w) t = dfc_add(t, wred[w][j]);
    out[j] = dfc_to_double2(t);
  }
}

__global__ void __launch_bounds__(kT, 4) mdot_df_kernel(DfArgs a) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (a.active && !a.active[rhs]) return;
  const long long base = (long long)blk * kChunk + threadIdx.x;
  const float4* w = a.w + rhs * a.nf;
  dfc wv[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const long long i = base + (long long)e * kT;
    wv[e] = (i < a.nf) ? dfc_load(w[i]) : dfc_zero();
  }
  df_dots(a, rhs, base, wv, a.part + ((long long)rhs * a.nblk + blk) * a.M1, a.nvec + a.self_dot);
}

// w -= V coef; then (mode 1) partial dots V^H w, or (mode 2) partial ||w||^2.
__global__ void __launch_bounds__(kT, 4) axpy_df_kernel(DfArgs a, int mode) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  if (a.active && !a.active[rhs]) return;
  __shared__ dfc cf[64];
  for (int j = threadIdx.x; j < a.nvec; j += kT) cf[j] = dfc_from(a.coef[(long long)rhs * a.cstride + j]);
  __syncthreads();
  const long long base = (long long)blk * kChunk + threadIdx.x;
  float4* w = a.w + rhs * a.nf;
  acc2 wr[kE], wi[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    const long long i = base + (long long)e * kT;
    const dfc x = (i < a.nf) ? dfc_load(w[i]) : dfc_zero();
    wr[e] = {x.re.h, x.re.l};
    wi[e] = {x.im.h, x.im.l};
  }
#pragma unroll 2
  for (int j = 0; j < a.nvec; ++j) {
    const float4* v = a.V + ((long long)j * a.nrhs + rhs) * a.nf;
    const dfc c = cf[j];
    float4 vv[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      const long long i = base + (long long)e * kT;
      vv[e] = (i < a.nf) ? v[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      const dfc x = dfc_load(vv[e]);
      // w -= c x:  re -= c.re x.re - c.im x.im,  im -= c.re x.im + c.im x.re
      acc2_msub(wr[e], c.re, x.re);
      acc2_madd(wr[e], c.im, x.im);
      acc2_msub(wi[e], c.re, x.im);
      acc2_msub(wi[e], c.im, x.re);
    }
  }
  dfc wv[kE];
#pragma unroll
  for (int e = 0; e < kE; ++e) {
    wv[e] = {acc2_value(wr[e]), acc2_value(wi[e])};
    const long long i = base + (long long)e * kT;
    if (i < a.nf) w[i] = dfc_store(wv[e]);
  }
  double2* out = a.part + ((long long)rhs * a.nblk + blk) * a.M1;
  if (mode == 1) {
    df_dots(a, rhs, base, wv, out, a.nvec);
  } else if (mode == 2) {
    dfc part[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) part[g] = dfc_zero();
    acc2 n2{0.f, 0.f};
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      acc2_madd(n2, wv[e].re, wv[e].re);
      acc2_madd(n2, wv[e].im, wv[e].im);
    }
    part[0].re = acc2_value(n2);
    block_reduce_store_df(part, 1, out);
  }
}

// w <- w * invn[rhs] in double-float; c32 (if given) receives the result rounded to complex FP32
// (the normalized double-float's high part), the operand of the tensor-core apply
__global__ void scale_df_kernel(float4* w, long long nf, const double* invn, float2* c32, const int* active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const dfr s = df_from_double(invn[rhs]);
  float4* p = w + rhs * nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const dfc v = dfc_load(p[i]);
    const dfc r = dfc{df_mul(v.re, s), df_mul(v.im, s)};
    p[i] = dfc_store(r);
    if (c32) c32[rhs * nf + i] = make_float2(r.re.h, r.im.h);
  }
}

// dst (double-float) = src (complex double) * invn[rhs]; c32 as in scale_df_kernel
__global__ void scale_copy_df_kernel(const double2* src, float4* dst, long long nf, const double* invn, float2* c32) {
  const int rhs = blockIdx.y;
  const double s = invn[rhs];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    const dfc r = dfc_from(cscale(src[rhs * nf + i], s));
    dst[rhs * nf + i] = dfc_store(r);
    if (c32) c32[rhs * nf + i] = make_float2(r.re.h, r.im.h);
  }
}

// u (complex double) = sum_{j<kmax} y_j v_j, accumulated in double-float; kmax = kcount[rhs]
__global__ void combine_df_kernel(const float4* V, int nrhs, long long nf, const int* kcount, int m, const double2* y,
                                  double2* u) {
  const int rhs = blockIdx.y;
  const int kmax = kcount[rhs];
  __shared__ dfc ys[64];
  for (int j = threadIdx.x; j < kmax; j += blockDim.x) ys[j] = dfc_from(y[(long long)rhs * m + j]);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    dfc s = dfc_zero();
    for (int j = 0; j < kmax; ++j) s = dfc_add(s, dfc_mul(ys[j], dfc_load(V[((long long)j * nrhs + rhs) * nf + i])));
    u[rhs * nf + i] = dfc_to_double2(s);
  }
}

// out[rhs][i] (=|+=) sum over blocks of part[rhs][blk][i].  One CTA per
// (i, rhs): thread t sums blocks t, t+256, ... in order, then a fixed shuffle
// tree and a fixed sum over warps, so the result is the same on every run.
__global__ void __launch_bounds__(kT) reduce_kernel(const double2* part, int nblk, int M1, double2* out, int ostride,
                                                    int accumulate, const int* active) {
  const int i = blockIdx.x, rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double2* p = part + (long long)rhs * nblk * M1 + i;
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += kT) s = cadd(s, p[(long long)b * M1]);
  s.x = warp_sum(s.x);
  s.y = warp_sum(s.y);
  __shared__ double2 red[kT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = red[0];
    for (int w = 1; w < kT / 32; ++w) t = cadd(t, red[w]);
    double2* o = out + (long long)rhs * ostride + i;
    *o = accumulate ? cadd(*o, t) : t;
  }
}

struct GivensArgs {
  int nrhs, m, j, M1, nblk;
  const double2* part;  // norm^2 partials in slot 0
  double2* hcol;        // [rhs][M1+1]: h1 (CGS pass 1)
  const double2* h2;    // [rhs][M1]: CGS pass 2
  double2* H;           // [rhs][M1][m]
  double* cs;           // [rhs][m]
  double2* sn;          // [rhs][m]
  double2* g;           // [rhs][M1]
  double* est;          // [rhs]
  double* invn;         // [rhs]
  int* active;          // [rhs]
  int* kcount;          // [rhs]
  const double* target; // [rhs]
  int* any_active;
};

// Finish column j of the Hessenberg matrix, apply the previous rotations, make
// the new one, update g.  One block of 64 threads per right-hand side: the new
// column and the stored rotations are staged in shared memory in parallel,
// thread 0 applies the rotations (a dependent chain) there, and the column is
// written back in parallel.  Requires m + 1 < 64 (restart <= 60).
__global__ void givens_kernel(GivensArgs a) {
  const int rhs = blockIdx.x;
  if (rhs >= a.nrhs || !a.active[rhs]) return;
  __shared__ double2 col[64];
  __shared__ double csv[64];
  __shared__ double2 snv[64];
  const int j = a.j, t = threadIdx.x;
  const double2* hc = a.hcol + (long long)rhs * (a.M1 + 1);
  const double2* h2 = a.h2 + (long long)rhs * a.M1;
  double* cs = a.cs + (long long)rhs * a.m;
  double2* sn = a.sn + (long long)rhs * a.m;
  if (t <= j) col[t] = cadd(hc[t], h2[t]);
  if (t < j) {
    csv[t] = cs[t];
    snv[t] = sn[t];
  }
  __syncthreads();
  if (t == 0) {
    // ||w||^2 was reduced into the spare last slot of hcol
    const double hn = sqrt(hc[a.M1].x);
    col[j + 1] = make_double2(hn, 0.0);
    for (int i = 0; i < j; ++i) {
      const double2 x = col[i], y = col[i + 1];
      col[i] = cadd(cscale(x, csv[i]), cmul(snv[i], y));
      const double2 sc = make_double2(snv[i].x, -snv[i].y);
      col[i + 1] = csub(cscale(y, csv[i]), cmul(sc, x));
    }
    const double2 x = col[j], y = col[j + 1];
    const double ax = sqrt(cabs2(x)), den = sqrt(cabs2(x) + cabs2(y));
    double c;
    double2 sv;
    if (ax == 0.0) {
      c = 0.0;
      sv = make_double2(1.0, 0.0);
    } else {
      c = ax / den;
      const double2 ph = cscale(x, 1.0 / ax);
      sv = cscale(cmul(ph, make_double2(y.x, -y.y)), 1.0 / den);
    }
    cs[j] = c;
    sn[j] = sv;
    col[j] = cadd(cscale(x, c), cmul(sv, y));
    col[j + 1] = make_double2(0.0, 0.0);
    double2* g = a.g + (long long)rhs * a.M1;
    const double2 gj = g[j];
    g[j + 1] = make_double2(-(sv.x * gj.x + sv.y * gj.y), -(sv.x * gj.y - sv.y * gj.x));  // -conj(s) g_j
    g[j] = cscale(gj, c);
    const double e = sqrt(cabs2(g[j + 1]));
    a.est[rhs] = e;
    a.kcount[rhs] = j + 1;
    const bool breakdown = !(hn > 1e-300 * fmax(1.0, den));
    a.invn[rhs] = breakdown ? 0.0 : 1.0 / hn;
    if (breakdown || e <= a.target[rhs] || j + 1 >= a.m) {
      a.active[rhs] = 0;
    } else {
      atomicOr(a.any_active, 1);
    }
  }
  __syncthreads();
  double2* Hc = a.H + (long long)rhs * a.M1 * a.m;  // Hc[i*m + j]
  if (t <= j + 1) Hc[t * a.m + j] = col[t];
}

// w <- w * invn[rhs]
__global__ void scale_kernel(double2* w, long long nf, int nrhs, const double* invn, const int* active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double s = invn[rhs];
  double2* p = w + rhs * nf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x)
    p[i] = cscale(p[i], s);
}

// dst = src * invn[rhs]
__global__ void scale_copy_kernel(const double2* src, double2* dst, long long nf, const double* invn) {
  const int rhs = blockIdx.y;
  const double s = invn[rhs];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x)
    dst[rhs * nf + i] = cscale(src[rhs * nf + i], s);
}

// y = H(0:k,0:k)^{-1} g(0:k) per rhs (upper triangular after the rotations).
__global__ void lsq_kernel(int nrhs, int m, int M1, const double2* H, const double2* g, const int* kcount, double2* y) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  const int k = kcount[rhs];
  const double2* Hc = H + (long long)rhs * M1 * m;
  double2* yr = y + (long long)rhs * m;
  for (int i = 0; i < m; ++i) yr[i] = make_double2(0.0, 0.0);
  for (int i = k - 1; i >= 0; --i) {
    double2 s = g[(long long)rhs * M1 + i];
    for (int l = i + 1; l < k; ++l) s = csub(s, cmul(Hc[i * m + l], yr[l]));
    const double2 d = Hc[i * m + i];
    yr[i] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cmul(s, cinv(d));
  }
}

// u = sum_{j<kmax} y_j v_j, kmax = kcount[rhs]
__global__ void combine_kernel(const double2* V, int nrhs, long long nf, const int* kcount, int m, const double2* y,
                               double2* u) {
  const int rhs = blockIdx.y;
  const int kmax = kcount[rhs];
  __shared__ double2 ys[64];
  for (int j = threadIdx.x; j < kmax; j += blockDim.x) ys[j] = y[(long long)rhs * m + j];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nf; i += (long long)gridDim.x * blockDim.x) {
    double2 s = make_double2(0.0, 0.0);
    for (int j = 0; j < kmax; ++j) {
      const double2 v = V[((long long)j * nrhs + rhs) * nf + i];
      cfma(s, ys[j], v);
    }
    u[rhs * nf + i] = s;
  }
}

template <class T>
__global__ void xpy_kernel(double2* x, const T* z, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] = cadd(x[i], cvt<double2>(z[i]));
}

// Second Gram-Schmidt pass only where needed: after one classical pass w' = w - V h, the
// computed w' is orthogonal to V up to about eps ||w|| / ||w'||, so a second pass is taken when
// the first cancelled most of w -- Rutishauser's criterion (1967), ||w'|| < ||w|| / 10, which
// bounds the loss of orthogonality per step by ~10 eps.  (The stricter DGKS threshold 1/sqrt(2)
// would fire at every step here: w = A v_j = v_j + Pi R v_j, and removing the v_j component
// alone takes about half of the energy.)  hcol[j+1] holds ||w||^2 (from the first dot pass),
// hcol[M1] ||w'||^2.  Steps that skip the second pass get h2 = 0.
__global__ void reorth_kernel(int nrhs, int j, int M1, const double2* hcol, const int* active, int* reorth, double2* h2,
                            int* nreorth) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  const double2* hc = hcol + (long long)rhs * (M1 + 1);
  const bool act = active[rhs] != 0;
  const bool need = act && hc[M1].x < 0.01 * hc[j + 1].x;
  reorth[rhs] = need ? 1 : 0;
  if (need) atomicAdd(nreorth, 1);
  else if (act)
    for (int t = 0; t <= j; ++t) h2[(long long)rhs * M1 + t] = make_double2(0.0, 0.0);
}

// norms[rhs] = ||x_rhs||_2 from block partials
__global__ void norm_partial_kernel(const double2* x, long long nf, int nblk, double* part) {
  const int rhs = blockIdx.y, blk = blockIdx.x;
  double s = 0.0;
  for (long long i = (long long)blk * blockDim.x + threadIdx.x; i < nf; i += (long long)nblk * blockDim.x) {
    const double2 v = x[rhs * nf + i];
    s += v.x * v.x + v.y * v.y;
  }
  s = warp_sum(s);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[(long long)rhs * nblk + blk] = t;
  }
}

__global__ void norm_final_kernel(const double* part, int nblk, int nrhs, double* out) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(long long)rhs * nblk + b];
  out[rhs] = sqrt(s);
}

}  // namespace

// ---------------------------------------------------------------------------
int krylov_alloc(hps_handle* h, int nrhs, long long nvec) {
  KrylovSpace& k = h->ks;
  const int m = h->opt.restart;
  if (nvec <= 0) nvec = h->nf;
  if (k.V && k.nrhs >= nrhs && k.m == m && k.nf == nvec) return HPS_OK;
  krylov_free(h);
  k.m = m;
  k.nrhs = nrhs;
  k.nf = nvec;
  k.nblk = (int)((nvec + kChunk - 1) / kChunk);
  const int M1 = m + 1;
  const long long nf = nvec;
  size_t total = 0;
  auto alloc = [&](void** p, size_t bytes) -> int {
    bytes = std::max<size_t>(bytes, 16);
    if (h->opt.hbm_budget && h->bytes + total + bytes > h->opt.hbm_budget) {
      set_error("Krylov workspace exceeds the HBM budget");
      return HPS_ENOMEM;
    }
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc failed for the Krylov workspace");
      return HPS_ENOMEM;
    }
    total += bytes;
    return HPS_OK;
  };
  int rc;
  const size_t vb = (size_t)nrhs * nf * sizeof(double2);
  if ((rc = alloc((void**)&k.V, vb * M1))) return rc;
  if ((rc = alloc((void**)&k.x, vb))) return rc;
  if ((rc = alloc((void**)&k.r, vb))) return rc;
  if ((rc = alloc((void**)&k.b, vb))) return rc;
  if ((rc = alloc((void**)&k.u, vb))) return rc;
  if ((rc = alloc(&k.z, vb))) return rc;
  const size_t ts = (size_t)std::max<long long>(1, h->ct.tsize) * nrhs * sizeof(double2);
  if ((rc = alloc(&k.zt, ts))) return rc;
  if ((rc = alloc((void**)&k.part, (size_t)nrhs * k.nblk * M1 * sizeof(double2)))) return rc;
  if ((rc = alloc((void**)&k.hcol, (size_t)nrhs * (M1 + 1) * sizeof(double2)))) return rc;
  if ((rc = alloc((void**)&k.y, (size_t)nrhs * M1 * sizeof(double2)))) return rc;  // also h2
  if ((rc = alloc((void**)&k.H, (size_t)nrhs * M1 * m * sizeof(double2)))) return rc;
  if ((rc = alloc((void**)&k.cs, (size_t)nrhs * m * sizeof(double)))) return rc;
  if ((rc = alloc((void**)&k.sn, (size_t)nrhs * m * sizeof(double2)))) return rc;
  if ((rc = alloc((void**)&k.g, (size_t)nrhs * M1 * sizeof(double2)))) return rc;
  if ((rc = alloc((void**)&k.est, (size_t)nrhs * 4 * sizeof(double)))) return rc;  // est, invn, target, norms
  if ((rc = alloc((void**)&k.nrm, (size_t)nrhs * std::max(256, k.nblk) * sizeof(double)))) return rc;
  // active[nrhs], kcount[nrhs], any_active, status, reorth[nrhs], nreorth
  if ((rc = alloc((void**)&k.active, (size_t)(3 * nrhs + 3) * sizeof(int)))) return rc;
  k.status = k.active + 2 * nrhs + 1;
  k.bytes = total;
  return HPS_OK;
}

namespace {
void destroy_graph(hps_handle* h) {
  CycleGraph& g = h->ks.graph;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  h->prof.release(g.recs);
  g = CycleGraph();
}
}  // namespace

void krylov_drop_graph(hps_handle* h) { destroy_graph(h); }

void krylov_free(hps_handle* h) {
  destroy_graph(h);
  h->prof.destroy();
  KrylovSpace& k = h->ks;
  void* ptrs[] = {k.V, k.x, k.r, k.b, k.u, k.z, k.zt, k.part, k.hcol, k.y, k.H, k.cs, k.sn, k.g, k.est, k.nrm, k.active,
                  k.s_dev, k.t_dev, k.f_dev};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  k = KrylovSpace();
}

namespace {

// ||x_rhs|| of every right-hand side into out (host); also copies n_ints ints from dev_ints
// (when given) in the same synchronization.
int vec_norms(hps_handle* h, const double2* x, int nrhs, std::vector<double>& out, cudaStream_t st,
              const int* dev_ints = nullptr, int* host_ints = nullptr, int n_ints = 0) {
  KrylovSpace& k = h->ks;
  const int nblk = 256;
  double* part = k.nrm;
  double* res = k.est + 3 * k.nrhs;
  norm_partial_kernel<<<dim3(nblk, nrhs), 256, 0, st>>>(x, k.nf, nblk, part);
  HPS_CUDA_TRY(cudaGetLastError());
  norm_final_kernel<<<(nrhs + 63) / 64, 64, 0, st>>>(part, nblk, nrhs, res);
  HPS_CUDA_TRY(cudaGetLastError());
  h->prof.launches += 2;
  out.resize(nrhs);
  HPS_CUDA_TRY(cudaMemcpyAsync(out.data(), res, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (dev_ints)
    HPS_CUDA_TRY(cudaMemcpyAsync(host_ints, dev_ints, n_ints * sizeof(int), cudaMemcpyDeviceToHost, st));
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  return HPS_OK;
}

}  // namespace

// Restarted GMRES (right preconditioning) with the operators of `ops`.  Per restart cycle:
// the host sets the per-RHS targets, then the first basis vector and up to m Arnoldi steps run
// on the device without any host synchronization -- replayed from a CUDA graph captured once
// per configuration, in which every kernel of step j + 1 returns at once when step j left no
// right-hand side active (device gate) -- then x += M^{-1} V y and the FP64 true residual,
// whose norms (and the step counts) are the cycle's one read-back.
int gmres_core(hps_handle* h, const GmresOps& ops, bool mixed, const double2* b, double2* x, int nrhs, double tol,
               hps_solve_info* info, cudaStream_t st, SolveFlags fl) {
  const auto t0 = std::chrono::steady_clock::now();
  int rc = krylov_alloc(h, nrhs, ops.n);
  if (rc) return rc;
  KrylovSpace& k = h->ks;
  const int m = k.m, M1 = m + 1;
  const long long nf = ops.n;
  const size_t vb = (size_t)nrhs * nf * sizeof(double2);
  double* est = k.est;
  double* invn = k.est + nrhs;
  double* target = k.est + 2 * nrhs;
  int* active = k.active;
  int* kcount = k.active + nrhs;
  int* any_active = k.active + 2 * nrhs;
  int* reorth = k.active + 2 * nrhs + 2;
  int* nreorth = k.active + 3 * nrhs + 2;
  double2* h2 = k.y;  // pass-2 coefficients reuse the y buffer until the cycle ends
  const int gblk = std::min<long long>(4 * h->nsm, (nf + 255) / 256);
  const dim3 vgrid(gblk, nrhs);
  const bool pc = ops.pc;
  const bool cgs2 = fl.cgs2;
  // unpreconditioned mixed form with a complex-FP32 operand: v_j is also kept rounded in z
  float2* vc32 = (mixed && !pc && ops.c64_operand) ? (float2*)k.z : nullptr;

  // first basis vector of the cycle: v_0 = r / ||r||
  auto first_vector = [&](cudaStream_t s) -> int {
    if (mixed)
      scale_copy_df_kernel<<<vgrid, 256, 0, s>>>(k.r, (float4*)k.V, nf, invn, vc32);
    else
      scale_copy_kernel<<<vgrid, 256, 0, s>>>(k.r, k.V, nf, invn);
    HPS_CUDA_TRY(cudaGetLastError());
    h->prof.launches += 1;
    return HPS_OK;
  };
  // Arnoldi step j: w = A M^{-1} v_j, orthogonalized against v_0..v_j, the Hessenberg
  // column rotated, v_{j+1} = w / h_{j+1,j}
  auto step = [&](int j, cudaStream_t s) -> int {
    h->prof.step = j;
    double2* vj = k.V + (long long)j * nrhs * nf;
    double2* w = k.V + (long long)(j + 1) * nrhs * nf;
    const VType vt = mixed ? VType::DF : VType::C128, zt = mixed ? VType::C64 : VType::C128;
    if (pc) {
      HPS_CUDA_TRY(ops.precond(vt, vj, zt, k.z, nrhs, s));
      HPS_CUDA_TRY(ops.apply(zt, k.z, vt, w, nrhs, s));
    } else if (vc32) {
      HPS_CUDA_TRY(ops.apply(VType::C64, vc32, vt, w, nrhs, s));
    } else {
      HPS_CUDA_TRY(ops.apply(vt, vj, vt, w, nrhs, s));
    }
    VecArgs va;
    va.V = k.V;
    va.w = w;
    va.nf = nf;
    va.nrhs = nrhs;
    va.nvec = j + 1;
    va.M1 = M1;
    va.nblk = k.nblk;
    va.part = k.part;
    va.active = active;
    va.self_dot = 0;
    DfArgs da;
    da.V = (const float4*)k.V;
    da.w = (float4*)w;
    da.nf = nf;
    da.nrhs = nrhs;
    da.nvec = j + 1;
    da.M1 = M1;
    da.nblk = k.nblk;
    da.part = k.part;
    da.active = active;
    da.self_dot = 0;
    const dim3 bgrid(k.nblk, nrhs);
    auto mdot = [&](const int* act, int self) {
      va.active = da.active = act;
      va.self_dot = da.self_dot = self;
      if (mixed) mdot_df_kernel<<<bgrid, kT, 0, s>>>(da);
      else mdot_kernel<<<bgrid, kT, 0, s>>>(va);
      va.self_dot = da.self_dot = 0;
    };
    auto axpy = [&](const int* act, const double2* coef, int cstride, int mode) {
      va.active = da.active = act;
      va.coef = da.coef = coef;
      va.cstride = da.cstride = cstride;
      if (mixed) axpy_df_kernel<<<bgrid, kT, 0, s>>>(da, mode);
      else axpy_kernel<<<bgrid, kT, 0, s>>>(va, mode);
    };
    auto reduce = [&](int n, double2* out, int ostride, const int* act) {
      reduce_kernel<<<dim3(n, nrhs), kT, 0, s>>>(k.part, k.nblk, M1, out, ostride, 0, act);
    };
    cudaEvent_t ev_arn = h->prof.begin(s);
    if (cgs2) {
      // classical Gram-Schmidt twice: dots; update + dots; update + norm
      mdot(active, 0);
      reduce(j + 1, k.hcol, M1 + 1, active);
      axpy(active, k.hcol, M1 + 1, 1);
      reduce(j + 1, h2, M1, active);
      axpy(active, h2, M1, 2);
      reduce(1, k.hcol + M1, M1 + 1, active);
      h->prof.launches += 6;
    } else {
      // one pass (dots and ||w||^2; update + norm), the second only where the norm test asks
      mdot(active, 1);
      reduce(j + 2, k.hcol, M1 + 1, active);
      axpy(active, k.hcol, M1 + 1, 2);
      reduce(1, k.hcol + M1, M1 + 1, active);
      reorth_kernel<<<(nrhs + 63) / 64, 64, 0, s>>>(nrhs, j, M1, k.hcol, active, reorth, h2, nreorth);
      mdot(reorth, 0);
      reduce(j + 1, h2, M1, reorth);
      axpy(reorth, h2, M1, 2);
      reduce(1, k.hcol + M1, M1 + 1, reorth);
      h->prof.launches += 9;
    }
    HPS_CUDA_TRY(cudaGetLastError());
    HPS_CUDA_TRY(cudaMemsetAsync(any_active, 0, sizeof(int), s));
    GivensArgs ga;
    ga.nrhs = nrhs;
    ga.m = m;
    ga.j = j;
    ga.M1 = M1;
    ga.nblk = k.nblk;
    ga.part = k.part;
    ga.hcol = k.hcol;
    ga.h2 = h2;
    ga.H = k.H;
    ga.cs = k.cs;
    ga.sn = k.sn;
    ga.g = k.g;
    ga.est = est;
    ga.invn = invn;
    ga.active = active;
    ga.kcount = kcount;
    ga.target = target;
    ga.any_active = any_active;
    givens_kernel<<<nrhs, 64, 0, s>>>(ga);
    HPS_CUDA_TRY(cudaGetLastError());
    if (mixed) scale_df_kernel<<<vgrid, 256, 0, s>>>((float4*)w, nf, invn, vc32, active);
    else scale_kernel<<<vgrid, 256, 0, s>>>(w, nf, nrhs, invn, active);
    HPS_CUDA_TRY(cudaGetLastError());
    h->prof.end(HPS_PHASE_ARNOLDI, ev_arn, s);
    h->prof.launches += 2;
    h->prof.step = -1;
    return HPS_OK;
  };

  // the tensor-core kernels' error word starts clear for every solve
  if (h->tc_error) HPS_CUDA_TRY(cudaMemsetAsync(h->tc_error, 0, sizeof(int), st));
  std::vector<double> bnorm, rnorm;
  if ((rc = vec_norms(h, b, nrhs, bnorm, st))) return rc;
  if (fl.x0) {
    HPS_CUDA_TRY(ops.residual(x, b, k.r, nrhs, st));
    if ((rc = vec_norms(h, k.r, nrhs, rnorm, st))) return rc;
  } else {
    HPS_CUDA_TRY(cudaMemsetAsync(x, 0, vb, st));
    HPS_CUDA_TRY(cudaMemcpyAsync(k.r, b, vb, cudaMemcpyDeviceToDevice, st));
    rnorm = bnorm;
  }
  // a residual norm that is not finite ends the solve (it would compare as converged)
  auto finite_norms = [&](const char* where) -> int {
    int nbad = 0, first = -1;
    for (int r = 0; r < nrhs; ++r)
      if (!std::isfinite(rnorm[r]) || !std::isfinite(bnorm[r])) {
        if (first < 0) first = r;
        ++nbad;
      }
    if (nbad == 0) return HPS_OK;
    set_error(std::string("GMRES: non-finite residual norm (") + where + ", " + std::to_string(nbad) + " of " +
              std::to_string(nrhs) + " right-hand sides, the first " + std::to_string(first) + ")");
    return HPS_EBREAKDOWN;
  };
  if ((rc = finite_norms("initial residual"))) return rc;
  int its = 0, cycles = 0;
  long long nre_total = 0;
  const double eps_inner = mixed ? 1e-6 : 0.0;
  std::vector<double> htarget(nrhs), hinv(nrhs);
  std::vector<int> hints(2 * nrhs + 1), hread(3 * nrhs + 3);
  std::vector<double2> g0((size_t)nrhs * M1);
  bool converged = false;
  while (true) {
    bool all = true;
    for (int r = 0; r < nrhs; ++r)
      if (bnorm[r] > 0.0 && rnorm[r] > tol * bnorm[r]) all = false;
    if (all) {
      converged = true;
      break;
    }
    if (its >= h->opt.maxit) break;
    std::fill(hints.begin(), hints.end(), 0);
    std::fill(g0.begin(), g0.end(), make_double2(0.0, 0.0));
    for (int r = 0; r < nrhs; ++r) {
      const bool act = bnorm[r] > 0.0 && rnorm[r] > tol * bnorm[r];
      hints[r] = act ? 1 : 0;  // active; kcount stays 0
      htarget[r] = std::max(0.5 * tol * bnorm[r], eps_inner * rnorm[r]);
      hinv[r] = act ? 1.0 / rnorm[r] : 0.0;
      g0[(size_t)r * M1] = make_double2(act ? rnorm[r] : 0.0, 0.0);
    }
    hints[2 * nrhs] = 1;  // any_active: the first step runs
    HPS_CUDA_TRY(cudaMemcpyAsync(active, hints.data(), hints.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    HPS_CUDA_TRY(cudaMemsetAsync(nreorth, 0, sizeof(int), st));
    HPS_CUDA_TRY(cudaMemcpyAsync(target, htarget.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    HPS_CUDA_TRY(cudaMemcpyAsync(invn, hinv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
    HPS_CUDA_TRY(cudaMemcpyAsync(k.g, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
    const int steps = std::min(m, h->opt.maxit - its);
    const bool use_graph = !fl.no_graph && steps == m;
    bool replayed = false;
    if (use_graph) {
      CycleGraph& gr = k.graph;
      const bool match = gr.exec && gr.nrhs == nrhs && gr.m == m && gr.ops_id == ops.id && gr.mixed == (int)mixed &&
                         gr.pc == (int)pc && gr.c64op == (vc32 != nullptr) && gr.cgs2 == (int)cgs2 &&
                         gr.prof == (int)h->prof.on && gr.n == nf && gr.V == (const void*)k.V;
      if (!match) {
        destroy_graph(h);
        // capture on the handle's own stream (the caller's may be the legacy default stream,
        // which cannot be captured); the graph is launched on the caller's stream
        cudaStream_t cs = h->stream;
        HPS_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        const long long l0 = h->prof.launches;
        const size_t r0 = h->prof.recs.size();
        h->gate = any_active;
        int crc = first_vector(cs);
        for (int j = 0; j < m && crc == HPS_OK; ++j) crc = step(j, cs);
        h->gate = nullptr;
        h->prof.step = -1;
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        std::vector<Profiler::Rec> recs = h->prof.take_recs(r0);
        const long long nl = h->prof.launches - l0;
        h->prof.launches = l0;
        cudaGraphExec_t exec = nullptr;
        cudaError_t ie = cudaSuccess;
        if (crc == HPS_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (crc != HPS_OK || ce != cudaSuccess || ie != cudaSuccess) {
          h->prof.release(recs);
          cudaGetLastError();
          if (crc != HPS_OK) return crc;
          set_error(std::string("capture of the GMRES cycle failed: ") +
                    cudaGetErrorString(ce != cudaSuccess ? ce : ie));
          return HPS_ECUDA;
        }
        gr.exec = exec;
        gr.nrhs = nrhs;
        gr.m = m;
        gr.ops_id = ops.id;
        gr.mixed = mixed;
        gr.pc = pc;
        gr.c64op = vc32 != nullptr;
        gr.cgs2 = cgs2;
        gr.prof = h->prof.on;
        gr.n = nf;
        gr.V = k.V;
        gr.launches = nl;
        gr.recs = std::move(recs);
      }
      HPS_CUDA_TRY(cudaGraphLaunch(gr.exec, st));
      h->prof.launches += gr.launches;
      replayed = true;
    } else {
      if ((rc = first_vector(st))) return rc;
      for (int j = 0; j < steps; ++j) {
        if ((rc = step(j, st))) return rc;
        int hany = 0;
        HPS_CUDA_TRY(cudaMemcpyAsync(&hany, any_active, sizeof(int), cudaMemcpyDeviceToHost, st));
        HPS_CUDA_TRY(cudaStreamSynchronize(st));
        if (!hany) break;
      }
    }
    // x += M^{-1} (V y)
    cudaEvent_t ev_up = h->prof.begin(st);
    lsq_kernel<<<(nrhs + 31) / 32, 32, 0, st>>>(nrhs, m, M1, k.H, k.g, kcount, k.y);
    HPS_CUDA_TRY(cudaGetLastError());
    if (mixed) combine_df_kernel<<<vgrid, 256, 0, st>>>((const float4*)k.V, nrhs, nf, kcount, m, k.y, k.u);
    else combine_kernel<<<vgrid, 256, 0, st>>>(k.V, nrhs, nf, kcount, m, k.y, k.u);
    HPS_CUDA_TRY(cudaGetLastError());
    const long long nall = (long long)nrhs * nf;
    if (pc) {
      if (mixed) {
        HPS_CUDA_TRY(ops.precond(VType::C128, k.u, VType::C64, k.z, nrhs, st));
        xpy_kernel<float2><<<4 * h->nsm, 256, 0, st>>>(x, (const float2*)k.z, nall);
      } else {
        HPS_CUDA_TRY(ops.precond(VType::C128, k.u, VType::C128, k.z, nrhs, st));
        xpy_kernel<double2><<<4 * h->nsm, 256, 0, st>>>(x, (const double2*)k.z, nall);
      }
    } else {
      xpy_kernel<double2><<<4 * h->nsm, 256, 0, st>>>(x, k.u, nall);
    }
    HPS_CUDA_TRY(cudaGetLastError());
    h->prof.end(HPS_PHASE_UPDATE, ev_up, st);
    h->prof.launches += 3;
    // true residual r = b - A x in FP64; its norms, the step counts and the
    // reorthogonalization count are the cycle's read-back
    HPS_CUDA_TRY(ops.residual(x, b, k.r, nrhs, st));
    if ((rc = vec_norms(h, k.r, nrhs, rnorm, st, k.active, hread.data(), 3 * nrhs + 3))) return rc;
    int done = 0;
    for (int r = 0; r < nrhs; ++r) done = std::max(done, hread[nrhs + r]);
    nre_total += hread[3 * nrhs + 2];
    if ((rc = finite_norms("restart residual"))) return rc;
    if (replayed && h->prof.on) h->prof.read_recs(k.graph.recs, done);
    its += done;
    if (h->tc_error) {
      int terr = 0;
      HPS_CUDA_TRY(cudaMemcpy(&terr, h->tc_error, sizeof(int), cudaMemcpyDeviceToHost));
      if (terr) {
        set_error("tensor-core apply: a bounded wait gave up");
        return HPS_ETIMEOUT;
      }
    }
    ++cycles;
    if (done == 0) break;  // nothing was active: no progress possible
  }
  double rel = 0.0;
  for (int r = 0; r < nrhs; ++r)
    if (bnorm[r] > 0.0) rel = std::max(rel, rnorm[r] / bnorm[r]);
  if (info) {
    info->iterations = its;
    info->cycles = cycles;
    info->converged = converged ? 1 : 0;
    info->rel_residual = rel;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->reorth_steps = (int)std::min<long long>(nre_total, 0x7fffffff);
  }
  if (!converged) {
    set_error("GMRES did not reach the tolerance within maxit iterations");
    return HPS_ENOCONV;
  }
  return HPS_OK;
}

// GMRES on the face system (I + Pi R) f = b: apply and preconditioner of
// apply.cu; FP64 residual with the FP64 maps (in lean mode the FP32 maps
// against FP64 vectors).
int gmres_solve(hps_handle* h, int form, const double2* b, double2* x, int nrhs, double tol, hps_solve_info* info,
                cudaStream_t st, bool use_precond, SolveFlags fl) {
  const bool mixed = (form == HPS_FORM_MIXED);
  GmresOps ops;
  ops.n = h->nf;
  ops.pc = h->has_precond && use_precond;
  ops.apply = [h, mixed](VType tin, const void* in, VType tout, void* out, int nrhs, cudaStream_t s) {
    return timed_apply(h, HPS_PHASE_APPLY, mixed, tin, in, tout, out, nullptr, nrhs, false, s);
  };
  ops.precond = [h, mixed](VType tin, const void* in, VType tout, void* out, int nrhs, cudaStream_t s) {
    return launch_precond(h, mixed, tin, in, tout, out, h->ks.zt, nrhs, s, mixed && h->Kc16 != nullptr);
  };
  // restart residual: FP64 maps, or the compensated FP32 maps (lean mode; the mixed form at
  // tolerances >= 1e-8)
  const bool cf_res = h->R64 == nullptr || (mixed && tol >= kCompensatedMinTol && compensated_maps(h));
  ops.residual = [h, cf_res](const double2* xx, const double2* bb, double2* r, int nrhs, cudaStream_t s) {
    return timed_apply(h, HPS_PHASE_RESIDUAL, cf_res, VType::C128, xx, VType::C128, r, bb, nrhs, true, s);
  };
  ops.c64_operand = mixed && apply_tc_eligible(h, nrhs);
  ops.id = 0;
  return gmres_core(h, ops, mixed, b, x, nrhs, tol, info, st, fl);
}

}  // namespace hps
