// Compensated FP32 leaf maps for the memory-lean form: a map M (the ItI map R
// or the body-load map H, Sec. 2.2) is kept as its FP32 rounding M32 plus the
// rounding remainder M - M32 in FP16, scaled per row by sigma_i = max_j of the
// remainder's components, so that M32 + sigma_i lo_ij reproduces M to about
// 2^-24 * 2^-11 ~ 3e-11 relative, at 12 bytes per complex entry instead of 16
// (complex FP64).  Products with complex-double vectors x = x_hi + x_lo (two
// FP32 parts) are accumulated in double-float on the FP32 pipe:
//
//   M32 x_hi   exactly, each real product split by the FMA TwoProduct and
//              summed by Knuth's TwoSum into (sum, error) pairs;
//   M32 x_lo + sigma lo x_hi   in plain FP32 (terms 2^-24 smaller, so their
//              rounding is below the FP64-level target).
//
// This gives the lean form an FP64-accurate restart residual
// b - (I + Pi R) x, an FP64-accurate right-hand side b = tbar - Pi H s and
// complex-double applies, instead of FP32-accurate ones.  Item = (leaf, face):
// the q^2 rows of that face's block; the swap Pi is fused into the store as in
// the other applies (one writer per output slot).
#include <algorithm>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

constexpr int kT = 256;
constexpr int kW = kT / 32;
constexpr int kRPW = 2;  // rows per warp pass
constexpr int kNRMax = 4;  // most right-hand sides per pass over the block
constexpr int kCR = 32;    // rows per work item: a face block is split so that the rows every
                           // pass over the right-hand sides re-reads stay in L2

// (sum, error) pair: value = s + c
struct cacc {
  float s, c;
};
__device__ __forceinline__ void cacc_prod(cacc& a, float x, float y) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  const dfr t = df_two_sum(a.s, p);
  a.s = t.h;
  a.c = __fadd_rn(a.c, __fadd_rn(t.l, e));
}
__device__ __forceinline__ cacc cacc_merge(cacc a, cacc b) {
  const dfr t = df_two_sum(a.s, b.s);
  return {t.h, __fadd_rn(__fadd_rn(a.c, b.c), t.l)};
}
__device__ __forceinline__ cacc cacc_shfl(cacc a, int o) {
  return {__shfl_xor_sync(0xffffffffu, a.s, o), __shfl_xor_sync(0xffffffffu, a.c, o)};
}

struct CfArgs {
  const float2* M;     // FP32 rounding of the maps, per leaf nb x ld row-major
  const __half2* lo;   // remainder / row scale, same layout
  const float* scale;  // per row (leaf * nb + row)
  int ld, ncols, nb, q2;
  long long leaf_stride;  // elements per leaf of M / lo
  GridDims g;
  const double2* x;    // input [rhs][xstride]: face vectors (R) or interior vectors (H)
  long long xstride, xleaf;  // rhs stride, per-leaf offset unit
  double2* y;          // output [rhs][nf]
  const double2* b;    // R: residual mode y = b - (x + Pi R x), or nullptr (apply y = x + Pi R x)
  const double2* t;    // H: boundary data for the boundary-face slots, or nullptr
  long long nf;
  int nrhs, rhs_mode;  // rhs_mode: the map is H (b = tbar - Pi H s) instead of R
  long long nitems;
};

// kNR right-hand sides per pass over the block (1, 2 or 4)
template <int kNR>
__global__ void __launch_bounds__(kT) cf_gemv_kernel(const CfArgs A, int ncp) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* xh = reinterpret_cast<float2*>(smraw);  // kNR x ncp
  float2* xl = xh + kNR * ncp;                    // kNR x ncp
  double2* outs = reinterpret_cast<double2*>(xl + kNR * ncp);  // kNR x kCR
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int q2 = A.q2;
  const int nchunk = (q2 + kCR - 1) / kCR;
  for (long long item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    const long long lf = item / nchunk;
    const int chunk = (int)(item % nchunk);
    const int leaf = (int)(lf / 6), face = (int)(lf % 6);
    const int row0 = chunk * kCR, nrow = min(kCR, q2 - row0);
    const int nbr = A.g.neighbor(leaf, face);
    const long long own = (long long)leaf * A.nb + (long long)face * q2;
    if (nbr < 0) {
      // boundary face: R rows unused (Pi is 0 there); H: the slot takes t (or 0)
      for (int idx = tid; idx < A.nrhs * nrow; idx += kT) {
        const int rr = idx / nrow, j = row0 + idx % nrow;
        const long long o = (long long)rr * A.nf + own + j;
        if (A.rhs_mode) {
          A.y[o] = A.t ? A.t[o] : make_double2(0.0, 0.0);
        } else {
          const double2 xv = A.x[(long long)rr * A.xstride + own + j];
          A.y[o] = A.b ? csub(A.b[o], xv) : xv;
        }
      }
      continue;
    }
    const long long dst = (long long)nbr * A.nb + (long long)(face ^ 1) * q2;
    if (A.rhs_mode && !A.x) {  // no body load: h = 0
      for (int idx = tid; idx < A.nrhs * nrow; idx += kT)
        A.y[(long long)(idx / nrow) * A.nf + dst + row0 + idx % nrow] = make_double2(0.0, 0.0);
      continue;
    }
    const float2* Mb = A.M + (long long)leaf * A.leaf_stride + (long long)(face * q2 + row0) * A.ld;
    const __half2* Lb = A.lo + (long long)leaf * A.leaf_stride + (long long)(face * q2 + row0) * A.ld;
    const float* Sb = A.scale + (long long)leaf * A.nb + (long long)face * q2 + row0;
    for (int r0 = 0; r0 < A.nrhs; r0 += kNR) {
      const int nr = min(kNR, A.nrhs - r0);
      __syncthreads();
      for (int idx = tid; idx < kNR * ncp; idx += kT) {
        const int rr = idx / ncp, c = idx % ncp;
        double2 v = make_double2(0.0, 0.0);
        if (rr < nr && c < A.ncols) v = A.x[(long long)(r0 + rr) * A.xstride + (long long)leaf * A.xleaf + c];
        const float hr = __double2float_rn(v.x), hi = __double2float_rn(v.y);
        xh[idx] = make_float2(hr, hi);
        xl[idx] = make_float2(__double2float_rn(v.x - (double)hr), __double2float_rn(v.y - (double)hi));
      }
      __syncthreads();
      for (int rw = warp * kRPW; rw < nrow; rw += kW * kRPW) {
        cacc are[kRPW][kNR], aim[kRPW][kNR];
        float sre[kRPW][kNR], sim[kRPW][kNR];
        float sig[kRPW];
#pragma unroll
        for (int i = 0; i < kRPW; ++i) {
          sig[i] = (rw + i < nrow) ? Sb[rw + i] : 0.f;
#pragma unroll
          for (int rr = 0; rr < kNR; ++rr) {
            are[i][rr] = {0.f, 0.f};
            aim[i][rr] = {0.f, 0.f};
            sre[i][rr] = 0.f;
            sim[i][rr] = 0.f;
          }
        }
        for (int c = lane * 2; c < ncp; c += 64) {
#pragma unroll
          for (int i = 0; i < kRPW; ++i) {
            if (rw + i >= nrow) continue;
            const float4 m = __ldg(reinterpret_cast<const float4*>(Mb + (long long)(rw + i) * A.ld + c));
            const uint2 lraw = __ldg(reinterpret_cast<const uint2*>(Lb + (long long)(rw + i) * A.ld + c));
            const float2 l0 = __half22float2(*reinterpret_cast<const __half2*>(&lraw.x));
            const float2 l1 = __half22float2(*reinterpret_cast<const __half2*>(&lraw.y));
            const float2 mv[2] = {make_float2(m.x, m.y), make_float2(m.z, m.w)};
            const float2 lv[2] = {make_float2(l0.x * sig[i], l0.y * sig[i]), make_float2(l1.x * sig[i], l1.y * sig[i])};
#pragma unroll
            for (int v = 0; v < 2; ++v) {
#pragma unroll
              for (int rr = 0; rr < kNR; ++rr) {
                const float2 h = xh[rr * ncp + c + v], l = xl[rr * ncp + c + v];
                // main part, exactly: (a + ib)(xr + i xi) with the high parts of x
                cacc_prod(are[i][rr], mv[v].x, h.x);
                cacc_prod(are[i][rr], -mv[v].y, h.y);
                cacc_prod(aim[i][rr], mv[v].x, h.y);
                cacc_prod(aim[i][rr], mv[v].y, h.x);
                // small part: M32 x_lo + sigma lo x_hi
                float tr = __fmaf_rn(mv[v].x, l.x, -__fmul_rn(mv[v].y, l.y));
                tr = __fmaf_rn(lv[v].x, h.x, tr);
                tr = __fmaf_rn(-lv[v].y, h.y, tr);
                float ti = __fmaf_rn(mv[v].x, l.y, __fmul_rn(mv[v].y, l.x));
                ti = __fmaf_rn(lv[v].x, h.y, ti);
                ti = __fmaf_rn(lv[v].y, h.x, ti);
                sre[i][rr] = __fadd_rn(sre[i][rr], tr);
                sim[i][rr] = __fadd_rn(sim[i][rr], ti);
              }
            }
          }
        }
        // warp sums in a fixed order, then value = s + c + small
#pragma unroll
        for (int i = 0; i < kRPW; ++i)
#pragma unroll
          for (int rr = 0; rr < kNR; ++rr) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              are[i][rr] = cacc_merge(are[i][rr], cacc_shfl(are[i][rr], o));
              aim[i][rr] = cacc_merge(aim[i][rr], cacc_shfl(aim[i][rr], o));
              sre[i][rr] = __fadd_rn(sre[i][rr], __shfl_xor_sync(0xffffffffu, sre[i][rr], o));
              sim[i][rr] = __fadd_rn(sim[i][rr], __shfl_xor_sync(0xffffffffu, sim[i][rr], o));
            }
          }
        if (lane == 0) {
#pragma unroll
          for (int i = 0; i < kRPW; ++i)
            if (rw + i < nrow)
#pragma unroll
              for (int rr = 0; rr < kNR; ++rr)
                outs[rr * kCR + rw + i] =
                    make_double2((double)are[i][rr].s + (double)are[i][rr].c + (double)sre[i][rr],
                                 (double)aim[i][rr].s + (double)aim[i][rr].c + (double)sim[i][rr]);
        }
      }
      __syncthreads();
      for (int idx = tid; idx < nr * nrow; idx += kT) {
        const int rr = idx / nrow, jj = idx % nrow, j = row0 + jj;
        const long long o = (long long)(r0 + rr) * A.nf + dst + j;
        const double2 gv = outs[rr * kCR + jj];
        if (A.rhs_mode) {
          A.y[o] = make_double2(-gv.x, -gv.y);
        } else {
          const double2 xv = A.x[(long long)(r0 + rr) * A.xstride + dst + j];
          const double2 yv = cadd(xv, gv);
          A.y[o] = A.b ? csub(A.b[o], yv) : yv;
        }
      }
    }
  }
}

// Row-wise split of an FP64 map into its FP32 rounding (written elsewhere) and the
// remainder in FP16: lo = (M - fl32(M)) / sigma_row, sigma_row = max |remainder
// component| over the row (1 when the row is exactly representable).  One warp per row.
__global__ void split_lo_kernel(const double2* M, long long rows, int ld, __half2* lo, float* scale) {
  const int lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (row >= rows) return;
  const double2* m = M + row * ld;
  float mx = 0.f;
  for (int c = lane; c < ld; c += 32) {
    const double2 v = m[c];
    mx = fmaxf(mx, fabsf((float)(v.x - (double)(float)v.x)));
    mx = fmaxf(mx, fabsf((float)(v.y - (double)(float)v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float sig = mx > 0.f ? mx : 1.f;
  if (lane == 0) scale[row] = sig;
  for (int c = lane; c < ld; c += 32) {
    const double2 v = m[c];
    const float rr = (float)((v.x - (double)(float)v.x) / (double)sig);
    const float ri = (float)((v.y - (double)(float)v.y) / (double)sig);
    lo[row * ld + c] = __floats2half2_rn(rr, ri);
  }
}

template <int kNR>
cudaError_t launch_cf_nr(const hps_handle* h, const CfArgs& A, int ncp, cudaStream_t st) {
  const size_t smem = (size_t)2 * kNR * ncp * sizeof(float2) + (size_t)kNR * kCR * sizeof(double2);
  auto kern = cf_gemv_kernel<kNR>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kT, smem);
  if (e != cudaSuccess) return e;
  const long long grid = std::min<long long>(A.nitems, (long long)h->nsm * std::max(occ, 1));
  kern<<<(unsigned)grid, kT, smem, st>>>(A, ncp);
  ++h->prof.launches;
  return cudaGetLastError();
}

// one pass per group of up to 4 right-hand sides (a single right-hand side computes one)
cudaError_t launch_cf(const hps_handle* h, const CfArgs& A, int ncp, cudaStream_t st) {
  if (A.nrhs == 1) return launch_cf_nr<1>(h, A, ncp, st);
  if (A.nrhs == 2) return launch_cf_nr<2>(h, A, ncp, st);
  return launch_cf_nr<kNRMax>(h, A, ncp, st);
}

}  // namespace

cudaError_t launch_split_lo(const double2* M, long long rows, int ld, __half2* lo, float* scale, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const int wpb = 8;
  split_lo_kernel<<<(unsigned)((rows + wpb - 1) / wpb), 32 * wpb, 0, st>>>(M, rows, ld, lo, scale);
  return cudaGetLastError();
}

bool compensated_maps(const hps_handle* h) { return h->R16lo != nullptr; }

// y = (I + Pi R) x (b == nullptr) or y = b - (I + Pi R) x with the compensated FP32 maps;
// x, y, b complex double [nrhs][nf].
cudaError_t launch_apply_cf(const hps_handle* h, const double2* x, double2* y, const double2* b, int nrhs,
                            cudaStream_t st) {
  if (!h->R32 || !h->R16lo) return cudaErrorInvalidValue;
  CfArgs A;
  A.M = h->R32;
  A.lo = h->R16lo;
  A.scale = h->R16ls;
  A.ld = h->ldR;
  A.ncols = h->nb;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.leaf_stride = (long long)h->nb * h->ldR;
  A.g = GridDims{h->nx, h->ny, h->nz};
  A.x = x;
  A.xstride = h->nf;
  A.xleaf = h->nb;
  A.y = y;
  A.b = b;
  A.t = nullptr;
  A.nf = h->nf;
  A.nrhs = nrhs;
  A.rhs_mode = 0;
  A.nitems = (long long)h->nl * 6 * ((A.q2 + kCR - 1) / kCR);
  return launch_cf(h, A, (int)round_up(h->ldR, 2), st);
}

// b = tbar - Pi (H s) with the compensated FP32 maps H; s: [nrhs][nint] or nullptr.
cudaError_t launch_rhs_cf(const hps_handle* h, const double2* s, const double2* t, double2* b, int nrhs,
                          cudaStream_t st) {
  if (!h->H32 || !h->H16lo) return cudaErrorInvalidValue;
  CfArgs A;
  A.M = h->H32;
  A.lo = h->H16lo;
  A.scale = h->H16ls;
  A.ld = h->ldH;
  A.ncols = h->ni;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.leaf_stride = (long long)h->nb * h->ldH;
  A.g = GridDims{h->nx, h->ny, h->nz};
  A.x = s;
  A.xstride = h->nint;
  A.xleaf = h->ni;
  A.y = b;
  A.b = nullptr;
  A.t = t;
  A.nf = h->nf;
  A.nrhs = nrhs;
  A.rhs_mode = 1;
  A.nitems = (long long)h->nl * 6 * ((A.q2 + kCR - 1) / kCR);
  return launch_cf(h, A, (int)round_up(h->ldH, 2), st);
}

}  // namespace hps
