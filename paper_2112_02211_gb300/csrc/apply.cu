// Per-iteration operators of the HPS face system, as one family of
// HBM-streaming batched GEMV kernels ("items" of q^2 matrix rows each):
//
//  * apply     y = f + Pi (R f)           (leaf ItI maps, Sec. 2.2, eq. (inter))
//  * residual  y = b - (f + Pi (R f))
//  * rhs       b = tbar - Pi (H s)        (body-load response of each leaf)
//  * precond   z = J^{-1} r on 2x2x2 clusters (Sec. 4, Algorithm 4 in face form):
//      stage B  z_ext = r_ext,  t = r_int - B r_ext   (B = internal rows of R~;
//               its own kernel, one thread per row, B stored transposed)
//      stage K  z_int = K_c t                          (K_c = (I + D)^{-1})
//
// An item is (leaf, face) for apply/rhs (rows of that face's block), a leaf
// for B, and for K one slot of a distinct K block against up to 8 clusters
// sharing that block (their t vectors take the place of right-hand sides, so
// a block shared by many clusters is read once per 8 of them).  The swap Pi is fused into the store: the rows
// of leaf tau's face k produce the incoming data of the neighbour across k,
// so every output slot has exactly one writer and no atomics are needed.
// Faces on the boundary of the cube only copy (their rows of R are never
// read).  A CTA stages the item's input vector in shared memory; each warp
// streams RPW matrix rows with 16-byte loads (1 complex double or 2 complex
// floats per lane per load), accumulates in the matrix's precision and
// reduces with warp shuffles.
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

// Returns the CUDA error of expr from a function that returns cudaError_t.
#define HPS_TRY_CUDA_E(expr)          \
  do {                                \
    const cudaError_t e_ = (expr);    \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// One 16-byte load per lane: VPL complex entries of the matrix type, widened to
// the accumulation type.
template <class TM> struct MT;
template <> struct MT<double2> {
  static constexpr int VPL = 1;
  using Acc = double2;
  __device__ static __forceinline__ void load(const double2* p, double2 (&v)[1]) { v[0] = __ldg(p); }
};
template <> struct MT<float2> {
  static constexpr int VPL = 2;
  using Acc = float2;
  __device__ static __forceinline__ void load(const float2* p, float2 (&v)[2]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = make_float2(t.x, t.y);
    v[1] = make_float2(t.z, t.w);
  }
};
template <> struct MT<__half2> {
  static constexpr int VPL = 4;
  using Acc = float2;
  __device__ static __forceinline__ void load(const __half2* p, float2 (&v)[4]) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(p));
    v[0] = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    v[1] = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    v[2] = __half22float2(*reinterpret_cast<const __half2*>(&t.z));
    v[3] = __half22float2(*reinterpret_cast<const __half2*>(&t.w));
  }
};
__device__ __forceinline__ float2 rscale(float2 v, const float* s, long long i) {
  if (!s) return v;
  const float f = s[i];
  return make_float2(v.x * f, v.y * f);
}
__device__ __forceinline__ double2 rscale(double2 v, const float*, long long) { return v; }

struct ItemInfo {
  const void* mat;
  long long xoff;  // base offset of the input vector (per rhs)
  long long ooff;  // base offset of the output (per rhs)
  long long aoff;  // auxiliary offset (neighbour input / residual base)
  int ld, ncols;
  int nrows;       // matrix rows of the item (q^2, or all internal-face rows of a leaf)
  int leaf, face, nbr;
  int mask;        // precond B: internal-face mask of the leaf
};

// ---------------------------------------------------------------------------
// y = f + g (apply) in the output's precision.  Double-float outputs (float4)
// keep f + g exactly (TwoSum), so the identity part of I + Pi R loses nothing.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void sum_out(double2& y, double2 f, double2 g) { y = cadd(f, g); }
__device__ __forceinline__ void sum_out(double2& y, float2 f, float2 g) {
  y = make_double2((double)f.x + (double)g.x, (double)f.y + (double)g.y);
}
__device__ __forceinline__ void sum_out(double2& y, double2 f, float2 g) {
  y = make_double2(f.x + (double)g.x, f.y + (double)g.y);
}
__device__ __forceinline__ void sum_out(float2& y, float2 f, float2 g) { y = cadd(f, g); }
__device__ __forceinline__ void sum_out(float4& y, float2 f, float2 g) {
  const dfr re = df_two_sum(f.x, g.x), im = df_two_sum(f.y, g.y);
  y = make_float4(re.h, im.h, re.l, im.l);
}
__device__ __forceinline__ void sum_out(float4& y, float4 f, float2 g) {
  y = dfc_store(dfc_add(dfc_load(f), dfc{{g.x, 0.f}, {g.y, 0.f}}));
}
// residual form y = b - (f + g): only produced in complex double
__device__ __forceinline__ void residual_out(double2& y, double2 b) { y = csub(b, y); }
template <class T> __device__ __forceinline__ void residual_out(T&, double2) {}

// ---------------------------------------------------------------------------
// Policies
// ---------------------------------------------------------------------------
template <class TM_, class TIN, class TOUT>
struct ApplyP {
  using TM = TM_;
  using Acc = typename MT<TM>::Acc;
  struct Args {
    const TM* R;
    int ldR, nb, q2;
    GridDims g;
    const TIN* f;
    TOUT* y;
    const double2* bvec;  // residual mode: y = b - (I + Pi R) f
    long long nf;
    int nrhs;
    long long nitems;
  };
  __device__ static bool decode(const Args& A, long long item, ItemInfo& it) {
    it.leaf = (int)(item / 6);
    it.face = (int)(item % 6);
    it.nbr = A.g.neighbor(it.leaf, it.face);
    it.xoff = (long long)it.leaf * A.nb;
    if (it.nbr < 0) {
      it.ooff = it.xoff + (long long)it.face * A.q2;
      return false;
    }
    it.mat = A.R + (long long)it.leaf * A.nb * A.ldR + (long long)it.face * A.q2 * A.ldR;
    it.ld = A.ldR;
    it.ncols = A.nb;
    it.nrows = A.q2;
    it.ooff = (long long)it.nbr * A.nb + (long long)(it.face ^ 1) * A.q2;
    return true;
  }
  __device__ static Acc load_x(const Args& A, const ItemInfo& it, int rhs, int c) {
    return cvt<Acc>(A.f[rhs * A.nf + it.xoff + c]);
  }
  __device__ static void finish(const Args& A, long long o, Acc g) {
    TOUT v;
    sum_out(v, A.f[o], g);
    if (A.bvec) residual_out(v, A.bvec[o]);
    A.y[o] = v;
  }
  __device__ static void store(const Args& A, const ItemInfo& it, const Acc* outs, int nr, int tid) {
    for (int idx = tid; idx < nr * A.q2; idx += kThreads) {
      const int rhs = idx / A.q2, j = idx % A.q2;
      finish(A, rhs * A.nf + it.ooff + j, outs[idx]);
    }
  }
  __device__ static void copy(const Args& A, const ItemInfo& it, int nr, int tid) {
    for (int idx = tid; idx < nr * A.q2; idx += kThreads) {
      const int rhs = idx / A.q2, j = idx % A.q2;
      finish(A, rhs * A.nf + it.ooff + j, czero<Acc>());
    }
  }
};

template <class TM_>
struct RhsP {
  using TM = TM_;
  using Acc = typename MT<TM>::Acc;
  struct Args {
    const TM* H;
    int ldH, ni, nb, q2;
    GridDims g;
    const double2* s;
    const double2* t;
    double2* out;
    long long nf, nint;
    int nrhs;
    long long nitems;
  };
  __device__ static bool decode(const Args& A, long long item, ItemInfo& it) {
    it.leaf = (int)(item / 6);
    it.face = (int)(item % 6);
    it.nbr = A.g.neighbor(it.leaf, it.face);
    if (it.nbr < 0) {
      it.ooff = (long long)it.leaf * A.nb + (long long)it.face * A.q2;
      return false;
    }
    it.ooff = (long long)it.nbr * A.nb + (long long)(it.face ^ 1) * A.q2;
    if (!A.s) return false;
    it.mat = A.H + (long long)it.leaf * A.nb * A.ldH + (long long)it.face * A.q2 * A.ldH;
    it.ld = A.ldH;
    it.ncols = A.ni;
    it.nrows = A.q2;
    it.xoff = (long long)it.leaf * A.ni;
    return true;
  }
  __device__ static Acc load_x(const Args& A, const ItemInfo& it, int rhs, int c) {
    return cvt<Acc>(A.s[rhs * A.nint + it.xoff + c]);
  }
  __device__ static void store(const Args& A, const ItemInfo& it, const Acc* outs, int nr, int tid) {
    for (int idx = tid; idx < nr * A.q2; idx += kThreads) {
      const int rhs = idx / A.q2, j = idx % A.q2;
      const double2 v = cvt<double2>(outs[idx]);
      A.out[rhs * A.nf + it.ooff + j] = make_double2(-v.x, -v.y);
    }
  }
  __device__ static void copy(const Args& A, const ItemInfo& it, int nr, int tid) {
    for (int idx = tid; idx < nr * A.q2; idx += kThreads) {
      const int rhs = idx / A.q2, j = idx % A.q2;
      const long long o = rhs * A.nf + it.ooff + j;
      A.out[o] = (it.nbr < 0 && A.t) ? A.t[o] : make_double2(0.0, 0.0);
    }
  }
};

// Stage K over distinct blocks: item = (block k, block slot s, first member,
// member count) with the members the clusters sharing block k; "right-hand
// side" rr of the item is member rr (one right-hand side per launch).
template <class TM_, class TIN, class TOUT>
struct PrecKP {
  using TM = TM_;
  using Acc = typename MT<TM>::Acc;
  struct Args {
    const TM* K;
    const float* kscale;  // FP16 blocks: row scales, index (kc_slot_begin[k] + s)*q2 + j
    const int4* items;
    const long long* kc_off;
    const int* kc_slot_begin;
    const int* members;
    const int* cl_slot_begin;
    const int* slot_lf;
    const long long* cl_tpos;
    int nb, q2;
    const TIN* t;
    TOUT* z;
    long long nf, tstride;
    int nrhs;  // group width of the launch
    long long nitems;
  };
  // item (k, s * kKRowSplit + part, first member, members): rows
  // [part * hq, min(q^2, (part + 1) * hq)) of slot s, hq = ceil(q^2 / kKRowSplit)
  __device__ static bool decode(const Args& A, long long item, ItemInfo& it) {
    const int4 e = A.items[item];
    const int k = e.x, s = e.y / kKRowSplit, part = e.y % kKRowSplit;
    const int hq = (A.q2 + kKRowSplit - 1) / kKRowSplit;
    const int r0 = min(A.q2, part * hq);
    const int s0 = A.kc_slot_begin[k], ns = A.kc_slot_begin[k + 1] - s0;
    it.ncols = ns * A.q2;
    it.ld = (int)rup4(it.ncols);
    it.mat = A.K + A.kc_off[k] + ((long long)s * A.q2 + r0) * it.ld;
    it.nrows = min(A.q2, r0 + hq) - r0;
    it.face = s;
    it.nbr = r0;    // first row within the slot
    it.xoff = e.z;  // first member
    it.mask = e.w;  // members
    it.aoff = (long long)(s0 + s) * A.q2 + r0;
    return it.nrows > 0;
  }
  __device__ static Acc load_x(const Args& A, const ItemInfo& it, int rr, int c) {
    if (rr >= it.mask) return czero<Acc>();
    const int cl = A.members[it.xoff + rr];
    return cvt<Acc>(A.t[A.cl_tpos[cl] + c]);
  }
  __device__ static void store(const Args& A, const ItemInfo& it, const Acc* outs, int, int tid) {
    for (int idx = tid; idx < it.mask * it.nrows; idx += kThreads) {
      const int rr = idx / it.nrows, jj = idx % it.nrows;
      const int cl = A.members[it.xoff + rr];
      const int lf = A.slot_lf[A.cl_slot_begin[cl] + it.face];
      const long long o = (long long)(lf / 6) * A.nb + (long long)(lf % 6) * A.q2 + it.nbr + jj;
      A.z[o] = cvt<TOUT>(rscale(outs[idx], A.kscale, it.aoff + jj));
    }
  }
  __device__ static void copy(const Args&, const ItemInfo&, int, int) {}
};

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
// gate: while a GMRES cycle is replayed from a graph, the word that says whether any
// right-hand side is still active (0: return at once); nullptr otherwise.
template <class P, int NR, int RPW>
__global__ void __launch_bounds__(kThreads) seg_gemv_kernel(const typename P::Args A, int xcap, int rowcap,
                                                            const int* gate) {
  if (gate && *gate == 0) return;
  using TM = typename P::TM;
  using Acc = typename P::Acc;
  constexpr int VPL = MT<TM>::VPL;
  extern __shared__ __align__(16) unsigned char smraw[];
  Acc* xs = reinterpret_cast<Acc*>(smraw);
  Acc* outs = xs + NR * xcap;  // NR x rowcap
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nr = A.nrhs < NR ? A.nrhs : NR;
  for (long long item = blockIdx.x; item < A.nitems; item += gridDim.x) {
    ItemInfo it;
    if (!P::decode(A, item, it)) {
      P::copy(A, it, nr, tid);
      continue;
    }
    const int ncp = (it.ncols + VPL - 1) / VPL * VPL;
    for (int idx = tid; idx < NR * ncp; idx += kThreads) {
      const int rr = idx / ncp, c = idx % ncp;
      xs[rr * ncp + c] = (rr < nr && c < it.ncols) ? P::load_x(A, it, rr, c) : czero<Acc>();
    }
    __syncthreads();
    const TM* mat = reinterpret_cast<const TM*>(it.mat);
    const int nrows = it.nrows;
    for (int r0 = warp * RPW; r0 < nrows; r0 += kWarps * RPW) {
      Acc acc[RPW][NR];
#pragma unroll
      for (int i = 0; i < RPW; ++i)
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) acc[i][rr] = czero<Acc>();
#pragma unroll 2
      for (int c = lane * VPL; c < ncp; c += 32 * VPL) {
        Acc mv[RPW][VPL];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
          if (r0 + i < nrows) {
            MT<TM>::load(mat + (long long)(r0 + i) * it.ld + c, mv[i]);
          } else {
#pragma unroll
            for (int v = 0; v < VPL; ++v) mv[i][v] = czero<Acc>();
          }
        }
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            const Acc xv = xs[rr * ncp + c + v];
#pragma unroll
            for (int i = 0; i < RPW; ++i) cfma(acc[i][rr], mv[i][v], xv);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RPW; ++i)
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          acc[i][rr].x = warp_sum(acc[i][rr].x);
          acc[i][rr].y = warp_sum(acc[i][rr].y);
        }
      if (lane == 0) {
#pragma unroll
        for (int i = 0; i < RPW; ++i)
          if (r0 + i < nrows)
#pragma unroll
            for (int rr = 0; rr < NR; ++rr) outs[rr * nrows + r0 + i] = acc[i][rr];
      }
    }
    __syncthreads();
    P::store(A, it, outs, nr, tid);
    __syncthreads();
  }
}

// Stage B: one CTA per leaf (persistent), one thread per row of the leaf's B
// block.  B is stored transposed (column c holds the nint q^2 rows), so a warp
// reads 32 consecutive rows of one column: coalesced loads and no cross-lane
// reductions.  The external-face values are staged in shared memory; t at the
// neighbours' internal slots gets r - B r_ext, z_ext = r_ext.  Several
// right-hand sides: NR of them per pass over the block, each B entry loaded
// once per pass and used NR times (rhs r of vector v at v + r * stride).
template <class TM, class TIN, class TOUT>
struct PrecBArgs {
  const TM* B;
  const float* bscale;  // FP16 blocks: row scales, index bsc[leaf*6 + k] + j
  const long long* b_off;
  const uint8_t* int_mask;
  const int* brd;  // per leaf, internal faces then external: input offsets
  const int* bto;  // per leaf, internal faces: t offsets
  const int* bsc;  // per leaf, internal faces: row-scale bases
  int nl, q2;
  const TIN* r;
  TOUT* z;
  TOUT* t;
  int nrhs;
  long long vstride, tstride;  // per right-hand side: r and z, t
  const int* gate;  // as in seg_gemv_kernel
  // optional: the largest |component| of t per (right-hand side, cluster), as float bits
  // (non-negative floats order like their bit patterns, so atomicMax gives the same result in
  // any order); the scale of the FP16 tensor-core stage K
  unsigned* tmax;
  const int* leaf_cluster;
  int ncl;
  // work items: groups of leaves sharing one B block, as (first index into gleaves, count)
  const int2* groups;
  const int* gleaves;
  int ngroups;
};

template <class TM> __device__ __forceinline__ typename MT<TM>::Acc load_one(const TM* p);
template <> __device__ __forceinline__ float2 load_one<__half2>(const __half2* p) { return __half22float2(*p); }
template <> __device__ __forceinline__ float2 load_one<float2>(const float2* p) { return *p; }
template <> __device__ __forceinline__ double2 load_one<double2>(const double2* p) { return *p; }

template <class TM, class TIN, class TOUT, int NR>
__global__ void __launch_bounds__(kThreads) prec_b_kernel(const PrecBArgs<TM, TIN, TOUT> A) {
  if (A.gate && *A.gate == 0) return;
  using Acc = typename MT<TM>::Acc;
  extern __shared__ __align__(16) unsigned char smraw[];
  Acc* xs = reinterpret_cast<Acc*>(smraw);  // NR x (external columns)
  const int q2 = A.q2;
  // item: a group of leaves sharing one B block (same block, same internal-face mask); the
  // vectors of a pass are NR (leaf of the group, right-hand side) pairs, so every entry of B
  // loaded from L2 serves NR independent accumulations
  for (int item = blockIdx.x; item < A.ngroups; item += gridDim.x) {
    const int2 grp = A.groups[item];
    const int leaf0 = A.gleaves[grp.x];
    const int nint = __popc((unsigned)A.int_mask[leaf0]);
    const int ncols = (6 - nint) * q2, nrows = nint * q2;
    const TM* Bm = A.B + A.b_off[leaf0];
    const int ldr = (int)rup4(nrows);
    const int nvec = grp.y * A.nrhs;
    for (int v0 = 0; v0 < nvec; v0 += NR) {
      const int nr = min(NR, nvec - v0);
      __syncthreads();
      for (int idx = threadIdx.x; idx < nr * ncols; idx += kThreads) {
        const int rr = idx / ncols, c = idx - rr * ncols;
        const int vid = v0 + rr, leaf = A.gleaves[grp.x + vid / A.nrhs], rhs = vid % A.nrhs;
        const int k = c / q2;
        const long long o = (long long)rhs * A.vstride + A.brd[leaf * 6 + nint + k] + (c - k * q2);
        const Acc v = cvt<Acc>(A.r[o]);
        xs[rr * ncols + c] = v;
        A.z[o] = cvt<TOUT>(v);
      }
      __syncthreads();
      if (nint == 0) continue;
      float tmx[NR];
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) tmx[rr] = 0.f;
      for (int row = threadIdx.x; row < nrows; row += kThreads) {
        Acc acc[NR];
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) acc[rr] = czero<Acc>();
#pragma unroll 4
        for (int c = 0; c < ncols; ++c) {
          const Acc bv = load_one<TM>(Bm + (long long)c * ldr + row);
#pragma unroll
          for (int rr = 0; rr < NR; ++rr)
            if (rr < nr) cfma(acc[rr], bv, xs[rr * ncols + c]);
        }
        const int k = row / q2, j = row - k * q2;
#pragma unroll
        for (int rr = 0; rr < NR; ++rr) {
          if (rr >= nr) break;
          const int vid = v0 + rr, leaf = A.gleaves[grp.x + vid / A.nrhs], rhs = vid % A.nrhs;
          const int e = leaf * 6 + k;
          const Acc g = rscale(acc[rr], A.bscale, (long long)A.bsc[e] + j);
          const Acc v = csub(cvt<Acc>(A.r[(long long)rhs * A.vstride + A.brd[e] + j]), g);
          const TOUT tv = cvt<TOUT>(v);
          A.t[(long long)rhs * A.tstride + A.bto[e] + j] = tv;
          if constexpr (std::is_same<TOUT, float2>::value) tmx[rr] = fmaxf(tmx[rr], fmaxf(fabsf(tv.x), fabsf(tv.y)));
        }
      }
      if constexpr (std::is_same<TOUT, float2>::value) {
        if (A.tmax) {
#pragma unroll
          for (int rr = 0; rr < NR; ++rr) {
            float m = tmx[rr];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0 && rr < nr && m > 0.f) {
              const int vid = v0 + rr, leaf = A.gleaves[grp.x + vid / A.nrhs], rhs = vid % A.nrhs;
              atomicMax(A.tmax + (long long)rhs * A.ncl + A.leaf_cluster[leaf], __float_as_uint(m));
            }
          }
        }
      }
    }
  }
}

template <class P, int NR, int RPW>
cudaError_t launch_one(const typename P::Args& A, int xcap, int rowcap, int nsm, cudaStream_t st, long long* counter,
                       const int* gate, int bps = 0) {
  using Acc = typename P::Acc;
  const size_t smem = ((size_t)NR * xcap + (size_t)NR * rowcap) * sizeof(Acc);
  auto kern = seg_gemv_kernel<P, NR, RPW>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
  if (e != cudaSuccess) return e;
  occ = std::max(occ, 1);
  if (bps > 0) occ = std::min(occ, bps);  // a tuned cap on resident CTAs per SM
  long long grid = std::min<long long>(A.nitems, (long long)nsm * occ);
  if (grid <= 0) return cudaSuccess;
  kern<<<(unsigned)grid, kThreads, smem, st>>>(A, xcap, rowcap, gate);
  ++*counter;
  return cudaGetLastError();
}

// launch_one with the rows per warp chosen at run time (1, 2, 4 or 8; at most 16
// accumulators of RPW rows x NR right-hand sides per thread, fewer rows otherwise)
template <class P, int NR>
cudaError_t launch_shaped(const typename P::Args& A, int xcap, int rowcap, int nsm, cudaStream_t st,
                          long long* counter, const int* gate, LaunchShape sh) {
  const int r = sh.rpw;
  if constexpr (NR <= 2) {
    if (r >= 8) return launch_one<P, NR, 8>(A, xcap, rowcap, nsm, st, counter, gate, sh.bps);
  }
  if constexpr (NR <= 4) {
    if (r >= 4) return launch_one<P, NR, 4>(A, xcap, rowcap, nsm, st, counter, gate, sh.bps);
  }
  if (r >= 2) return launch_one<P, NR, 2>(A, xcap, rowcap, nsm, st, counter, gate, sh.bps);
  return launch_one<P, NR, 1>(A, xcap, rowcap, nsm, st, counter, gate, sh.bps);
}

// group of nr right-hand sides -> index into the shape tables
inline int group_index(int nr) { return nr == 1 ? 0 : nr == 2 ? 1 : nr <= 4 ? 2 : 3; }

template <class P>
cudaError_t launch_group(const typename P::Args& B, int nr, int xcap, int rowcap, int nsm, cudaStream_t st,
                         long long* counter, const int* gate, LaunchShape sh) {
  if (nr == 1) return launch_shaped<P, 1>(B, xcap, rowcap, nsm, st, counter, gate, sh);
  if (nr == 2) return launch_shaped<P, 2>(B, xcap, rowcap, nsm, st, counter, gate, sh);
  if (nr <= 4) return launch_shaped<P, 4>(B, xcap, rowcap, nsm, st, counter, gate, sh);
  return launch_shaped<P, 8>(B, xcap, rowcap, nsm, st, counter, gate, sh);
}

// Launch over right-hand-side groups of at most 8 (each group re-reads the matrix);
// shapes[g]: the launch shape of group index g.
template <class P, class Shift>
cudaError_t launch_groups(const hps_handle* h, typename P::Args A, int nrhs, int xcap, int rowcap, cudaStream_t st,
                          Shift shift, const LaunchShape* shapes) {
  const int nsm = h->nsm;
  long long* counter = &h->prof.launches;
  for (int r0 = 0; r0 < nrhs; r0 += 8) {
    typename P::Args B = A;
    const int nr = std::min(8, nrhs - r0);
    shift(B, r0);
    B.nrhs = nr;
    const cudaError_t e = launch_group<P>(B, nr, xcap, rowcap, nsm, st, counter, h->gate, shapes[group_index(nr)]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Shared-memory columns staged per vector: the leaf's face data (apply), its interior source
// (right-hand side), or a cluster's internal right-hand side (stage K).
enum class XCap { Apply, Rhs, StageK };
int xcap_of(const hps_handle* h, XCap which) {
  int mx = which == XCap::Apply ? h->nb : which == XCap::Rhs ? h->ni : 0;
  if (which == XCap::StageK && h->has_precond)
    for (int c = 0; c < h->ct.ncl; ++c)
      mx = std::max(mx, (h->ct.cl_slot_begin[c + 1] - h->ct.cl_slot_begin[c]) * h->q * h->q);
  return (int)round_up(std::max(mx, 1), 64);
}

template <class TM, class TIN, class TOUT>
cudaError_t apply_t(const hps_handle* h, const TM* R, const TIN* f, TOUT* y, const double2* bvec, int nrhs,
                    cudaStream_t st) {
  using P = ApplyP<TM, TIN, TOUT>;
  typename P::Args A;
  A.R = R;
  A.ldR = h->ldR;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.g = GridDims{h->nx, h->ny, h->nz};
  A.f = f;
  A.y = y;
  A.bvec = bvec;
  A.nf = h->nf;
  A.nrhs = nrhs;
  A.nitems = (long long)h->nl * 6;
  const LaunchShape* shapes = h->shapes.apply[std::is_same<TM, double2>::value ? 1 : 0];
  return launch_groups<P>(h, A, nrhs, xcap_of(h, XCap::Apply), A.q2, st, [&](typename P::Args& B, int r0) {
    B.f += (long long)r0 * h->nf;
    B.y += (long long)r0 * h->nf;
    if (B.bvec) B.bvec += (long long)r0 * h->nf;
  }, shapes);
}

template <class TM, class TIN, class TOUT>
cudaError_t precond_t(const hps_handle* h, const TM* B, const TM* K, const TIN* r, TOUT* z, TOUT* t, int nrhs,
                      cudaStream_t st, const float* bscale = nullptr, const float* kscale = nullptr,
                      bool use_tc = false) {
  const int q2 = h->q * h->q;
  const long long tstride = h->ct.tsize;
  // FP16 blocks with complex-float output on the uniform layout: stage K of every block on the
  // tensor cores with FP16 operands, t scaled per cluster (stage B records the scales)
  bool tc16 = false;
  if constexpr (std::is_same<TM, __half2>::value && std::is_same<TOUT, float2>::value)
    tc16 = precond_tc16_eligible(h, nrhs);
  {
    PrecBArgs<TM, TIN, TOUT> A;
    A.B = B;
    A.bscale = bscale;
    A.b_off = h->dct.b_off;
    A.int_mask = h->dct.int_mask;
    A.brd = h->dct.brd;
    A.bto = h->dct.bto;
    A.bsc = h->dct.bsc;
    A.nl = h->nl;
    A.q2 = q2;
    A.gate = h->gate;
    A.r = r;
    A.z = z;
    A.t = t;
    A.nrhs = nrhs;
    A.vstride = h->nf;
    A.tstride = tstride;
    A.tmax = nullptr;
    A.leaf_cluster = h->dct.leaf_cluster;
    A.ncl = h->ct.ncl;
    A.groups = h->dct.bgroups;
    A.gleaves = h->dct.bgroup_leaves;
    A.ngroups = (int)h->ct.bgroups.size();
    if (tc16) {
      HPS_TRY_CUDA_E(cudaMemsetAsync(h->tmax, 0, (size_t)h->ct.ncl * nrhs * sizeof(float), st));
      A.tmax = reinterpret_cast<unsigned*>(h->tmax);
    }
    using Acc = typename MT<TM>::Acc;
    cudaEvent_t ev = h->prof.begin(st);
    auto launch_b = [&](auto kern, int nr) -> cudaError_t {
      const size_t smem = (size_t)nr * h->ct.max_ext * q2 * sizeof(Acc) + 16;
      cudaError_t e2 = allow_dynamic_smem((const void*)kern, smem);
      int occ = 0;
      if (e2 == cudaSuccess) e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, smem);
      if (e2 != cudaSuccess) return e2;
      const int grid = (int)std::min<long long>(A.ngroups, (long long)h->nsm * std::max(occ, 1));
      kern<<<grid, kThreads, smem, st>>>(A);
      ++h->prof.launches;
      return cudaGetLastError();
    };
    // NR vectors (leaf of a group, right-hand side) per pass; shared memory for NR x (the most
    // external columns of any leaf: 3 q^2 when every cluster is 2x2x2, up to 6 q^2 for a leaf
    // alone in its cluster), halved while it does not fit
    const long long nvec = (long long)std::max(h->ct.max_group, 1) * nrhs;
    // (32 at a time with FP32 accumulators and many right-hand sides: each B entry read from L2
    // then feeds 32 accumulations)
    constexpr bool kWide = sizeof(Acc) == 8;
    int nr = nvec <= 1 ? 1 : nvec == 2 ? 2 : nvec <= 4 ? 4 : (kWide && nvec >= 32) ? 32 : 8;
    while (nr > 1 && (size_t)nr * h->ct.max_ext * q2 * sizeof(Acc) + 16 > (size_t)kMaxDynSmem) nr >>= 1;
    cudaError_t e;
    if (nr == 1) e = launch_b(prec_b_kernel<TM, TIN, TOUT, 1>, 1);
    else if (nr == 2) e = launch_b(prec_b_kernel<TM, TIN, TOUT, 2>, 2);
    else if (nr == 4) e = launch_b(prec_b_kernel<TM, TIN, TOUT, 4>, 4);
    else if (nr == 8) e = launch_b(prec_b_kernel<TM, TIN, TOUT, 8>, 8);
    else if constexpr (kWide) e = nr == 32 ? launch_b(prec_b_kernel<TM, TIN, TOUT, 32>, 32)
                                           : launch_b(prec_b_kernel<TM, TIN, TOUT, 16>, 16);
    else e = launch_b(prec_b_kernel<TM, TIN, TOUT, 8>, 8);
    h->prof.end(HPS_PHASE_PRECOND_B, ev, st);
    if (e != cudaSuccess) return e;
  }
  if (h->ct.nslots == 0) return cudaSuccess;
  if (tc16) {
    cudaEvent_t ev = h->prof.begin(st);
    const cudaError_t e = launch_precond_tc16(h, (const float2*)t, (float2*)z, nrhs, st);
    h->prof.end(HPS_PHASE_PRECOND_K, ev, st);
    return e;
  }
  if constexpr (std::is_same<TOUT, float2>::value) {
    // many right-hand sides: every block once per 64 of them, on the tensor cores
    if (precond_tc_multi_eligible(h, nrhs)) {
      cudaEvent_t ev = h->prof.begin(st);
      const cudaError_t e = launch_precond_tc_multi(h, (const float2*)t, (float2*)z, nrhs, h->tc_error, st);
      h->prof.end(HPS_PHASE_PRECOND_K, ev, st);
      return e;
    }
  }
  {
    using P = PrecKP<TM, TOUT, TOUT>;
    typename P::Args A;
    A.K = K;
    A.kscale = kscale;
    A.kc_off = h->dct.kc_off;
    A.kc_slot_begin = h->dct.kc_slot_begin;
    A.members = h->dct.kc_members;
    A.cl_slot_begin = h->dct.cl_slot_begin;
    A.slot_lf = h->dct.slot_lf;
    A.cl_tpos = h->dct.cl_tpos;
    A.nb = h->nb;
    A.q2 = q2;
    A.nf = h->nf;
    A.tstride = tstride;
    const int xcap = xcap_of(h, XCap::StageK);
    long long* counter = &h->prof.launches;
    cudaEvent_t ev = h->prof.begin(st);
    cudaError_t e = cudaSuccess;
    for (int rhs = 0; rhs < nrhs && e == cudaSuccess; ++rhs) {
      A.t = t + (long long)rhs * tstride;
      A.z = z + (long long)rhs * h->nf;
      if (use_tc) {
        if constexpr (std::is_same<TOUT, float2>::value)
          e = launch_precond_tc(h, (const float2*)A.t, (float2*)A.z, h->tc_error, st);
        else
          e = cudaErrorInvalidValue;
      }
      for (int g = 0; g < 4 && e == cudaSuccess; ++g) {
        const long long n = use_tc ? h->ct.kitems_ntc[g] : (long long)h->ct.kitems[g].size();
        if (n == 0) continue;
        A.items = h->dct.kitems[g];
        A.nitems = n;
        A.nrhs = 1 << g;
        e = launch_group<P>(A, 1 << g, xcap, q2, h->nsm, st, counter, h->gate, h->shapes.k[g]);
      }
    }
    h->prof.end(HPS_PHASE_PRECOND_K, ev, st);
    return e;
  }
}

}  // namespace

bool apply_tc_eligible(const hps_handle* h, int nrhs) {
  return h->opt.tc_apply && h->tc_error && h->R32 && nrhs >= 64 && nrhs % 64 == 0;
}

cudaError_t launch_apply(const hps_handle* h, bool fp32_matrix, VType tin, const void* f, VType tout, void* y,
                         const double2* bvec, int nrhs, bool residual, cudaStream_t st) {
  if (!residual) bvec = nullptr;
  if (!fp32_matrix) {
    if (tin == VType::C128 && tout == VType::C128)
      return apply_t(h, h->R64, (const double2*)f, (double2*)y, bvec, nrhs, st);
    return cudaErrorInvalidValue;
  }
  // the residual form b - (I + Pi R) f only exists for complex-double vectors
  if (bvec && !(tin == VType::C128 && tout == VType::C128)) return cudaErrorInvalidValue;
  // complex-double vectors on a lean handle: the compensated FP32 maps (FP64-accurate)
  if (tin == VType::C128 && tout == VType::C128 && compensated_maps(h)) return launch_apply_cf(h, (const double2*)f,
                                                                                               (double2*)y, bvec, nrhs, st);
  const bool tc = apply_tc_eligible(h, nrhs) && !bvec;
  if (tc && tin == VType::C64 && tout == VType::C64)
    return launch_apply_tc(h, (const float2*)f, y, false, nrhs, h->tc_error, st);
  if (tc && tin == VType::C64 && tout == VType::DF)
    return launch_apply_tc(h, (const float2*)f, y, true, nrhs, h->tc_error, st);
  if (tin == VType::C64 && tout == VType::C64)
    return apply_t(h, h->R32, (const float2*)f, (float2*)y, nullptr, nrhs, st);
  if (tin == VType::C64 && tout == VType::C128)
    return apply_t(h, h->R32, (const float2*)f, (double2*)y, nullptr, nrhs, st);
  if (tin == VType::C128 && tout == VType::C128)
    return apply_t(h, h->R32, (const double2*)f, (double2*)y, bvec, nrhs, st);
  if (tin == VType::C64 && tout == VType::DF)
    return apply_t(h, h->R32, (const float2*)f, (float4*)y, nullptr, nrhs, st);
  if (tin == VType::DF && tout == VType::DF)
    return apply_t(h, h->R32, (const float4*)f, (float4*)y, nullptr, nrhs, st);
  return cudaErrorInvalidValue;
}

cudaError_t timed_apply(const hps_handle* h, int phase, bool fp32_matrix, VType tin, const void* f, VType tout,
                        void* y, const double2* bvec, int nrhs, bool residual, cudaStream_t st) {
  cudaEvent_t ev = h->prof.begin(st);
  cudaError_t e = launch_apply(h, fp32_matrix, tin, f, tout, y, bvec, nrhs, residual, st);
  h->prof.end(phase, ev, st);
  return e;
}

template <class TM>
cudaError_t rhs_t(const hps_handle* h, const TM* H, const double2* s, const double2* t, double2* b, int nrhs,
                  cudaStream_t st) {
  using P = RhsP<TM>;
  typename P::Args A;
  A.H = H;
  A.ldH = h->ldH;
  A.ni = h->ni;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.g = GridDims{h->nx, h->ny, h->nz};
  A.s = s;
  A.t = t;
  A.out = b;
  A.nf = h->nf;
  A.nint = h->nint;
  A.nrhs = nrhs;
  A.nitems = (long long)h->nl * 6;
  static const LaunchShape kDefault[4] = {{4, 0}, {4, 0}, {2, 0}, {1, 0}};
  return launch_groups<P>(h, A, nrhs, xcap_of(h, XCap::Rhs), A.q2, st, [&](typename P::Args& B, int r0) {
    if (B.s) B.s += (long long)r0 * h->nint;
    if (B.t) B.t += (long long)r0 * h->nf;
    B.out += (long long)r0 * h->nf;
  }, kDefault);
}

cudaError_t launch_rhs(const hps_handle* h, const double2* s, const double2* t, double2* b, int nrhs,
                       cudaStream_t st, bool compensated) {
  if (compensated && h->H16lo && h->H32) return launch_rhs_cf(h, s, t, b, nrhs, st);
  if (h->H64) return rhs_t(h, h->H64, s, t, b, nrhs, st);
  if (h->H16lo) return launch_rhs_cf(h, s, t, b, nrhs, st);
  return rhs_t(h, h->H32, s, t, b, nrhs, st);
}

cudaError_t launch_precond(const hps_handle* h, bool fp32_matrix, VType tin, const void* r, VType tout, void* z,
                           void* scratch, int nrhs, cudaStream_t st, bool fp16_blocks) {
  if (!fp32_matrix) {
    if (tin == VType::C128 && tout == VType::C128)
      return precond_t(h, h->B64, h->Kc64, (const double2*)r, (double2*)z, (double2*)scratch, nrhs, st);
    return cudaErrorInvalidValue;
  }
  if (tout != VType::C64) return cudaErrorInvalidValue;
  // shared K blocks with many member clusters: complex-FP32 blocks on the tensor cores
  const bool tc = h->opt.tc_apply && h->Kc32 && h->tc_error && !h->ct.kc_tc.empty();
  if (fp16_blocks) {
    if (!h->Kc16 || !h->B16) return cudaErrorInvalidValue;
    if (tin == VType::C64)
      return precond_t(h, h->B16, h->Kc16, (const float2*)r, (float2*)z, (float2*)scratch, nrhs, st, h->B16s, h->Kc16s,
                       tc);
    if (tin == VType::DF)
      return precond_t(h, h->B16, h->Kc16, (const float4*)r, (float2*)z, (float2*)scratch, nrhs, st, h->B16s, h->Kc16s,
                       tc);
    return precond_t(h, h->B16, h->Kc16, (const double2*)r, (float2*)z, (float2*)scratch, nrhs, st, h->B16s, h->Kc16s,
                     tc);
  }
  if (tin == VType::C64)
    return precond_t(h, h->B32, h->Kc32, (const float2*)r, (float2*)z, (float2*)scratch, nrhs, st, nullptr, nullptr,
                     tc);
  if (tin == VType::DF)
    return precond_t(h, h->B32, h->Kc32, (const float4*)r, (float2*)z, (float2*)scratch, nrhs, st, nullptr, nullptr,
                     tc);
  return precond_t(h, h->B32, h->Kc32, (const double2*)r, (float2*)z, (float2*)scratch, nrhs, st, nullptr, nullptr, tc);
}

// ---------------------------------------------------------------------------
// Autotuner of the launch shapes (rows per warp, resident CTAs per SM) of the
// batched GEMV kernels, run once per shape at setup: every candidate is timed
// with CUDA events (one warm-up launch, then three) on the handle's own data,
// the fastest kept in a process-wide table keyed by (device, kernel, q,
// leaves, right-hand-side group, work items), so later handles of the same
// size reuse it.  The shapes do not change results (see LaunchShape).
// ---------------------------------------------------------------------------
namespace {

std::mutex g_tune_mu;
std::map<std::array<long long, 6>, LaunchShape> g_tuned;

template <class P>
LaunchShape tune_group(const hps_handle* h, const typename P::Args& A, int nr, int xcap, int rowcap,
                       const std::array<long long, 6>& key, LaunchShape dflt, cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) return it->second;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return dflt;
  }
  long long dummy = 0;
  auto time_one = [&](LaunchShape sh) -> float {
    if (launch_group<P>(A, nr, xcap, rowcap, h->nsm, st, &dummy, nullptr, sh) != cudaSuccess) return 1e30f;
    cudaEventRecord(e0, st);
    for (int i = 0; i < 3; ++i)
      if (launch_group<P>(A, nr, xcap, rowcap, h->nsm, st, &dummy, nullptr, sh) != cudaSuccess) return 1e30f;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 3.f;
  };
  LaunchShape best = dflt;
  float tbest = time_one(dflt);
  const int rmax = nr <= 2 ? 8 : nr <= 4 ? 4 : 2;
  for (int rpw = 1; rpw <= rmax; rpw *= 2)
    for (int bps = 0; bps <= 3; ++bps) {
      const LaunchShape sh{rpw, bps};
      if (sh.rpw == dflt.rpw && sh.bps == dflt.bps) continue;
      const float t = time_one(sh);
      if (t < 0.98f * tbest) {  // a clear win over the incumbent only
        tbest = t;
        best = sh;
      }
    }
  cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[key] = best;
  return best;
}

template <class TM, class TIN, class TOUT>
cudaError_t tune_apply(hps_handle* h, const TM* R, int kind, void* fbuf, void* ybuf, int nr, cudaStream_t st) {
  using P = ApplyP<TM, TIN, TOUT>;
  typename P::Args A;
  A.R = R;
  A.ldR = h->ldR;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.g = GridDims{h->nx, h->ny, h->nz};
  A.f = (const TIN*)fbuf;
  A.y = (TOUT*)ybuf;
  A.bvec = nullptr;
  A.nf = h->nf;
  A.nrhs = nr;
  A.nitems = (long long)h->nl * 6;
  const int g = group_index(nr);
  const std::array<long long, 6> key{h->dev, kind, h->q, h->nl, nr, A.nitems};
  h->shapes.apply[kind][g] = tune_group<P>(h, A, nr, xcap_of(h, XCap::Apply), A.q2, key, h->shapes.apply[kind][g], st);
  return cudaSuccess;
}

template <class TM>
cudaError_t tune_stage_k(hps_handle* h, const TM* K, const float* kscale, void* t, void* z, bool tc, cudaStream_t st) {
  using P = PrecKP<TM, float2, float2>;
  typename P::Args A;
  A.K = K;
  A.kscale = kscale;
  A.kc_off = h->dct.kc_off;
  A.kc_slot_begin = h->dct.kc_slot_begin;
  A.members = h->dct.kc_members;
  A.cl_slot_begin = h->dct.cl_slot_begin;
  A.slot_lf = h->dct.slot_lf;
  A.cl_tpos = h->dct.cl_tpos;
  A.nb = h->nb;
  A.q2 = h->q * h->q;
  A.nf = h->nf;
  A.tstride = h->ct.tsize;
  A.t = (const float2*)t;
  A.z = (float2*)z;
  for (int g = 0; g < 4; ++g) {
    const long long n = tc ? h->ct.kitems_ntc[g] : (long long)h->ct.kitems[g].size();
    if (n == 0) continue;
    A.items = h->dct.kitems[g];
    A.nitems = n;
    A.nrhs = 1 << g;
    const std::array<long long, 6> key{h->dev, 10 + (long long)sizeof(TM), h->q, h->nl, g, n};
    h->shapes.k[g] = tune_group<P>(h, A, 1 << g, xcap_of(h, XCap::StageK), A.q2, key, h->shapes.k[g], st);
  }
  return cudaSuccess;
}

}  // namespace

int autotune_shapes(hps_handle* h, cudaStream_t st) {
  const long long nf = h->nf;
  const int nr_max = std::min(8, std::max(1, h->opt.max_rhs));
  void *fbuf = nullptr, *ybuf = nullptr;
  const size_t bytes = (size_t)nr_max * nf * sizeof(double2);
  if (cudaMalloc(&fbuf, bytes) != cudaSuccess || cudaMalloc(&ybuf, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (fbuf) cudaFree(fbuf);
    return HPS_OK;  // tuning is an optimization: keep the default shapes
  }
  cudaMemsetAsync(fbuf, 0, bytes, st);
  cudaMemsetAsync(ybuf, 0, bytes, st);
  std::vector<int> groups{1};
  if (nr_max > 1) groups.push_back(nr_max);
  for (int nr : groups) {
    // the inner apply of each form: complex-FP32 operand into the double-float basis, and FP64
    if (h->R32) tune_apply<float2, float2, float4>(h, h->R32, 0, fbuf, ybuf, nr, st);
    if (h->R64) tune_apply<double2, double2, double2>(h, h->R64, 1, fbuf, ybuf, nr, st);
  }
  // SIMT stage K of the mixed solve (FP16 blocks when kept, else FP32)
  if (h->has_precond && h->ct.nslots > 0 && h->pc_scratch) {
    cudaMemsetAsync(h->pc_scratch, 0, (size_t)h->ct.tsize * sizeof(float2), st);
    const bool tc = h->opt.tc_apply && h->Kc32 && h->tc_error && !h->ct.kc_tc.empty();
    if (h->Kc16) tune_stage_k<__half2>(h, h->Kc16, h->Kc16s, h->pc_scratch, ybuf, tc, st);
    else if (h->Kc32) tune_stage_k<float2>(h, h->Kc32, nullptr, h->pc_scratch, ybuf, tc, st);
  }
  cudaStreamSynchronize(st);
  cudaGetLastError();
  cudaFree(fbuf);
  cudaFree(ybuf);
  h->shapes.tuned = true;
  return HPS_OK;
}

}  // namespace hps
