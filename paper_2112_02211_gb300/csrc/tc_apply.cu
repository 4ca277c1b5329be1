// Multi-right-hand-side ItI apply on the 5th-generation tensor cores (sm_103a).
//
// For one leaf tau and 64 right-hand sides the apply is a complex GEMM
// G = R F (R: n_b x n_b, F: n_b x 64).  With R stored row-major as
// interleaved complex FP32 it is, read as real numbers, an n_b x 2n_b matrix
// A whose columns alternate (re, im).  Against it
//   B^T row s      = conj(f_s)            (re, -im, re, -im, ...)
//   B^T row 64 + s = f_s with re/im swapped (im, re, im, re, ...)
// give A B = [Re G | Im G] (rows of A times conj/swap pairs reproduce
// Re(R f) = Rr fr - Ri fi and Im(R f) = Rr fi + Ri fr).  Both B rows come
// from the contiguous vector f_s, so the tiles are loaded by TMA straight from
// the face-vector layout and rewritten in shared memory.
//
// Precision: three TF32 products (A_hi B_hi + A_hi B_lo + A_lo B_hi, with
// x_hi = x rounded to TF32 and x_lo = x - x_hi rounded to TF32) keep about 22
// bits per product term; FP32 accumulation in tensor memory (TMEM).
//
// Kernel (one CTA per SM, persistent over items = (leaf, 128-row tile)):
//   warp 0       TMA producer: A tile (128 rows x 32 floats) and F tile
//                (64 rhs x 32 floats), 128-byte swizzle, into a 3-stage ring
//   warps 2..7   split the stage: A -> A_hi (in place) + A_lo, F -> B_hi, B_lo
//   warp 1       tcgen05.alloc of 256 TMEM columns (two accumulators); one lane
//                issues 12 tcgen05.mma (4 K-steps x 3 products) per stage and
//                commits to mbarriers
//   warps 8..11  epilogue: tcgen05.ld of the 128 x 128 FP32 accumulator,
//                y = f + G written to the neighbour across the row's face (the
//                swap Pi fused into the store)
// Every wait is bounded: after a limit the CTA raises an error word, stops
// issuing work, waits (bounded) for its own tensor-core work, frees TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "hps_internal.h"
#include "tc_common.cuh"

namespace hps {

namespace {

using namespace tc;

constexpr int kStages = 3;
constexpr int kTileM = 128;
constexpr int kTileN = 128;   // 64 right-hand sides x (re, im)
constexpr int kRhs = 64;
constexpr int kTileK = 32;    // floats per K block (128 bytes)
constexpr int kABytes = kTileM * kTileK * 4;  // 16 KB
constexpr int kFBytes = kRhs * kTileK * 4;    // 8 KB
constexpr int kBBytes = kTileN * kTileK * 4;  // 16 KB
// stage layout (each part 1024-byte aligned): Ahi(=A) | Alo | Bhi | Blo | F
constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes + kFBytes;  // 72 KB
constexpr int kThreads = 384;  // 12 warps
constexpr int kTmemCols = 256;

struct TcArgs {
  int nl, nb, q2, nx, ny, nz;
  int mtiles, kblocks;
  long long nf;
  const float2* f;  // [rhs][nf] complex float, the 64 right-hand sides of this launch
  void* y;          // output [rhs][nf]: float2 or double-float float4
  int out_df;
  int* error;
  const int* gate;  // while a GMRES cycle is replayed: 0 = no right-hand side active, return at once
  long long spin;   // tries per bounded wait
  int skip_arrival; // test hook: CTA 0's first transform warp does not arrive on the first stage
};

struct __align__(8) Bars {
  uint64_t full[kStages];   // TMA bytes of A and F landed
  uint64_t split[kStages];  // transform warps done with the stage
  uint64_t empty[kStages];  // MMAs reading the stage completed
  uint64_t acc_full[2];     // accumulator b complete
  uint64_t acc_empty[2];    // accumulator b read by the epilogue
  uint64_t drain;           // all MMAs of this CTA completed
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(kThreads, 1)
    tc_apply_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapF, TcArgs a) {
  if (a.gate && *a.gate == 0) return;  // before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the stage ring (swizzle atoms)
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars* bars = reinterpret_cast<Bars*>(ring + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nitems = (long long)a.nl * a.mtiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->split[s], 6);  // one arrival per transform warp
      mbar_init(&bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars->acc_full[b], 1);
      mbar_init(&bars->acc_empty[b], 4);  // one arrival per epilogue warp
    }
    mbar_init(&bars->drain, 1);
    bars->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&bars->tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = bars->tmem_base;

  auto fail = [&]() {
    atomicExch(a.error, 1);
    atomicExch(&bars->abort, 1);
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      long long it = 0;
      bool ok = true;
      for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x) {
        const int leaf = (int)(item / a.mtiles), mt = (int)(item % a.mtiles);
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (bars->abort || (it >= kStages && !mbar_wait(&bars->empty[s], ph ^ 1, a.spin))) {
            fail();
            ok = false;
            break;
          }
          unsigned char* st = ring + s * kStageBytes;
          mbar_expect_tx(&bars->full[s], kABytes + kFBytes);
          tma_load_3d(st, &mapA, &bars->full[s], kb * kTileK, mt * kTileM, leaf);
          tma_load_2d(st + 2 * kABytes + 2 * kBBytes, &mapF, &bars->full[s], leaf * 2 * a.nb + kb * kTileK, 0);
        }
      }
      // copies still in flight land before the CTA leaves (bounded wait)
      for (long long j = (it > kStages ? it - kStages : 0); j < it; ++j)
        if (!mbar_wait(&bars->full[(int)(j % kStages)], (uint32_t)((j / kStages) & 1), a.spin)) fail();
    }
  } else if (warp >= 2 && warp < 8) {
    // ---------------- split into TF32 hi/lo operands ----------------
    const int t = threadIdx.x - 64;  // 0..191
    long long it = 0;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kStages);
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (bars->abort || !mbar_wait(&bars->full[s], ph, a.spin)) {
          fail();
          goto split_done;
        }
        unsigned char* st = ring + s * kStageBytes;
        float4* Ahi = reinterpret_cast<float4*>(st);
        float4* Alo = reinterpret_cast<float4*>(st + kABytes);
        float4* Bhi = reinterpret_cast<float4*>(st + 2 * kABytes);
        float4* Blo = reinterpret_cast<float4*>(st + 2 * kABytes + kBBytes);
        const float4* F = reinterpret_cast<const float4*>(st + 2 * kABytes + 2 * kBBytes);
        for (int c = t; c < kABytes / 16; c += 192) {
          const float4 v = Ahi[c];
          const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
          Ahi[c] = h;
          Alo[c] = make_float4(tf32_hi(v.x - h.x), tf32_hi(v.y - h.y), tf32_hi(v.z - h.z), tf32_hi(v.w - h.w));
        }
        // F rows s (64 x 128 bytes): B row s = conj(f_s), B row 64+s = swap(f_s); the
        // 16-byte chunk positions (and so the swizzle) are the same in both halves.
        for (int c = t; c < kFBytes / 16; c += 192) {
          const float4 v = F[c];
          const float4 cj = make_float4(v.x, -v.y, v.z, -v.w);
          const float4 sw = make_float4(v.y, v.x, v.w, v.z);
          const float4 cjh = make_float4(tf32_hi(cj.x), tf32_hi(cj.y), tf32_hi(cj.z), tf32_hi(cj.w));
          const float4 swh = make_float4(tf32_hi(sw.x), tf32_hi(sw.y), tf32_hi(sw.z), tf32_hi(sw.w));
          Bhi[c] = cjh;
          Blo[c] = make_float4(tf32_hi(cj.x - cjh.x), tf32_hi(cj.y - cjh.y), tf32_hi(cj.z - cjh.z),
                               tf32_hi(cj.w - cjh.w));
          Bhi[c + kFBytes / 16] = swh;
          Blo[c + kFBytes / 16] = make_float4(tf32_hi(sw.x - swh.x), tf32_hi(sw.y - swh.y), tf32_hi(sw.z - swh.z),
                                              tf32_hi(sw.w - swh.w));
        }
        // make the generic-proxy writes visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        // (test hook: one missing arrival makes the MMA issuer's bounded wait run out)
        const bool skip = a.skip_arrival && blockIdx.x == 0 && warp == 2 && it == 0;
        if (lane == 0 && !skip) mbar_arrive(&bars->split[s]);
      }
    }
  split_done:;
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = instr_desc_tf32(kTileN, kTileM);
      long long it = 0;
      long long local = 0;
      bool ok = true;
      for (long long item = blockIdx.x; item < nitems && ok; item += gridDim.x, ++local) {
        const int b = (int)(local & 1);
        const uint32_t acc = tmem + (uint32_t)(b * kTileN);
        if (local >= 2 && !mbar_wait(&bars->acc_empty[b], (uint32_t)(((local >> 1) - 1) & 1), a.spin)) {
          fail();
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (bars->abort || !mbar_wait(&bars->split[s], ph, a.spin)) {
            fail();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(ring + s * kStageBytes);
          const uint32_t ahi = base, alo = base + kABytes, bhi = base + 2 * kABytes, blo = bhi + kBBytes;
#pragma unroll
          for (int kk = 0; kk < kTileK / 8; ++kk) {
            const uint32_t off = kk * 32;
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            mma_tf32(acc, smem_desc(ahi + off), smem_desc(bhi + off), idesc, first);
            mma_tf32(acc, smem_desc(ahi + off), smem_desc(blo + off), idesc, 1u);
            mma_tf32(acc, smem_desc(alo + off), smem_desc(bhi + off), idesc, 1u);
          }
          mma_commit(&bars->empty[s]);
        }
        if (!ok) break;
        mma_commit(&bars->acc_full[b]);
      }
      // every MMA issued above completes before TMEM is freed (bounded wait)
      mma_commit(&bars->drain);
      if (!mbar_wait(&bars->drain, 0, a.spin)) fail();
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 8..11 = TMEM lanes 0..127 ----------------
    const int ew = warp - 8;  // TMEM lane quarter
    long long local = 0;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x, ++local) {
      const int b = (int)(local & 1);
      if (bars->abort || !mbar_wait(&bars->acc_full[b], (uint32_t)((local >> 1) & 1), a.spin)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int leaf = (int)(item / a.mtiles), mt = (int)(item % a.mtiles);
      const int row = mt * kTileM + ew * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * kTileN);
      float re[32], im[32];
      // columns 0..63 = Re G for rhs 0..63, 64..127 = Im G
      for (int half = 0; half < 2; ++half) {
        tmem_ld32(taddr + half * 32, re);
        tmem_ld32(taddr + 64 + half * 32, im);
        if (row < a.nb) {
          const int face = row / a.q2, j = row % a.q2;
          const int ix = leaf % a.nx, iy = (leaf / a.nx) % a.ny, iz = leaf / (a.nx * a.ny);
          int nx_ = ix, ny_ = iy, nz_ = iz;
          const int d = (face & 1) ? 1 : -1;
          bool inside = true;
          if ((face >> 1) == 0) { nx_ += d; inside = nx_ >= 0 && nx_ < a.nx; }
          else if ((face >> 1) == 1) { ny_ += d; inside = ny_ >= 0 && ny_ < a.ny; }
          else { nz_ += d; inside = nz_ >= 0 && nz_ < a.nz; }
          if (inside) {
            const int nbr = nx_ + a.nx * (ny_ + a.ny * nz_);
            const long long dst = (long long)nbr * a.nb + (long long)(face ^ 1) * a.q2 + j;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int rhs = half * 32 + c;
              const long long o = rhs * a.nf + dst;
              const float2 fv = a.f[o];
              if (a.out_df) {
                const dfr r1 = df_two_sum(fv.x, re[c]), r2 = df_two_sum(fv.y, im[c]);
                reinterpret_cast<float4*>(a.y)[o] = make_float4(r1.h, r2.h, r1.l, r2.l);
              } else {
                reinterpret_cast<float2*>(a.y)[o] = make_float2(fv.x + re[c], fv.y + im[c]);
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->acc_empty[b]);
    }
  }

  // Boundary faces: y = f (identity part), written by the CTA that owns the leaf's tile 0.
  __syncthreads();
  if (!bars->abort) {
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
      const int leaf = (int)(item / a.mtiles), mt = (int)(item % a.mtiles);
      if (mt != 0) continue;
      const int ix = leaf % a.nx, iy = (leaf / a.nx) % a.ny, iz = leaf / (a.nx * a.ny);
      for (int face = 0; face < 6; ++face) {
        const int d = (face & 1) ? 1 : -1;
        bool inside;
        if ((face >> 1) == 0) inside = ix + d >= 0 && ix + d < a.nx;
        else if ((face >> 1) == 1) inside = iy + d >= 0 && iy + d < a.ny;
        else inside = iz + d >= 0 && iz + d < a.nz;
        if (inside) continue;
        for (int e = threadIdx.x; e < kRhs * a.q2; e += kThreads) {
          const int rhs = e / a.q2, j = e % a.q2;
          const long long o = rhs * a.nf + (long long)leaf * a.nb + (long long)face * a.q2 + j;
          const float2 fv = a.f[o];
          if (a.out_df) reinterpret_cast<float4*>(a.y)[o] = make_float4(fv.x, fv.y, 0.f, 0.f);
          else reinterpret_cast<float2*>(a.y)[o] = fv;
        }
      }
    }
  }
  // Drain: every MMA this CTA issued has been committed; wait (bounded) for the
  // last commits before freeing TMEM.
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

// y = (I + Pi R) f for 64-RHS groups with FP32 maps, on the tensor cores.
// f: complex float [nrhs][nf]; y: complex float or double-float.  nrhs must be a
// multiple of 64.
cudaError_t launch_apply_tc(const hps_handle* h, const float2* f, void* y, bool out_df, int nrhs, int* d_error,
                            cudaStream_t st) {
  if (!h->R32 || nrhs % kRhs != 0) return cudaErrorInvalidValue;
  if ((2LL * h->nb * 4) % 16 != 0 || (2LL * h->ldR * 4) % 16 != 0) return cudaErrorInvalidValue;
  auto g_encode = encoder();
  if (!g_encode) return cudaErrorNotSupported;
  const int mtiles = (h->nb + kTileM - 1) / kTileM;
  const int kblocks = (2 * h->nb + kTileK - 1) / kTileK;
  CUtensorMap mapA;
  {
    cuuint64_t dims[3] = {(cuuint64_t)(2 * h->nb), (cuuint64_t)h->nb, (cuuint64_t)h->nl};
    cuuint64_t strides[2] = {(cuuint64_t)h->ldR * 8, (cuuint64_t)h->nb * h->ldR * 8};
    cuuint32_t box[3] = {kTileK, kTileM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (g_encode(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)h->R32, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  const int smem = kStages * kStageBytes + (int)sizeof(Bars) + 1024;
  cudaError_t e = allow_dynamic_smem((const void*)tc_apply_kernel, smem);
  if (e != cudaSuccess) return e;
  for (int r0 = 0; r0 < nrhs; r0 += kRhs) {
    CUtensorMap mapF;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * h->nf), (cuuint64_t)kRhs};
    cuuint64_t strides[1] = {(cuuint64_t)h->nf * 8};
    cuuint32_t box[2] = {kTileK, kRhs};
    cuuint32_t es[2] = {1, 1};
    const float2* fr = f + (long long)r0 * h->nf;
    if (g_encode(&mapF, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)fr, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    TcArgs a;
    a.nl = h->nl;
    a.nb = h->nb;
    a.q2 = h->q * h->q;
    a.nx = h->nx;
    a.ny = h->ny;
    a.nz = h->nz;
    a.mtiles = mtiles;
    a.kblocks = kblocks;
    a.nf = h->nf;
    a.f = fr;
    a.out_df = out_df ? 1 : 0;
    a.y = out_df ? (void*)((float4*)y + (long long)r0 * h->nf) : (void*)((float2*)y + (long long)r0 * h->nf);
    a.error = d_error;
    a.gate = h->gate;
    a.spin = h->test_spin > 0 ? h->test_spin : kSpinLimit;
    a.skip_arrival = h->test_skip_arrival;
    const long long items = (long long)h->nl * mtiles;
    const int grid = (int)std::min<long long>(items, h->nsm);
    tc_apply_kernel<<<grid, kThreads, smem, st>>>(mapA, mapF, a);
    ++h->prof.launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace hps
