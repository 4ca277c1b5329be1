// Stage K of the cluster preconditioner for shared K blocks, on the
// 5th-generation tensor cores (sm_103a).
//
// When many clusters carry the same homogenized constants (Sec. 4.1 remark:
// one local solver for leaves with nearly the same medium) they share one
// K_c = (I + D)^{-1}, and z_int = K_c t for all of them is one complex GEMM
// Z = K_c T (K_c: n x n, T: n x members, n = 24 q^2 for 2x2x2 clusters).  The
// members' t vectors are consecutive in the stage-K input (class-ordered
// layout), so T is one strided matrix for TMA.
//
// As in the multi-RHS apply (tc_apply.cu): K_c's interleaved complex FP32
// storage is read as a real n x 2n matrix A; the B operand rows are conj(t_m)
// and the re/im swap of t_m, so A B = [Re Z | Im Z].  One TF32 product per
// term (both operands rounded to TF32, 2^-11 relative, the precision of the
// FP16 blocks used for the other clusters); FP32 accumulation in TMEM.
//
// Many right-hand sides (MULTI): every block against the columns (member
// cluster, right-hand side) in one launch.  Items are (stage-K position m,
// 128-row tile, 64-RHS tile); the blocks are one 3D array [block][row][col]
// and t one [rhs][position][nint] array, so both tiles come from one tensor
// map each: K_c rows of block pos_class[m], and the member's t for 64
// right-hand sides (box 32 floats x 1 member x 64 rhs).
//
// Kernel (one CTA per SM, persistent over items = (128-row tile, 64-member tile)):
//   warp 0       TMA producer: A tile (128 rows x 32 floats) and T tile
//                (64 members x 32 floats), 128-byte swizzle, 5-stage ring
//   warps 2..7   round A to TF32 in place, build the conj/swap rows of B
//   warp 1       TMEM allocation (256 columns, two accumulators); one lane
//                issues the MMAs and commits to mbarriers
//   warps 8..11  epilogue: TMEM -> registers -> z at each member cluster's
//                internal face slots
// Every wait is bounded: after a limit the CTA raises the error word, stops
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

constexpr int kStages = 5;
constexpr int kTileM = 128;
constexpr int kMem = 64;        // member clusters per tile
constexpr int kTileN = 2 * kMem;  // (re, im) columns
constexpr int kTileK = 32;      // floats per K block (128 bytes)
constexpr int kABytes = kTileM * kTileK * 4;  // 16 KB
constexpr int kTBytes = kMem * kTileK * 4;    // 8 KB
constexpr int kBBytes = kTileN * kTileK * 4;  // 16 KB
// stage layout (each part 1024-byte aligned): A | B | T
constexpr int kStageBytes = kABytes + kBBytes + kTBytes;  // 40 KB
constexpr int kThreads = 384;
constexpr int kTmemCols = 256;

struct PkArgs {
  int nint, nmem, mtiles, ntiles, kblocks, q2, nb;
  const int* members;        // the block's member clusters (nmem); MULTI: all clusters in stage-K order
  const int* cl_slot_begin;  // first global slot of each cluster
  const int* slot_lf;        // leaf*6 + face of each global slot
  float2* z;
  int* error;
  const int* gate;  // while a GMRES cycle is replayed: 0 = no right-hand side active, return at once
  // MULTI only
  const int* pos_class;      // K block of the member at each stage-K position
  int npos, rtiles, nrhs;
  long long nf;              // right-hand-side stride of z
};

struct __align__(8) Bars {
  uint64_t full[kStages];
  uint64_t split[kStages];
  uint64_t empty[kStages];
  uint64_t acc_full[2];
  uint64_t acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort;
};

template <bool MULTI>
__global__ void __launch_bounds__(kThreads, 1)
    tc_precond_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapT, PkArgs a) {
  if (a.gate && *a.gate == 0) return;  // before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars* bars = reinterpret_cast<Bars*>(ring + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nitems = MULTI ? (long long)a.npos * a.mtiles * a.rtiles : (long long)a.mtiles * a.ntiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&bars->full[s], 1);
      mbar_init(&bars->split[s], 6);
      mbar_init(&bars->empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bars->acc_full[b], 1);
      mbar_init(&bars->acc_empty[b], 4);
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
        int mt, nt, pos = 0, rt = 0, blk = 0;
        if (MULTI) {
          // item = (position, row tile, rhs tile), rhs tile fastest
          pos = (int)(item / ((long long)a.mtiles * a.rtiles));
          const int rem = (int)(item % ((long long)a.mtiles * a.rtiles));
          mt = rem / a.rtiles;
          rt = rem % a.rtiles;
          nt = 0;
          blk = a.pos_class[pos];
        } else {
          mt = (int)(item % a.mtiles);
          nt = (int)(item / a.mtiles);
        }
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (bars->abort || (it >= kStages && !mbar_wait(&bars->empty[s], ph ^ 1))) {
            fail();
            ok = false;
            break;
          }
          unsigned char* st = ring + s * kStageBytes;
          mbar_expect_tx(&bars->full[s], kABytes + kTBytes);
          if (MULTI) {
            tma_load_3d(st, &mapA, &bars->full[s], kb * kTileK, mt * kTileM, blk);
            tma_load_3d(st + kABytes + kBBytes, &mapT, &bars->full[s], kb * kTileK, pos, rt * kMem);
          } else {
            tma_load_2d(st, &mapA, &bars->full[s], kb * kTileK, mt * kTileM);
            tma_load_2d(st + kABytes + kBBytes, &mapT, &bars->full[s], kb * kTileK, nt * kMem);
          }
        }
      }
      for (long long j = (it > kStages ? it - kStages : 0); j < it; ++j)
        if (!mbar_wait(&bars->full[(int)(j % kStages)], (uint32_t)((j / kStages) & 1))) fail();
    }
  } else if (warp >= 2 && warp < 8) {
    // ---------------- split into TF32 hi/lo operands ----------------
    const int t = threadIdx.x - 64;  // 0..191
    long long it = 0;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x) {
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kStages);
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (bars->abort || !mbar_wait(&bars->full[s], ph)) {
          fail();
          goto split_done;
        }
        unsigned char* st = ring + s * kStageBytes;
        float4* A = reinterpret_cast<float4*>(st);
        float4* B = reinterpret_cast<float4*>(st + kABytes);
        const float4* T = reinterpret_cast<const float4*>(st + kABytes + kBBytes);
        for (int c = t; c < kABytes / 16; c += 192) {
          const float4 v = A[c];
          A[c] = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
        }
        // B row m = conj(t_m), B row 64 + m = swap(t_m): same 16-byte chunk positions
        for (int c = t; c < kTBytes / 16; c += 192) {
          const float4 v = T[c];
          B[c] = make_float4(tf32_hi(v.x), tf32_hi(-v.y), tf32_hi(v.z), tf32_hi(-v.w));
          B[c + kTBytes / 16] = make_float4(tf32_hi(v.y), tf32_hi(v.x), tf32_hi(v.w), tf32_hi(v.z));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->split[s]);
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
        if (local >= 2 && !mbar_wait(&bars->acc_empty[b], (uint32_t)(((local >> 1) - 1) & 1))) {
          fail();
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (bars->abort || !mbar_wait(&bars->split[s], ph)) {
            fail();
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t base = smem_u32(ring + s * kStageBytes);
          const uint32_t aa = base, bb = base + kABytes;
#pragma unroll
          for (int kk = 0; kk < kTileK / 8; ++kk) {
            const uint32_t off = kk * 32;
            mma_tf32(acc, smem_desc(aa + off), smem_desc(bb + off), idesc, (kb == 0 && kk == 0) ? 0u : 1u);
          }
          mma_commit(&bars->empty[s]);
        }
        if (!ok) break;
        mma_commit(&bars->acc_full[b]);
      }
      mma_commit(&bars->drain);
      if (!mbar_wait(&bars->drain, 0)) fail();
    }
    __syncwarp();
  } else {
    // ---------------- epilogue: warps 8..11 = TMEM lanes 0..127 ----------------
    const int ew = warp - 8;
    long long local = 0;
    for (long long item = blockIdx.x; item < nitems; item += gridDim.x, ++local) {
      const int b = (int)(local & 1);
      if (bars->abort || !mbar_wait(&bars->acc_full[b], (uint32_t)((local >> 1) & 1))) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int mt, nt, pos = 0, rt = 0;
      if (MULTI) {
        pos = (int)(item / ((long long)a.mtiles * a.rtiles));
        const int rem = (int)(item % ((long long)a.mtiles * a.rtiles));
        mt = rem / a.rtiles;
        rt = rem % a.rtiles;
        nt = 0;
      } else {
        mt = (int)(item % a.mtiles);
        nt = (int)(item / a.mtiles);
      }
      const int row = mt * kTileM + ew * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * kTileN);
      float re[32], im[32];
      // columns 0..63 = Re Z for members 0..63 of the tile, 64..127 = Im Z
      for (int half = 0; half < 2; ++half) {
        tmem_ld32(taddr + half * 32, re);
        tmem_ld32(taddr + kMem + half * 32, im);
        if (row < a.nint) {
          const int sl = row / a.q2, j = row % a.q2;
          if (MULTI) {
            // columns: 64 right-hand sides of one member
            const int cl = a.members[pos];
            const int lf = a.slot_lf[a.cl_slot_begin[cl] + sl];
            const long long o = (long long)(lf / 6) * a.nb + (long long)(lf % 6) * a.q2 + j;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int rhs = rt * kMem + half * 32 + c;
              if (rhs < a.nrhs) a.z[(long long)rhs * a.nf + o] = make_float2(re[c], im[c]);
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int m = nt * kMem + half * 32 + c;
              if (m < a.nmem) {
                const int cl = a.members[m];
                const int lf = a.slot_lf[a.cl_slot_begin[cl] + sl];
                a.z[(long long)(lf / 6) * a.nb + (long long)(lf % 6) * a.q2 + j] = make_float2(re[c], im[c]);
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

  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

}  // namespace

// z_int = K_c t for the member clusters of every block in ct.kc_tc (complex
// FP32 blocks Kc32, one right-hand side, t in the class-ordered layout).
cudaError_t launch_precond_tc(const hps_handle* h, const float2* t, float2* z, int* d_error, cudaStream_t st) {
  const ClusterTables& ct = h->ct;
  if (!h->Kc32 || !d_error) return cudaErrorInvalidValue;
  auto encode = encoder();
  if (!encode) return cudaErrorNotSupported;
  const int q2 = h->q * h->q;
  const int smem = kStages * kStageBytes + (int)sizeof(Bars) + 1024;
  cudaError_t e = allow_dynamic_smem((const void*)tc_precond_kernel<false>, smem);
  if (e != cudaSuccess) return e;
  for (int k : ct.kc_tc) {
    const int ns = ct.kc_slot_begin[k + 1] - ct.kc_slot_begin[k];
    const int nint = ns * q2;
    const int ld = (int)round_up(nint, 4);
    const int mb = ct.kc_mem_begin[k], nmem = ct.kc_mem_begin[k + 1] - mb;
    const float2* Kk = h->Kc32 + ct.kc_off[k];
    const float2* Tk = t + ct.cl_tpos[ct.kc_members[mb]];
    // TMA: 16-byte aligned bases and row strides (checked, not assumed)
    if ((reinterpret_cast<uintptr_t>(Kk) | reinterpret_cast<uintptr_t>(Tk)) % 16 != 0 || (8LL * ld) % 16 != 0 ||
        (8LL * nint) % 16 != 0)
      return cudaErrorInvalidValue;
    CUtensorMap mapA, mapT;
    {
      cuuint64_t dims[2] = {(cuuint64_t)(2 * nint), (cuuint64_t)nint};
      cuuint64_t strides[1] = {(cuuint64_t)ld * 8};
      cuuint32_t box[2] = {kTileK, kTileM};
      cuuint32_t es[2] = {1, 1};
      if (encode(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)Kk, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    {
      cuuint64_t dims[2] = {(cuuint64_t)(2 * nint), (cuuint64_t)nmem};
      cuuint64_t strides[1] = {(cuuint64_t)nint * 8};
      cuuint32_t box[2] = {kTileK, kMem};
      cuuint32_t es[2] = {1, 1};
      if (encode(&mapT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)Tk, dims, strides, box, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    }
    PkArgs a;
    a.nint = nint;
    a.nmem = nmem;
    a.mtiles = (nint + kTileM - 1) / kTileM;
    a.ntiles = (nmem + kMem - 1) / kMem;
    a.kblocks = (2 * nint + kTileK - 1) / kTileK;
    a.q2 = q2;
    a.nb = h->nb;
    a.members = h->dct.kc_members + mb;
    a.cl_slot_begin = h->dct.cl_slot_begin;
    a.slot_lf = h->dct.slot_lf;
    a.z = z;
    a.error = d_error;
    a.gate = h->gate;
    a.pos_class = nullptr;
    a.npos = a.rtiles = a.nrhs = 0;
    a.nf = 0;
    const long long items = (long long)a.mtiles * a.ntiles;
    const int grid = (int)std::min<long long>(items, h->nsm);
    tc_precond_kernel<false><<<grid, kThreads, smem, st>>>(mapA, mapT, a);
    ++h->prof.launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool precond_tc_multi_eligible(const hps_handle* h, int nrhs) {
  return h->has_precond && h->opt.tc_apply && h->Kc32 && h->tc_error && h->ct.uniform && h->ct.nslots > 0 &&
         nrhs >= kMem && nrhs % kMem == 0;
}

// z_int = K_c t for every cluster and nrhs right-hand sides: one launch, every
// block on the tensor cores (see MULTI above).
cudaError_t launch_precond_tc_multi(const hps_handle* h, const float2* t, float2* z, int nrhs, int* d_error,
                                    cudaStream_t st) {
  const ClusterTables& ct = h->ct;
  if (!precond_tc_multi_eligible(h, nrhs) || !d_error) return cudaErrorInvalidValue;
  auto encode = encoder();
  if (!encode) return cudaErrorNotSupported;
  const int q2 = h->q * h->q;
  const int nint = (ct.kc_slot_begin[1] - ct.kc_slot_begin[0]) * q2;  // uniform: every block the same
  const long long tstride = ct.tsize;
  // TMA: 16-byte aligned bases and strides (checked, not assumed)
  if ((reinterpret_cast<uintptr_t>(h->Kc32) | reinterpret_cast<uintptr_t>(t)) % 16 != 0 || (8LL * nint) % 16 != 0 ||
      (8LL * tstride) % 16 != 0)
    return cudaErrorInvalidValue;
  const int smem = kStages * kStageBytes + (int)sizeof(Bars) + 1024;
  cudaError_t e = allow_dynamic_smem((const void*)tc_precond_kernel<true>, smem);
  if (e != cudaSuccess) return e;
  CUtensorMap mapA, mapT;
  {
    // [block][row][2 nint floats], rows nint apart (ld = nint: nint is a multiple of 16)
    cuuint64_t dims[3] = {(cuuint64_t)(2 * nint), (cuuint64_t)nint, (cuuint64_t)ct.nkc};
    cuuint64_t strides[2] = {(cuuint64_t)nint * 8, (cuuint64_t)nint * nint * 8};
    cuuint32_t box[3] = {kTileK, kTileM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (encode(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)h->Kc32, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  {
    // [rhs][position][2 nint floats]; box: 32 floats x 1 member x 64 right-hand sides
    cuuint64_t dims[3] = {(cuuint64_t)(2 * nint), (cuuint64_t)ct.ncl, (cuuint64_t)nrhs};
    cuuint64_t strides[2] = {(cuuint64_t)nint * 8, (cuuint64_t)tstride * 8};
    cuuint32_t box[3] = {kTileK, 1, kMem};
    cuuint32_t es[3] = {1, 1, 1};
    if (encode(&mapT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)t, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  PkArgs a;
  a.nint = nint;
  a.nmem = 0;
  a.mtiles = (nint + kTileM - 1) / kTileM;
  a.ntiles = 0;
  a.kblocks = (2 * nint + kTileK - 1) / kTileK;
  a.q2 = q2;
  a.nb = h->nb;
  a.members = h->dct.kc_members;
  a.cl_slot_begin = h->dct.cl_slot_begin;
  a.slot_lf = h->dct.slot_lf;
  a.z = z;
  a.error = d_error;
  a.gate = h->gate;
  a.pos_class = h->dct.pos_class;
  a.npos = ct.ncl;
  a.rtiles = nrhs / kMem;
  a.nrhs = nrhs;
  a.nf = h->nf;
  const long long items = (long long)a.npos * a.mtiles * a.rtiles;
  const int grid = (int)std::min<long long>(items, h->nsm);
  tc_precond_kernel<true><<<grid, kThreads, smem, st>>>(mapA, mapT, a);
  ++h->prof.launches;
  return cudaGetLastError();
}

}  // namespace hps
