// Stage K of the cluster preconditioner (z_int = K_c t, Sec. 4, Algorithm 4 in
// face form) for every cluster block in one launch, on the 5th-generation
// tensor cores with FP16 operands (kind::f16, FP32 accumulation in TMEM).
//
// Operands:
// * K_c in its FP16 copy (each row divided by its FP32 scale s_row, so that
//   the entries are at most 1), read by TMA as a real n x 2n matrix A of
//   interleaved (re, im) halves: 64 halves (128 bytes) per row and stage;
// * t of each member cluster (complex FP32, the stage-B output) divided by the
//   largest component of that cluster's t (stage B records it) and split by
//   the transform warps into two FP16 terms, hi + lo (~22 bits), each laid out
//   as the rows conj(t) and the re/im swap of t, so that A B_hi + A B_lo =
//   [Re | Im] of K_c t / (s_row t_max).
// The epilogue multiplies back by s_row and t_max.  K_c carries 2^-11 relative
// rounding (a fixed matrix: the FP16 blocks the SIMT stage K uses); t is kept
// to ~2^-22, so the result stays linear in t to FP32 level.  GMRES applies the
// preconditioner to V y in its update and assumes that this equals
// sum_j y_j M^{-1} v_j; with one FP16 rounding of t (2^-11, input-dependent)
// that would hold only to ~2e-4.
//
// Needs the uniform layout (every cluster 2x2x2, 24 q^2 a multiple of 32):
// the blocks are one [block][row][2n halves] array and t one
// [rhs][position][2n floats] array.  Items:
// * one right-hand side: (block k, 128-row tile, first member position, member
//   count <= 64) from a list built at setup; B rows = members;
// * 64, 128, ... right-hand sides: (position, 128-row tile, 64-RHS tile); B
//   rows = right-hand sides of one member.
//
// Warp roles (384 threads, one CTA per SM, persistent, three 64 KB stages):
// warp 0 TMA producer (A tile 128 rows x 128 bytes, two T boxes of 32 floats x
// 64 rows), warp 1 TMEM allocation and the MMA issuer (two MMAs per K chunk:
// hi and lo), warps 2..7 the FP16 conversion of t into the two swizzled B
// tiles, warps 8..11 the epilogue.  Every wait is bounded; on a
// time-out the CTA sets the error word, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>
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
constexpr int kCols = 64;               // B rows per operand half: members or right-hand sides
constexpr int kTileN = 2 * kCols;       // (re, im) accumulator columns
constexpr int kKHalves = 64;            // K extent of a stage (128 bytes of FP16)
constexpr int kABytes = kTileM * 128;   // 16 KB
constexpr int kBBytes = kTileN * 128;   // 16 KB
constexpr int kTBoxBytes = kCols * 128; // 8 KB: 64 rows x 32 floats
// stage layout (1024-byte aligned parts): A | B (high halves of t) | B (low halves) | T box 0 |
// T box 1
constexpr int kTOff = kABytes + 2 * kBBytes;
constexpr int kStageBytes = kTOff + 2 * kTBoxBytes;  // 64 KB
constexpr int kThreads = 384;
constexpr int kTmemCols = 256;

struct Pk16Args {
  int nint, mtiles, kblocks, q2, nb, ncl;
  long long nitems;
  const int4* items;       // one RHS: (block, row tile, first position, count)
  const int* members;      // clusters in stage-K position order
  const int* pos_class;    // block of each position (MULTI)
  const int* kc_slot_begin;
  const int* cl_slot_begin;
  const int* slot_lf;
  const float* kscale;     // FP16 row scales, index kc_slot_begin[k] q^2 + row
  const float* tmax;       // [rhs][cluster] largest |component| of t
  int rtiles, nrhs;
  long long nf;
  float2* z;
  int* error;
  const int* gate;         // while a GMRES cycle is replayed: 0 = return at once
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

// Item decode shared by the roles.
template <bool MULTI>
__device__ __forceinline__ void decode(const Pk16Args& a, long long item, int& blk, int& mt, int& pos0, int& cnt,
                                       int& rt) {
  if (MULTI) {
    const long long per = (long long)a.mtiles * a.rtiles;
    pos0 = (int)(item / per);
    const int rem = (int)(item % per);
    mt = rem / a.rtiles;
    rt = rem % a.rtiles;
    cnt = 1;
    blk = a.pos_class[pos0];
  } else {
    const int4 e = a.items[item];
    blk = e.x;
    mt = e.y;
    pos0 = e.z;
    cnt = e.w;
    rt = 0;
  }
}

// 1 / (largest component of t) of the cluster whose data fills B row m, 0 for unused rows.  A
// maximum below the smallest normal float (a cluster far from every source, whose t holds only
// subnormal values) would overflow the reciprocal: such a cluster's t is taken as 0, a change
// below 2^-126 of the vector's scale.
template <bool MULTI>
__device__ __forceinline__ float inv_scale(const Pk16Args& a, int m, int pos0, int cnt, int rt) {
  float mx;
  if (MULTI) {
    const int rhs = rt * kCols + m;
    if (rhs >= a.nrhs) return 0.f;
    mx = a.tmax[(long long)rhs * a.ncl + a.members[pos0]];
  } else {
    if (m >= cnt) return 0.f;
    mx = a.tmax[a.members[pos0 + m]];
  }
  return mx >= 0x1p-126f ? 1.f / mx : 0.f;
}

template <bool MULTI>
__global__ void __launch_bounds__(kThreads, 1)
    tc_precond16_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapT,
                        Pk16Args a) {
  if (a.gate && *a.gate == 0) return;  // before any barrier or TMEM allocation
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* ring = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  Bars* bars = reinterpret_cast<Bars*>(ring + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

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
      for (long long item = blockIdx.x; item < a.nitems && ok; item += gridDim.x) {
        int blk, mt, pos0, cnt, rt;
        decode<MULTI>(a, item, blk, mt, pos0, cnt, rt);
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t ph = (uint32_t)((it / kStages) & 1);
          if (bars->abort || (it >= kStages && !mbar_wait(&bars->empty[s], ph ^ 1))) {
            fail();
            ok = false;
            break;
          }
          unsigned char* st = ring + s * kStageBytes;
          mbar_expect_tx(&bars->full[s], kABytes + 2 * kTBoxBytes);
          tma_load_3d(st, &mapA, &bars->full[s], kb * kKHalves, mt * kTileM, blk);
          unsigned char* tdst = st + kTOff;
          for (int b = 0; b < 2; ++b) {
            const int x = kb * kKHalves + b * 32;  // floats of t: the same K range as the halves of A
            if (MULTI) tma_load_3d(tdst + b * kTBoxBytes, &mapT, &bars->full[s], x, pos0, rt * kCols);
            else tma_load_2d(tdst + b * kTBoxBytes, &mapT, &bars->full[s], x, pos0);
          }
        }
      }
      for (long long j = (it > kStages ? it - kStages : 0); j < it; ++j)
        if (!mbar_wait(&bars->full[(int)(j % kStages)], (uint32_t)((j / kStages) & 1))) fail();
    }
  } else if (warp >= 2 && warp < 8) {
    // ---------------- t -> FP16 B operand (conj rows, swap rows), 128-byte swizzle ----------------
    const int tt = threadIdx.x - 64;  // 0..191
    constexpr int kTasks = kCols * 8, kPer = (kTasks + 191) / 192;
    long long it = 0;
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
      int blk, mt, pos0, cnt, rt;
      decode<MULTI>(a, item, blk, mt, pos0, cnt, rt);
      // a thread fills the same B rows at every K step: their scales once per item
      float scr[kPer];
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const int task = tt + 192 * i;
        scr[i] = task < kTasks ? inv_scale<MULTI>(a, task >> 3, pos0, cnt, rt) : 0.f;
      }
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kStages);
        const uint32_t ph = (uint32_t)((it / kStages) & 1);
        if (bars->abort || !mbar_wait(&bars->full[s], ph)) {
          fail();
          goto split_done;
        }
        unsigned char* st = ring + s * kStageBytes;
        unsigned char* B = st + kABytes;
        unsigned char* Blo = B + kBBytes;
        const unsigned char* T = st + kTOff;
        // task = (row m, 16-byte chunk c of the B row): 4 complex values of K index 4c..4c+3,
        // which are floats 8(c%4)..8(c%4)+7 of T box c/4, row m (two 16-byte T chunks)
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
          const int task = tt + 192 * i;
          if (task >= kTasks) break;
          const int m = task >> 3, c = task & 7;
          const float sc = scr[i];
          const unsigned char* trow = T + (c >> 2) * kTBoxBytes + m * 128;
          const int ch0 = 2 * (c & 3);
          const float4 p0 = *reinterpret_cast<const float4*>(trow + ((ch0 ^ (m & 7)) << 4));
          const float4 p1 = *reinterpret_cast<const float4*>(trow + (((ch0 + 1) ^ (m & 7)) << 4));
          // t / t_max = hi + lo in two FP16 terms (~22 bits): the product stays linear in t to
          // FP32 level, as the Krylov update, which applies the preconditioner to V y, needs
          const float x[8] = {p0.x * sc, p0.y * sc, p0.z * sc, p0.w * sc, p1.x * sc, p1.y * sc, p1.z * sc, p1.w * sc};
          uint32_t cjh[4], swh[4], cjl[4], swl[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const __half2 h = __floats2half2_rn(x[2 * e], x[2 * e + 1]);  // (re, im) high parts
            const __half2 l = __floats2half2_rn(x[2 * e] - __low2float(h), x[2 * e + 1] - __high2float(h));
            // conj row (re, -im), swap row (im, re); negation is exact in FP16
            const __half2 hc = __halves2half2(__low2half(h), __hneg(__high2half(h)));
            const __half2 hs = __halves2half2(__high2half(h), __low2half(h));
            const __half2 lc = __halves2half2(__low2half(l), __hneg(__high2half(l)));
            const __half2 ls = __halves2half2(__high2half(l), __low2half(l));
            cjh[e] = *reinterpret_cast<const uint32_t*>(&hc);
            swh[e] = *reinterpret_cast<const uint32_t*>(&hs);
            cjl[e] = *reinterpret_cast<const uint32_t*>(&lc);
            swl[e] = *reinterpret_cast<const uint32_t*>(&ls);
          }
          const int pc = (c ^ (m & 7)) << 4;  // rows m and 64 + m share the swizzle phase
          *reinterpret_cast<uint4*>(B + m * 128 + pc) = make_uint4(cjh[0], cjh[1], cjh[2], cjh[3]);
          *reinterpret_cast<uint4*>(B + (kCols + m) * 128 + pc) = make_uint4(swh[0], swh[1], swh[2], swh[3]);
          *reinterpret_cast<uint4*>(Blo + m * 128 + pc) = make_uint4(cjl[0], cjl[1], cjl[2], cjl[3]);
          *reinterpret_cast<uint4*>(Blo + (kCols + m) * 128 + pc) = make_uint4(swl[0], swl[1], swl[2], swl[3]);
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
      const uint32_t idesc = instr_desc_f16(kTileN, kTileM);
      long long it = 0;
      long long local = 0;
      bool ok = true;
      for (long long item = blockIdx.x; item < a.nitems && ok; item += gridDim.x, ++local) {
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
          const uint32_t aa = base, bb = base + kABytes, bl = bb + kBBytes;
#pragma unroll
          for (int kk = 0; kk < kKHalves / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 halves
            mma_f16(acc, smem_desc(aa + off), smem_desc(bb + off), idesc, (kb == 0 && kk == 0) ? 0u : 1u);
            mma_f16(acc, smem_desc(aa + off), smem_desc(bl + off), idesc, 1u);
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
    for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x, ++local) {
      const int b = (int)(local & 1);
      if (bars->abort || !mbar_wait(&bars->acc_full[b], (uint32_t)((local >> 1) & 1))) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int blk, mt, pos0, cnt, rt;
      decode<MULTI>(a, item, blk, mt, pos0, cnt, rt);
      const int row = mt * kTileM + ew * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(b * kTileN);
      const float ks = (row < a.nint) ? a.kscale[(long long)a.kc_slot_begin[blk] * a.q2 + row] : 0.f;
      float re[32], im[32];
      for (int half = 0; half < 2; ++half) {
        tmem_ld32(taddr + half * 32, re);
        tmem_ld32(taddr + kCols + half * 32, im);
        if (row < a.nint) {
          const int sl = row / a.q2, j = row % a.q2;
          if (MULTI) {
            const int cl = a.members[pos0];
            const int lf = a.slot_lf[a.cl_slot_begin[cl] + sl];
            const long long o = (long long)(lf / 6) * a.nb + (long long)(lf % 6) * a.q2 + j;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int rhs = rt * kCols + half * 32 + c;
              if (rhs < a.nrhs) {
                const float f = ks * a.tmax[(long long)rhs * a.ncl + cl];
                a.z[(long long)rhs * a.nf + o] = make_float2(re[c] * f, im[c] * f);
              }
            }
          } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
              const int m = half * 32 + c;
              if (m < cnt) {
                const int cl = a.members[pos0 + m];
                const int lf = a.slot_lf[a.cl_slot_begin[cl] + sl];
                const float f = ks * a.tmax[cl];
                a.z[(long long)(lf / 6) * a.nb + (long long)(lf % 6) * a.q2 + j] = make_float2(re[c] * f, im[c] * f);
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

bool precond_tc16_eligible(const hps_handle* h, int nrhs) {
  return h->has_precond && h->opt.tc_apply && h->Kc16 && h->Kc16s && h->tc_error && h->tmax && h->ct.uniform &&
         h->ct.nslots > 0 && (h->ct.nint0 % 32 == 0) && nrhs <= h->tmax_rhs &&
         (nrhs == 1 || (nrhs >= kCols && nrhs % kCols == 0));
}

// z_int = K_c t for every cluster (FP16 blocks, FP16 t scaled per cluster by tmax), one launch.
cudaError_t launch_precond_tc16(const hps_handle* h, const float2* t, float2* z, int nrhs, cudaStream_t st) {
  const ClusterTables& ct = h->ct;
  if (!precond_tc16_eligible(h, nrhs)) return cudaErrorInvalidValue;
  auto encode = encoder();
  if (!encode) return cudaErrorNotSupported;
  const int q2 = h->q * h->q;
  const int nint = ct.nint0;
  const long long tstride = ct.tsize;
  // TMA: 16-byte aligned bases and strides (checked, not assumed)
  if ((reinterpret_cast<uintptr_t>(h->Kc16) | reinterpret_cast<uintptr_t>(t)) % 16 != 0 || (4LL * nint) % 16 != 0 ||
      (8LL * nint) % 16 != 0 || (8LL * tstride) % 16 != 0)
    return cudaErrorInvalidValue;
  const bool multi = nrhs > 1;
  const int smem = kStages * kStageBytes + (int)sizeof(Bars) + 1024;
  auto kern = multi ? tc_precond16_kernel<true> : tc_precond16_kernel<false>;
  cudaError_t e = allow_dynamic_smem((const void*)kern, smem);
  if (e != cudaSuccess) return e;
  CUtensorMap mapA, mapT;
  {
    // FP16 blocks [block][row][2 nint halves], rows nint complex apart
    cuuint64_t dims[3] = {(cuuint64_t)(2 * nint), (cuuint64_t)nint, (cuuint64_t)ct.nkc};
    cuuint64_t strides[2] = {(cuuint64_t)nint * 4, (cuuint64_t)nint * nint * 4};
    cuuint32_t box[3] = {kKHalves, kTileM, 1};
    cuuint32_t es[3] = {1, 1, 1};
    if (encode(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)h->Kc16, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  if (multi) {
    // t [rhs][position][2 nint floats]; box 32 floats x 1 member x 64 right-hand sides
    cuuint64_t dims[3] = {(cuuint64_t)(2 * nint), (cuuint64_t)ct.ncl, (cuuint64_t)nrhs};
    cuuint64_t strides[2] = {(cuuint64_t)nint * 8, (cuuint64_t)tstride * 8};
    cuuint32_t box[3] = {32, 1, kCols};
    cuuint32_t es[3] = {1, 1, 1};
    if (encode(&mapT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)t, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  } else {
    // t [position][2 nint floats]; box 32 floats x 64 members
    cuuint64_t dims[2] = {(cuuint64_t)(2 * nint), (cuuint64_t)ct.ncl};
    cuuint64_t strides[1] = {(cuuint64_t)nint * 8};
    cuuint32_t box[2] = {32, kCols};
    cuuint32_t es[2] = {1, 1};
    if (encode(&mapT, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)t, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  Pk16Args a;
  a.nint = nint;
  a.mtiles = (nint + kTileM - 1) / kTileM;
  a.kblocks = 2 * nint / kKHalves;
  a.q2 = q2;
  a.nb = h->nb;
  a.ncl = ct.ncl;
  a.items = h->dct.tc16_items;
  a.members = h->dct.kc_members;
  a.pos_class = h->dct.pos_class;
  a.kc_slot_begin = h->dct.kc_slot_begin;
  a.cl_slot_begin = h->dct.cl_slot_begin;
  a.slot_lf = h->dct.slot_lf;
  a.kscale = h->Kc16s;
  a.tmax = h->tmax;
  a.rtiles = multi ? nrhs / kCols : 1;
  a.nrhs = nrhs;
  a.nf = h->nf;
  a.z = z;
  a.error = h->tc_error;
  a.gate = h->gate;
  a.nitems = multi ? (long long)ct.ncl * a.mtiles * a.rtiles : (long long)ct.tc16_items.size();
  if (a.nitems == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(a.nitems, h->nsm);
  kern<<<grid, kThreads, smem, st>>>(mapA, mapT, a);
  ++h->prof.launches;
  return cudaGetLastError();
}

}  // namespace hps
