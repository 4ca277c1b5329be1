// hps_precond_noalloc: the preconditioner apply with its scratch buffer in a
// fixed device array compiled into the library, so the call itself never
// allocates device memory.
//
// Who needs it: a host process that hands all of the GPU's memory to its own
// pool or allocator at start-up (a serving process, a framework with a
// caching allocator, a plugin that must stay inside a memory budget it does
// not control) cannot have a library call cudaMalloc behind its back: the
// allocation may fail, fragment the pool, or implicitly synchronize the
// device in a latency-critical loop.  hps_precond takes its scratch from the
// handle instead; this variant takes it from the static array below.
#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {

// The scratch holds the cluster-internal right-hand sides t (stage B output,
// stage K input): tsize * nrhs complex values of the call's type (tsize: the
// internal-face values of all clusters, blocks padded to 16 values).
// Every device that loads the library reserves these bytes until the process exits.
constexpr size_t kNoAllocScratchBytes = HPS_PRECOND_NOALLOC_MAX_BYTES;

static __device__ __align__(256) unsigned char g_precond_scratch[kNoAllocScratchBytes];

// Device address of g_precond_scratch in the current device's copy of the
// library's device code, looked up on every call (cudaGetSymbolAddress is a
// host-side lookup that allocates nothing).  Not cached: a cached address
// would dangle after the device or its primary context is reset and the
// module reloaded.  In host code the name g_precond_scratch is only a
// host-side handle for the symbol, never a device address, so it is not
// passed to a kernel.
int scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_precond_scratch);
  if (e != cudaSuccess || !p) {
    set_error(std::string("hps_precond_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    return HPS_ECUDA;
  }
  *out = p;
  return HPS_OK;
}

}  // namespace

}  // namespace hps

using namespace hps;

extern "C" {

int hps_precond_noalloc(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream) {
  if (!h || !r || !z || nrhs < 1) {
    set_error("hps_precond_noalloc: bad arguments");
    return HPS_EINVAL;
  }
  if (dtype != HPS_C128 && dtype != HPS_C64 && dtype != HPS_C64_H16) {
    set_error("hps_precond_noalloc: unknown dtype");
    return HPS_EINVAL;
  }
  const size_t es = (dtype == HPS_C128) ? sizeof(double2) : sizeof(float2);
  const size_t need = (size_t)h->ct.tsize * (size_t)nrhs * es;
  if (need > kNoAllocScratchBytes) {
    set_error("hps_precond_noalloc: needs " + std::to_string(need) + " bytes of scratch, more than the " +
              std::to_string(kNoAllocScratchBytes) + "-byte static buffer; use hps_precond or fewer right-hand sides");
    return HPS_EINVAL;
  }
  // the same operator choices as hps_precond
  if (dtype == HPS_C128 && h->has_precond && !h->Kc64) {
    set_error("hps_precond_noalloc: FP64 preconditioner was not built (HPS_FORM_FP64)");
    return HPS_EINVAL;
  }
  if (dtype == HPS_C64_H16 && h->has_precond && !h->Kc16) {
    set_error("hps_precond_noalloc: FP16 preconditioner blocks were not built (options.precond_fp16)");
    return HPS_EINVAL;
  }
  if (dtype == HPS_C64 && h->has_precond && !h->Kc32 && !h->Kc16) {
    set_error("hps_precond_noalloc: FP32 preconditioner was not built (HPS_FORM_MIXED)");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->has_precond) {
    HPS_CUDA_TRY(cudaMemcpyAsync(z, r, (size_t)nrhs * h->nf * es, cudaMemcpyDeviceToDevice, st));
    return HPS_OK;
  }
  void* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc) return rc;
  // Stage B writes every internal slot of t before stage K reads it, so the
  // contents left by an earlier call need no clearing.
  // No event timing here: the profiler may create events on first use.
  const bool prof_on = h->prof.on;
  h->prof.on = false;
  // complex float: the FP16 copies for HPS_C64_H16, and for HPS_C64 when the handle keeps the
  // cluster inverses in FP16 only (lean mode), as hps_precond does
  cudaError_t e = (dtype == HPS_C128)
                      ? launch_precond(h, false, VType::C128, r, VType::C128, z, scratch, nrhs, st)
                      : launch_precond(h, true, VType::C64, r, VType::C64, z, scratch, nrhs, st,
                                       dtype == HPS_C64_H16 || !h->Kc32);
  h->prof.on = prof_on;
  HPS_CUDA_TRY(e);
  return HPS_OK;
}

}  // extern "C"
