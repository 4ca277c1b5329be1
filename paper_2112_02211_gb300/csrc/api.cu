// C ABI of the HPS library (declared in include/hps.h).  Argument checks,
// allocation of the handle's device state, and dispatch to the kernels of
// setup.cu, apply.cu and krylov.cu.  Nothing here throws across the ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "hps_internal.h"

namespace hps {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }

cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> limits;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_pair(kernel, dev);
  auto it = limits.find(key);
  if (it == limits.end()) {
    int mx = 0;
    e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    // the opt-in maximum covers static plus dynamic shared memory
    const int dyn = mx - (int)fa.sharedSizeBytes;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    it = limits.emplace(key, dyn).first;
  }
  return bytes <= (size_t)it->second ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_cdiag(const double2* b, double kappa, long long count, double2* c, cudaStream_t st);

}  // namespace hps

using namespace hps;

namespace {

int validate_grid(const hps_grid* g) {
  if (!g) {
    set_error("grid is NULL");
    return HPS_EINVAL;
  }
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > 4096 || g->ny > 4096 || g->nz > 4096) {
    set_error("leaf counts per axis must be in 1..4096");
    return HPS_EINVAL;
  }
  if ((long long)g->nx * g->ny * g->nz > (1LL << 22)) {
    set_error("too many leaves");
    return HPS_EINVAL;
  }
  if (g->p < 4 || g->p > 16) {
    set_error("Chebyshev order p must be in 4..16");
    return HPS_EINVAL;
  }
  if (g->q != g->p - 2) {
    set_error("q must equal p - 2 (square Chebyshev-to-Gauss face interpolation)");
    return HPS_EINVAL;
  }
  return HPS_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int dalloc(hps_handle* h, void** p, size_t bytes) {
  bytes = bytes ? bytes : 16;
  if (h->opt.hbm_budget && h->bytes + bytes > h->opt.hbm_budget) {
    set_error("allocation exceeds the HBM budget of the handle");
    return HPS_ENOMEM;
  }
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    return HPS_ENOMEM;
  }
  h->bytes += bytes;
  return HPS_OK;
}

void free_handle(hps_handle* h) {
  if (!h) return;
  cudaSetDevice(h->dev);
  if (h->stream) cudaStreamSynchronize(h->stream);
  krylov_free(h);
  void* ptrs[] = {h->tables, h->R64, h->R32, h->H64, h->H32, h->R16lo, h->R16ls, h->H16lo, h->H16ls, h->lambda, h->lambda_q, h->Kc64, h->Kc32, h->B64,
                  h->B32, h->pc_scratch, h->Kc16, h->Kc16s, h->B16, h->B16s, h->tc_error, h->cdiag,
                  h->dct.slot_lf, h->dct.slot_cluster, h->dct.cl_slot_begin, h->dct.cl_kc_off, h->dct.lf_slot,
                  h->dct.int_mask, h->dct.b_off, h->dct.leaf_bcls, h->dct.bc_rep, h->dct.kc_off,
                  h->dct.kc_slot_begin, h->dct.kslot_class, h->dct.kc_members, h->dct.kitems[0], h->dct.kitems[1],
                  h->dct.kitems[2], h->dct.kitems[3], h->dct.cl_tpos, h->dct.lf_tpos, h->dct.brd, h->dct.bto,
                  h->dct.bsc, h->dct.pos_class, h->dct.leaf_cluster, h->dct.tc16_items, h->dct.bgroup_leaves, h->dct.bgroups, h->tmax, h->fs.d_cls, h->fs.Sinv64, h->fs.Sinv32, h->fs.eig};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

void init_fields(hps_handle* h, const hps_grid* g, double kappa, double eta, const hps_options& o) {
  h->opt = o;
  h->dev = o.device;
  h->nx = g->nx;
  h->ny = g->ny;
  h->nz = g->nz;
  h->p = g->p;
  h->q = g->q;
  h->n1 = g->p - 2;
  h->ni = h->n1 * h->n1 * h->n1;
  h->nb = 6 * h->q * h->q;
  h->n = h->ni + h->nb;
  h->nl = g->nx * g->ny * g->nz;
  h->nf = (long long)h->nl * h->nb;
  h->nint = (long long)h->nl * h->ni;
  h->kappa = kappa;
  h->eta = eta;
  h->h[0] = 1.0 / g->nx;
  h->h[1] = 1.0 / g->ny;
  h->h[2] = 1.0 / g->nz;
  h->tl = TableLayout(g->p);
  h->ldR = (int)rup4(h->nb);
  h->ldH = (int)rup4(h->ni);
}

int check_options(const hps_options& o) {
  if (o.restart < 1 || o.restart > 60) {
    set_error("restart must be in 1..60");
    return HPS_EINVAL;
  }
  if (o.cluster != 0 && o.cluster != 2) {
    set_error("cluster must be 0 (no preconditioner) or 2");
    return HPS_EINVAL;
  }
  if (o.max_rhs < 1 || o.max_rhs > 1024 || o.maxit < 1 || !(o.forms & (HPS_FORM_FP64 | HPS_FORM_MIXED))) {
    set_error("bad options (max_rhs, maxit or forms)");
    return HPS_EINVAL;
  }
  if (o.lean && o.forms != HPS_FORM_MIXED) {
    set_error("lean mode keeps FP32 maps only: forms must be HPS_FORM_MIXED");
    return HPS_EINVAL;
  }
  if (!std::isfinite(o.lambda_bin) || o.lambda_bin < 0.0) {
    set_error("lambda_bin must be finite and >= 0");
    return HPS_EINVAL;
  }
  return HPS_OK;
}

constexpr int kSolveFlagBits = HPS_SOLVE_NO_PRECOND | HPS_SOLVE_X0 | HPS_SOLVE_NO_GRAPH | HPS_SOLVE_CGS2;

SolveFlags solve_flags(int form) {
  SolveFlags f;
  f.x0 = (form & HPS_SOLVE_X0) != 0;
  f.no_graph = (form & HPS_SOLVE_NO_GRAPH) != 0;
  f.cgs2 = (form & HPS_SOLVE_CGS2) != 0;
  return f;
}

int check_finite(const double* v, long long n, const char* what) {
  for (long long i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) {
      set_error(std::string(what) + " contains NaN or Inf");
      return HPS_EINVAL;
    }
  return HPS_OK;
}

}  // namespace

extern "C" {

void hps_default_options(hps_options* o) {
  if (!o) return;
  o->forms = HPS_FORM_FP64 | HPS_FORM_MIXED;
  o->restart = 50;
  o->cluster = 2;
  o->maxit = 5000;
  o->max_rhs = 1;
  o->hbm_budget = 0;
  o->device = 0;
  o->precond_fp16 = 1;
  o->tc_apply = 1;
  o->lean = 0;
  o->lambda_bin = 0.0;
  o->autotune = 1;
  o->full_system = 0;
}

const char* hps_last_error(void) { return g_err.c_str(); }

int hps_nodes(const hps_grid* g, double* xi, double* xf, double* xc) {
  int rc = validate_grid(g);
  if (rc) return rc;
  TableLayout tl(g->p);
  const long long nl = (long long)g->nx * g->ny * g->nz;
  const long long ni = (long long)(g->p - 2) * (g->p - 2) * (g->p - 2), nb = 6LL * g->q * g->q;
  double *T = nullptr, *dxi = nullptr, *dxf = nullptr, *dxc = nullptr;
  auto cleanup = [&]() {
    if (T) cudaFree(T);
    if (dxi) cudaFree(dxi);
    if (dxf) cudaFree(dxf);
    if (dxc) cudaFree(dxc);
  };
  auto body = [&]() -> int {
    HPS_CUDA_TRY(cudaMalloc(&T, tl.total * sizeof(double)));
    if (xi) HPS_CUDA_TRY(cudaMalloc(&dxi, nl * ni * 3 * sizeof(double)));
    if (xf) HPS_CUDA_TRY(cudaMalloc(&dxf, nl * nb * 3 * sizeof(double)));
    if (xc) HPS_CUDA_TRY(cudaMalloc(&dxc, nl * nb * 3 * sizeof(double)));
    HPS_CUDA_TRY(launch_tables(T, tl, 1.0 / g->nx, 1.0 / g->ny, 1.0 / g->nz, 0));
    HPS_CUDA_TRY(launch_nodes(T, tl, g->nx, g->ny, g->nz, dxi, dxf, dxc, 0));
    if (xi) HPS_CUDA_TRY(cudaMemcpy(xi, dxi, nl * ni * 3 * sizeof(double), cudaMemcpyDeviceToHost));
    if (xf) HPS_CUDA_TRY(cudaMemcpy(xf, dxf, nl * nb * 3 * sizeof(double), cudaMemcpyDeviceToHost));
    if (xc) HPS_CUDA_TRY(cudaMemcpy(xc, dxc, nl * nb * 3 * sizeof(double), cudaMemcpyDeviceToHost));
    return HPS_OK;
  };
  rc = body();
  cleanup();
  return rc;
}

int hps_setup(const hps_grid* g, double kappa, double eta, const double* b, const hps_options* opt,
              hps_handle** out) {
  if (!out) {
    set_error("out is NULL");
    return HPS_EINVAL;
  }
  *out = nullptr;
  int rc = validate_grid(g);
  if (rc) return rc;
  if (!std::isfinite(kappa) || !std::isfinite(eta) || eta == 0.0) {
    set_error("kappa must be finite and eta finite with Re(eta) != 0");
    return HPS_EINVAL;
  }
  hps_options o;
  hps_default_options(&o);
  if (opt) o = *opt;
  if ((rc = check_options(o))) return rc;
  hps_handle* h = new hps_handle();
  init_fields(h, g, kappa, eta, o);
  if (b && (rc = check_finite(b, 2 * h->nint, "b"))) {
    delete h;
    return rc;
  }
  double2 *db = nullptr, *dc = nullptr;
  auto body = [&]() -> int {
    HPS_CUDA_TRY(cudaSetDevice(h->dev));
    HPS_CUDA_TRY(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev));
    HPS_CUDA_TRY(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    cudaStream_t st = h->stream;
    const bool want64 = (o.forms & HPS_FORM_FP64) != 0;
    const bool want32 = (o.forms & HPS_FORM_MIXED) != 0;
    int r;
    if ((r = dalloc(h, (void**)&h->tables, h->tl.total * sizeof(double)))) return r;
    const size_t rel = (size_t)h->nl * h->nb * h->ldR;
    const size_t hel = (size_t)h->nl * h->nb * h->ldH;
    if (!o.lean && (r = dalloc(h, (void**)&h->R64, rel * sizeof(double2)))) return r;
    if (want32 && (r = dalloc(h, (void**)&h->R32, rel * sizeof(float2)))) return r;
    if (!o.lean && (r = dalloc(h, (void**)&h->H64, hel * sizeof(double2)))) return r;
    // complex-FP32 H and the FP16 remainders of the FP32 maps (compensated maps, compensated.cu):
    // lean mode's only accurate maps, and the mixed form's fast restart residual and right-hand
    // side at tolerances >= 1e-8
    if (want32 && (r = dalloc(h, (void**)&h->H32, hel * sizeof(float2)))) return r;
    if (want32) {
      if ((r = dalloc(h, (void**)&h->R16lo, rel * sizeof(__half2)))) return r;
      if ((r = dalloc(h, (void**)&h->R16ls, (size_t)h->nl * h->nb * sizeof(float)))) return r;
      if ((r = dalloc(h, (void**)&h->H16lo, hel * sizeof(__half2)))) return r;
      if ((r = dalloc(h, (void**)&h->H16ls, (size_t)h->nl * h->nb * sizeof(float)))) return r;
    }
    if ((r = dalloc(h, (void**)&h->lambda, (size_t)h->nl * sizeof(double2)))) return r;
    if ((r = dalloc(h, (void**)&h->tc_error, sizeof(int)))) return r;
    HPS_CUDA_TRY(cudaMemsetAsync(h->tc_error, 0, sizeof(int), st));
    if (h->R64) HPS_CUDA_TRY(cudaMemsetAsync(h->R64, 0, rel * sizeof(double2), st));
    if (h->R32) HPS_CUDA_TRY(cudaMemsetAsync(h->R32, 0, rel * sizeof(float2), st));
    if (h->H64) HPS_CUDA_TRY(cudaMemsetAsync(h->H64, 0, hel * sizeof(double2), st));
    if (h->H32) HPS_CUDA_TRY(cudaMemsetAsync(h->H32, 0, hel * sizeof(float2), st));
    HPS_CUDA_TRY(cudaMalloc(&db, (size_t)h->nint * sizeof(double2)));
    if ((r = dalloc(h, (void**)&h->cdiag, (size_t)h->nint * sizeof(double2)))) return r;
    dc = h->cdiag;
    if (b)
      HPS_CUDA_TRY(cudaMemcpyAsync(db, b, (size_t)h->nint * sizeof(double2), cudaMemcpyHostToDevice, st));
    else
      HPS_CUDA_TRY(cudaMemsetAsync(db, 0, (size_t)h->nint * sizeof(double2), st));
    HPS_CUDA_TRY(launch_tables(h->tables, h->tl, h->h[0], h->h[1], h->h[2], st));
    HPS_CUDA_TRY(launch_cdiag(db, kappa, h->nint, dc, st));
    if ((r = build_exact_maps(h, dc, st))) return r;
    if (o.cluster == 2) {
      build_cluster_tables(h, 2);
      h->has_precond = true;
      if ((r = classify_preconditioner(h, dc, st))) return r;
      const ClusterTables& ct = h->ct;
      const size_t ke = std::max<long long>(1, ct.kc_elems), be = std::max<long long>(1, ct.b_elems);
      if (want64) {
        if ((r = dalloc(h, (void**)&h->Kc64, ke * sizeof(double2)))) return r;
        if ((r = dalloc(h, (void**)&h->B64, be * sizeof(double2)))) return r;
        HPS_CUDA_TRY(cudaMemsetAsync(h->Kc64, 0, ke * sizeof(double2), st));
        HPS_CUDA_TRY(cudaMemsetAsync(h->B64, 0, be * sizeof(double2), st));
      }
      const bool fp16 = want32 && (o.precond_fp16 || o.lean);
      // lean mode keeps K_c only in FP16, except when the shared blocks are few enough that
      // their complex-FP32 copies (needed by the tensor-core stage K) take at most 4 GiB
      // (and when solves with 64 or more right-hand sides will run stage K on the tensor cores)
      const bool kc32 = !o.lean || (!ct.kc_tc.empty() && ke * sizeof(float2) <= ((size_t)4 << 30)) ||
                        (o.tc_apply && ct.uniform && o.max_rhs >= 64);
      if (want32) {
        if (kc32 && (r = dalloc(h, (void**)&h->Kc32, ke * sizeof(float2)))) return r;
        if ((r = dalloc(h, (void**)&h->B32, be * sizeof(float2)))) return r;
        if (h->Kc32) HPS_CUDA_TRY(cudaMemsetAsync(h->Kc32, 0, ke * sizeof(float2), st));
        HPS_CUDA_TRY(cudaMemsetAsync(h->B32, 0, be * sizeof(float2), st));
      }
      if (fp16) {
        const int q2 = h->q * h->q;
        if ((r = dalloc(h, (void**)&h->Kc16, ke * sizeof(__half2)))) return r;
        if ((r = dalloc(h, (void**)&h->B16, be * sizeof(__half2)))) return r;
        const size_t kr = std::max<size_t>(1, (size_t)ct.kc_slot_begin[ct.nkc] * q2);
        if ((r = dalloc(h, (void**)&h->Kc16s, kr * sizeof(float)))) return r;
        if ((r = dalloc(h, (void**)&h->B16s, std::max<size_t>(1, (size_t)ct.nbc * 6 * q2) * sizeof(float)))) return r;
        HPS_CUDA_TRY(cudaMemsetAsync(h->Kc16, 0, ke * sizeof(__half2), st));
        HPS_CUDA_TRY(cudaMemsetAsync(h->B16, 0, be * sizeof(__half2), st));
      }
      const size_t ts = (size_t)ct.tsize * o.max_rhs * sizeof(double2);
      if ((r = dalloc(h, &h->pc_scratch, ts))) return r;
      if (fp16) {  // per-cluster scales of t for the FP16 tensor-core stage K
        if ((r = dalloc(h, (void**)&h->tmax, (size_t)ct.ncl * o.max_rhs * sizeof(float)))) return r;
        h->tmax_rhs = o.max_rhs;
      }
      if ((r = build_preconditioner(h, dc, st))) return r;
      if (fp16 && (r = build_precond_fp16(h, st))) return r;
    }
    if (o.full_system && (r = build_full_system(h, dc, st))) return r;
    if (o.autotune && (r = autotune_shapes(h, st))) return r;
    HPS_CUDA_TRY(cudaStreamSynchronize(st));
    return HPS_OK;
  };
  rc = body();
  if (db) cudaFree(db);
  if (rc) {
    free_handle(h);
    return rc;
  }
  *out = h;
  return HPS_OK;
}

size_t hps_setup_bytes(const hps_grid* g, const hps_options* opt, int nrhs) {
  if (validate_grid(g)) return 0;
  hps_options o;
  hps_default_options(&o);
  if (opt) o = *opt;
  if (check_options(o) || nrhs < 1) return 0;
  hps_handle h;
  init_fields(&h, g, 1.0, 1.0, o);
  if (cudaDeviceGetAttribute(&h.nsm, cudaDevAttrMultiProcessorCount, o.device) != cudaSuccess) {
    cudaGetLastError();
    h.nsm = 152;
  }
  const bool want64 = (o.forms & HPS_FORM_FP64) != 0, want32 = (o.forms & HPS_FORM_MIXED) != 0;
  const size_t c16 = sizeof(double2), c8 = sizeof(float2);
  const size_t rel = (size_t)h.nl * h.nb * h.ldR;
  const size_t hel = (size_t)h.nl * h.nb * h.ldH;
  size_t bytes = h.tl.total * sizeof(double) + (o.lean ? 0 : rel * c16) + (want32 ? rel * c8 : 0) +
                 hel * (o.lean ? c8 : c16) + (size_t)h.nl * c16;
  if (want32)  // FP16 remainders of R and H and their row scales; FP32 H beside FP64 H
    bytes += (rel + hel) * sizeof(__half2) + (size_t)2 * h.nl * h.nb * sizeof(float) + (o.lean ? 0 : hel * c8);
  const int q2 = h.q * h.q;
  size_t nslots = 0, tsize = 1;
  if (o.cluster == 2) {
    build_cluster_tables(&h, 2);
    const ClusterTables& ct = h.ct;
    nslots = ct.nslots;
    bytes += 2 * ct.slot_lf.size() * sizeof(int) + ct.cl_slot_begin.size() * sizeof(int) +
             ct.cl_kc_off.size() * sizeof(long long) + ct.lf_slot.size() * sizeof(int) + ct.int_mask.size() +
             ct.b_off.size() * sizeof(long long);
    bytes += (size_t)h.nl * (2 * sizeof(int) + c16) + ct.kc_off.size() * sizeof(long long) +
             (ct.kc_slot_begin.size() + ct.kslot_class.size() + ct.kc_members.size()) * sizeof(int);
    for (const auto& v : ct.kitems) bytes += std::max<size_t>(1, v.size()) * sizeof(int4);
    bytes += (size_t)h.nl * 6 * 3 * sizeof(int) + (size_t)ct.ncl * sizeof(long long) +
             (size_t)h.nl * 6 * sizeof(long long);  // stage-B offsets, t positions
    if (want64) bytes += (size_t)(ct.kc_elems + ct.b_elems) * c16;
    if (want32) bytes += (size_t)((o.lean ? 0 : ct.kc_elems) + ct.b_elems) * c8;
    if (want32 && o.lean)  // complex-FP32 copies of shared blocks (if any), capped; all of them for
                           // the multi-RHS tensor-core stage K
      bytes += (o.tc_apply && ct.uniform && o.max_rhs >= 64) ? (size_t)ct.kc_elems * c8
                                                              : std::min<size_t>((size_t)ct.kc_elems * c8, (size_t)4 << 30);
    bytes += (size_t)ct.ncl * sizeof(int) + (size_t)h.nl * sizeof(int) +      // position -> block, leaf -> cluster
             (size_t)ct.ncl * o.max_rhs * sizeof(float) + ct.tc16_items.size() * sizeof(int4) +  // t scales, items
             (size_t)h.nl * (sizeof(int) + sizeof(int2));  // stage-B groups
    if (want32 && (o.precond_fp16 || o.lean))
      bytes += (size_t)(ct.kc_elems + ct.b_elems) * sizeof(__half2) + nslots * q2 * sizeof(float) +
               (size_t)h.nl * 6 * q2 * sizeof(float);
    bytes += (size_t)ct.tsize * o.max_rhs * c16;
    tsize = ct.tsize;
  }
  bytes += (size_t)h.nint * c16 + sizeof(int);  // medium C kept for recovery, error word
  if (o.full_system)  // S~^{-1} per leaf at most, class index, lambda values, Algorithm 3 tables
    bytes += (size_t)h.nl * h.nb * h.nb * ((want64 && !o.lean ? c16 : 0) + (want32 ? c8 : 0)) +
             (size_t)h.nl * (sizeof(int) + c16) + (size_t)3 * (2 * h.n1 * h.n1 + h.n1) * sizeof(double);
  // Krylov workspace of one solve (host inputs staged on the device)
  const int M1 = o.restart + 1;
  const size_t vb = (size_t)nrhs * h.nf * c16;
  const long long nblk = (h.nf + 1023) / 1024;
  bytes += vb * (M1 + 5) + tsize * nrhs * c16 + (size_t)nrhs * nblk * M1 * c16 +
           (size_t)o.max_rhs * (h.nint + h.nf) * c16 + (size_t)nrhs * (3 * M1 + 4 * o.restart + 8) * c16 +
           (size_t)nrhs * std::max<long long>(256, nblk) * sizeof(double);
  // transient setup workspace (largest phase) + medium staging
  const size_t cap = workspace_cap(&h);
  size_t trans = exact_maps_workspace(&h, cap, nullptr);
  if (o.cluster == 2) trans = std::max(trans, precond_workspace(&h, cap, nullptr));
  return bytes + trans + (size_t)h.nint * c16;
}

int hps_apply(hps_handle* h, int dtype, const void* f, void* y, int nrhs, void* stream) {
  if (!h || !f || !y || nrhs < 1) {
    set_error("hps_apply: bad arguments");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == HPS_C128) {
    if (!h->R64 && !h->R16lo) {
      set_error("hps_apply: complex-double applies need the FP64 or the compensated FP32 maps");
      return HPS_EINVAL;
    }
    // lean mode: the compensated FP32 maps (FP64-accurate, double-float accumulation)
    HPS_CUDA_TRY(launch_apply(h, h->R64 == nullptr, VType::C128, f, VType::C128, y, nullptr, nrhs, false, st));
  } else if (dtype == HPS_C64) {
    if (!h->R32) {
      set_error("hps_apply: complex-FP32 operators were not built (HPS_FORM_MIXED)");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_apply(h, true, VType::C64, f, VType::C64, y, nullptr, nrhs, false, st));
  } else {
    set_error("hps_apply: unknown dtype");
    return HPS_EINVAL;
  }
  return HPS_OK;
}

int hps_full_apply(hps_handle* h, int dtype, const void* u, void* y, int nrhs, void* stream) {
  if (!h || !u || !y || nrhs < 1 || u == y) {
    set_error("hps_full_apply: bad arguments");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == HPS_C128) {
    if (h->p > 14) {
      set_error("hps_full_apply: complex-double global apply supports p <= 14");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_full_apply(h, true, VType::C128, u, VType::C128, y, nullptr, nrhs, st));
  } else if (dtype == HPS_C64) {
    HPS_CUDA_TRY(launch_full_apply(h, false, VType::C64, u, VType::C64, y, nullptr, nrhs, st));
  } else {
    set_error("hps_full_apply: unknown dtype");
    return HPS_EINVAL;
  }
  return HPS_OK;
}

int hps_full_precond(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream) {
  if (!h || !r || !z || nrhs < 1 || r == z) {
    set_error("hps_full_precond: bad arguments");
    return HPS_EINVAL;
  }
  if (!h->fs.built) {
    set_error("hps_full_precond: the global-system path was not built (options.full_system)");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == HPS_C128) {
    if (!h->fs.Sinv64 || h->p > 14) {
      set_error("hps_full_precond: complex-double blocks not built (HPS_FORM_FP64, p <= 14)");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_full_precond(h, true, VType::C128, r, VType::C128, z, nrhs, st));
  } else if (dtype == HPS_C64) {
    if (!h->fs.Sinv32) {
      set_error("hps_full_precond: complex-float blocks not built (HPS_FORM_MIXED)");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_full_precond(h, false, VType::C64, r, VType::C64, z, nrhs, st));
  } else {
    set_error("hps_full_precond: unknown dtype");
    return HPS_EINVAL;
  }
  return HPS_OK;
}

int hps_full_solve(hps_handle* h, int form, const double* s, const double* t, int nrhs, double tol, double* u_out,
                   hps_solve_info* info, void* stream) {
  if (!h || !u_out || nrhs < 1 || !(tol > 0.0)) {
    set_error("hps_full_solve: bad arguments");
    return HPS_EINVAL;
  }
  const bool no_pc = (form & HPS_SOLVE_NO_PRECOND) != 0;
  const SolveFlags fl = solve_flags(form);
  form &= ~kSolveFlagBits;
  if (form != HPS_FORM_FP64 && form != HPS_FORM_MIXED) {
    set_error("hps_full_solve: form must be HPS_FORM_FP64 or HPS_FORM_MIXED");
    return HPS_EINVAL;
  }
  if (!h->fs.built) {
    set_error("hps_full_solve: the global-system path was not built (options.full_system)");
    return HPS_EINVAL;
  }
  if (nrhs > h->opt.max_rhs || h->p > 14 || (form == HPS_FORM_FP64 && !h->fs.Sinv64) ||
      (form == HPS_FORM_MIXED && !h->fs.Sinv32)) {
    set_error("hps_full_solve: nrhs > max_rhs, p > 14, or the form's blocks were not built");
    return HPS_EINVAL;
  }
  // device pointers only
  for (const void* ptr : {(const void*)s, (const void*)t, (const void*)u_out}) {
    if (!ptr) continue;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, ptr) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      set_error("hps_full_solve: s, t and u_out must be device pointers");
      return HPS_EINVAL;
    }
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  int rc = full_solve(h, form, !no_pc, (const double2*)s, (const double2*)t, nrhs, tol, (double2*)u_out, info, st, fl);
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

int hps_precond(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream) {
  if (!h || !r || !z || nrhs < 1) {
    set_error("hps_precond: bad arguments");
    return HPS_EINVAL;
  }
  if (nrhs > h->opt.max_rhs) {
    set_error("hps_precond: nrhs exceeds options.max_rhs");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  const size_t es = (dtype == HPS_C128) ? sizeof(double2) : sizeof(float2);
  if (dtype != HPS_C128 && dtype != HPS_C64 && dtype != HPS_C64_H16) {
    set_error("hps_precond: unknown dtype");
    return HPS_EINVAL;
  }
  if (!h->has_precond) {
    HPS_CUDA_TRY(cudaMemcpyAsync(z, r, (size_t)nrhs * h->nf * es, cudaMemcpyDeviceToDevice, st));
    return HPS_OK;
  }
  if (dtype == HPS_C128) {
    if (!h->Kc64) {
      set_error("hps_precond: FP64 preconditioner was not built (HPS_FORM_FP64)");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_precond(h, false, VType::C128, r, VType::C128, z, h->pc_scratch, nrhs, st));
  } else if (dtype == HPS_C64_H16) {
    if (!h->Kc16) {
      set_error("hps_precond: FP16 preconditioner blocks were not built (options.precond_fp16)");
      return HPS_EINVAL;
    }
    HPS_CUDA_TRY(launch_precond(h, true, VType::C64, r, VType::C64, z, h->pc_scratch, nrhs, st, true));
  } else {
    if (!h->Kc32 && !h->Kc16) {
      set_error("hps_precond: FP32 preconditioner was not built (HPS_FORM_MIXED)");
      return HPS_EINVAL;
    }
    // lean mode keeps the cluster inverses in FP16 only
    HPS_CUDA_TRY(launch_precond(h, true, VType::C64, r, VType::C64, z, h->pc_scratch, nrhs, st, !h->Kc32));
  }
  return HPS_OK;
}

int hps_rhs(hps_handle* h, const double* s, const double* t, int nrhs, double* b_out, void* stream) {
  if (!h || !b_out || nrhs < 1) {
    set_error("hps_rhs: bad arguments");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  HPS_CUDA_TRY(launch_rhs(h, (const double2*)s, (const double2*)t, (double2*)b_out, nrhs, (cudaStream_t)stream));
  return HPS_OK;
}

int hps_gmres_solve(hps_handle* h, int form, const double* s, const double* t, int nrhs, double tol, double* f_out,
                    hps_solve_info* info, void* stream) {
  if (!h || !f_out || nrhs < 1 || !(tol > 0.0)) {
    set_error("hps_gmres_solve: bad arguments");
    return HPS_EINVAL;
  }
  const bool no_pc = (form & HPS_SOLVE_NO_PRECOND) != 0;
  const SolveFlags fl = solve_flags(form);
  form &= ~kSolveFlagBits;
  if (form != HPS_FORM_FP64 && form != HPS_FORM_MIXED) {
    set_error("hps_gmres_solve: form must be HPS_FORM_FP64 or HPS_FORM_MIXED");
    return HPS_EINVAL;
  }
  if (nrhs > h->opt.max_rhs) {
    set_error("hps_gmres_solve: nrhs exceeds options.max_rhs");
    return HPS_EINVAL;
  }
  if (form == HPS_FORM_MIXED && (!h->R32 || (h->has_precond && !no_pc && !h->Kc32 && !h->Kc16))) {
    set_error("hps_gmres_solve: mixed-form operators were not built");
    return HPS_EINVAL;
  }
  if (form == HPS_FORM_FP64 && !h->R64) {
    set_error("hps_gmres_solve: the FP64 form needs the complex-double maps (not kept in lean mode)");
    return HPS_EINVAL;
  }
  if (form == HPS_FORM_FP64 && h->has_precond && !no_pc && !h->Kc64) {
    set_error("hps_gmres_solve: FP64 preconditioner was not built");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  cudaStream_t st = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  int rc = krylov_alloc(h, nrhs);
  if (rc) return rc;
  KrylovSpace& k = h->ks;
  const double2* sd = (const double2*)s;
  const double2* td = (const double2*)t;
  if (s && !is_device_ptr(s)) {
    if ((rc = check_finite(s, 2LL * nrhs * h->nint, "s"))) return rc;
    if (!k.s_dev && (rc = dalloc(h, (void**)&k.s_dev, (size_t)h->opt.max_rhs * h->nint * sizeof(double2)))) return rc;
    HPS_CUDA_TRY(cudaMemcpyAsync(k.s_dev, s, (size_t)nrhs * h->nint * sizeof(double2), cudaMemcpyHostToDevice, st));
    sd = k.s_dev;
  }
  if (t && !is_device_ptr(t)) {
    if ((rc = check_finite(t, 2LL * nrhs * h->nf, "t"))) return rc;
    if (!k.t_dev && (rc = dalloc(h, (void**)&k.t_dev, (size_t)h->opt.max_rhs * h->nf * sizeof(double2)))) return rc;
    HPS_CUDA_TRY(cudaMemcpyAsync(k.t_dev, t, (size_t)nrhs * h->nf * sizeof(double2), cudaMemcpyHostToDevice, st));
    td = k.t_dev;
  }
  // the compensated FP32 maps reproduce the FP64 ones to ~3e-11: the mixed form uses them for the
  // right-hand side and the restart residual when the tolerance is at least 1e-8
  const bool cf = form == HPS_FORM_MIXED && tol >= kCompensatedMinTol && h->R16lo && h->H16lo;
  {
    cudaEvent_t ev = h->prof.begin(st);
    HPS_CUDA_TRY(launch_rhs(h, sd, td, k.b, nrhs, st, cf || !h->H64));
    h->prof.end(HPS_PHASE_RHS, ev, st);
  }
  const bool fdev = is_device_ptr(f_out);
  double2* x = fdev ? (double2*)f_out : k.x;
  if (fl.x0 && !fdev) {
    if ((rc = check_finite(f_out, 2LL * nrhs * h->nf, "initial guess"))) return rc;
    HPS_CUDA_TRY(cudaMemcpyAsync(x, f_out, (size_t)nrhs * h->nf * sizeof(double2), cudaMemcpyHostToDevice, st));
  }
  rc = gmres_solve(h, form, k.b, x, nrhs, tol, info, st, !no_pc, fl);
  if (rc != HPS_OK && rc != HPS_ENOCONV) return rc;
  if (!fdev) {
    HPS_CUDA_TRY(cudaMemcpyAsync(f_out, x, (size_t)nrhs * h->nf * sizeof(double2), cudaMemcpyDeviceToHost, st));
  }
  HPS_CUDA_TRY(cudaStreamSynchronize(st));
  if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}

int hps_recover(hps_handle* h, const double* s, const double* f, int nrhs, double* u_out, double* u_face_out,
                void* stream) {
  if (!h || !f || !u_out || nrhs < 1 || nrhs > 1024) {
    set_error("hps_recover: bad arguments");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  return recover_interior(h, (const double2*)s, (const double2*)f, nrhs, (double2*)u_out, (double2*)u_face_out,
                          (cudaStream_t)stream);
}

int hps_precond_info(const hps_handle* h, int* clusters, int* k_blocks, int* b_blocks) {
  if (!h || !h->has_precond) {
    set_error("hps_precond_info: no preconditioner");
    return HPS_EINVAL;
  }
  if (clusters) *clusters = h->ct.ncl;
  if (k_blocks) *k_blocks = h->ct.nkc;
  if (b_blocks) *b_blocks = h->ct.nbc;
  return HPS_OK;
}

int hps_plan_blocks(const hps_grid* g, const double* lambda_q, int* leaf_b_block, int* cluster_k_block,
                    int* clusters, int* k_blocks, int* b_blocks) {
  if (validate_grid(g)) return HPS_EINVAL;
  if (!lambda_q) {
    set_error("hps_plan_blocks: lambda_q is NULL");
    return HPS_EINVAL;
  }
  hps_options o;
  hps_default_options(&o);
  hps_handle h;
  init_fields(&h, g, 1.0, 1.0, o);
  std::vector<double2> lamq(h.nl);
  for (int i = 0; i < h.nl; ++i) {
    const double re = lambda_q[2 * (size_t)i], im = lambda_q[2 * (size_t)i + 1];
    if (!std::isfinite(re) || !std::isfinite(im)) {
      set_error("hps_plan_blocks: non-finite constant");
      return HPS_EINVAL;
    }
    lamq[i] = make_double2(re, im);
  }
  build_cluster_tables(&h, 2);
  assign_blocks(&h, &lamq);
  const ClusterTables& ct = h.ct;
  if (leaf_b_block)
    for (int i = 0; i < h.nl; ++i) leaf_b_block[i] = ct.leaf_bcls[i];
  if (cluster_k_block)
    for (int c = 0; c < ct.ncl; ++c) cluster_k_block[c] = ct.cl_class[c];
  if (clusters) *clusters = ct.ncl;
  if (k_blocks) *k_blocks = ct.nkc;
  if (b_blocks) *b_blocks = ct.nbc;
  return HPS_OK;
}

int hps_axis_eig(int n, const double* M, double* V, double* Vinv, double* E) {
  if (n < 1 || n > 64 || !M || !V || !Vinv || !E) {
    set_error("hps_axis_eig: n must be in 1..64 and no pointer NULL");
    return HPS_EINVAL;
  }
  for (long long i = 0; i < (long long)n * n; ++i)
    if (!std::isfinite(M[i])) {
      set_error("hps_axis_eig: non-finite entry");
      return HPS_EINVAL;
    }
  if (!axis_eig(n, M, V, Vinv, E)) {
    set_error("hps_axis_eig: no real eigen-decomposition within its checks");
    return HPS_EBREAKDOWN;
  }
  return HPS_OK;
}

long long hps_export(hps_handle* h, int what, int index, double* host_out) {
  if (!h) {
    set_error("hps_export: NULL handle");
    return HPS_EINVAL;
  }
  if (cudaSetDevice(h->dev) != cudaSuccess) {
    set_error("hps_export: cudaSetDevice failed");
    return HPS_ECUDA;
  }
  cudaStreamSynchronize(h->stream);
  const int q2 = h->q * h->q;
  auto copy2d = [&](const void* src, size_t es, int rows, int cols, int ld, bool f32) -> long long {
    const long long count = 2LL * rows * cols;
    if (!host_out) return count;
    if (!f32) {
      if (cudaMemcpy2D(host_out, cols * sizeof(double2), src, (size_t)ld * es, cols * sizeof(double2), rows,
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("hps_export: copy failed");
        return HPS_ECUDA;
      }
    } else {
      std::vector<float2> tmp((size_t)rows * cols);
      if (cudaMemcpy2D(tmp.data(), cols * sizeof(float2), src, (size_t)ld * es, cols * sizeof(float2), rows,
                       cudaMemcpyDeviceToHost) != cudaSuccess) {
        set_error("hps_export: copy failed");
        return HPS_ECUDA;
      }
      for (size_t i = 0; i < tmp.size(); ++i) {
        host_out[2 * i] = tmp[i].x;
        host_out[2 * i + 1] = tmp[i].y;
      }
    }
    return count;
  };
  switch (what) {
    case HPS_EXPORT_R:
      if (index < 0 || index >= h->nl) break;
      if (!h->R64) return copy2d(h->R32 + (size_t)index * h->nb * h->ldR, sizeof(float2), h->nb, h->nb, h->ldR, true);
      return copy2d(h->R64 + (size_t)index * h->nb * h->ldR, sizeof(double2), h->nb, h->nb, h->ldR, false);
    case HPS_EXPORT_H:
      if (index < 0 || index >= h->nl) break;
      if (!h->H64) return copy2d(h->H32 + (size_t)index * h->nb * h->ldH, sizeof(float2), h->nb, h->ni, h->ldH, true);
      return copy2d(h->H64 + (size_t)index * h->nb * h->ldH, sizeof(double2), h->nb, h->ni, h->ldH, false);
    case HPS_EXPORT_LAMBDA:
      if (index < 0 || index >= h->nl || !h->has_precond) break;
      return copy2d(h->lambda + index, sizeof(double2), 1, 1, 1, false);
    case HPS_EXPORT_KC: {
      if (!h->has_precond || index < 0 || index >= h->ct.ncl) break;
      const int nint = (h->ct.cl_slot_begin[index + 1] - h->ct.cl_slot_begin[index]) * q2;
      const int ld = (int)rup4(nint);
      if (h->Kc64) return copy2d(h->Kc64 + h->ct.cl_kc_off[index], sizeof(double2), nint, nint, ld, false);
      return copy2d(h->Kc32 + h->ct.cl_kc_off[index], sizeof(float2), nint, nint, ld, true);
    }
    case HPS_EXPORT_B: {
      if (!h->has_precond || index < 0 || index >= h->nl) break;
      const int ni_ = __builtin_popcount(h->ct.int_mask[index]);
      const int rows = ni_ * q2, cols = (6 - ni_) * q2, ldr = (int)rup4(rows);
      if (rows == 0) return 0;
      // stored transposed (column c holds the rows): copy cols x rows, return rows x cols
      const long long count = 2LL * rows * cols;
      if (!host_out) return count;
      std::vector<double> tmp((size_t)count);
      double* keep = host_out;
      host_out = tmp.data();
      const long long rc2 = h->B64 ? copy2d(h->B64 + h->ct.b_off[index], sizeof(double2), cols, rows, ldr, false)
                                   : copy2d(h->B32 + h->ct.b_off[index], sizeof(float2), cols, rows, ldr, true);
      host_out = keep;
      if (rc2 < 0) return rc2;
      for (int r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) {
          host_out[2 * ((size_t)r * cols + c)] = tmp[2 * ((size_t)c * rows + r)];
          host_out[2 * ((size_t)r * cols + c) + 1] = tmp[2 * ((size_t)c * rows + r) + 1];
        }
      return count;
    }
    default:
      break;
  }
  set_error("hps_export: bad 'what' or index");
  return HPS_EINVAL;
}

int hps_import_map(hps_handle* h, int what, int index, const double* host_in) {
  if (!h || !host_in) {
    set_error("hps_import_map: NULL handle or input");
    return HPS_EINVAL;
  }
  if (what != HPS_EXPORT_R || index < 0 || index >= h->nl) {
    set_error("hps_import_map: only HPS_EXPORT_R with a leaf index in range is accepted");
    return HPS_EINVAL;
  }
  if (int rc = check_finite(host_in, 2LL * h->nb * h->nb, "R")) return rc;
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  HPS_CUDA_TRY(cudaStreamSynchronize(h->stream));
  const size_t rows = h->nb, cols = h->nb;
  if (h->R64) {
    HPS_CUDA_TRY(cudaMemcpy2D(h->R64 + (size_t)index * h->nb * h->ldR, (size_t)h->ldR * sizeof(double2), host_in,
                              cols * sizeof(double2), cols * sizeof(double2), rows, cudaMemcpyHostToDevice));
  }
  if (h->R32) {
    std::vector<float2> tmp(rows * cols);
    for (size_t i = 0; i < tmp.size(); ++i) tmp[i] = make_float2((float)host_in[2 * i], (float)host_in[2 * i + 1]);
    HPS_CUDA_TRY(cudaMemcpy2D(h->R32 + (size_t)index * h->nb * h->ldR, (size_t)h->ldR * sizeof(float2), tmp.data(),
                              cols * sizeof(float2), cols * sizeof(float2), rows, cudaMemcpyHostToDevice));
  }
  return HPS_OK;
}

int hps_test_inject(hps_handle* h, int what, long long spin_limit) {
  if (!h || (what != HPS_INJECT_NONE && what != HPS_INJECT_SKIP_ARRIVAL) || spin_limit < 0) {
    set_error("hps_test_inject: bad arguments");
    return HPS_EINVAL;
  }
  h->test_skip_arrival = (what == HPS_INJECT_SKIP_ARRIVAL) ? 1 : 0;
  h->test_spin = spin_limit;
  krylov_drop_graph(h);  // a captured cycle would keep the old launch parameters
  return HPS_OK;
}

int hps_get_launch_shapes(const hps_handle* h, hps_launch_shapes* out) {
  if (!h || !out) {
    set_error("hps_get_launch_shapes: bad arguments");
    return HPS_EINVAL;
  }
  for (int k = 0; k < 2; ++k)
    for (int g = 0; g < 4; ++g) {
      out->apply_rows_per_warp[k][g] = h->shapes.apply[k][g].rpw;
      out->apply_ctas_per_sm[k][g] = h->shapes.apply[k][g].bps;
    }
  for (int g = 0; g < 4; ++g) {
    out->stage_k_rows_per_warp[g] = h->shapes.k[g].rpw;
    out->stage_k_ctas_per_sm[g] = h->shapes.k[g].bps;
  }
  out->tuned = h->shapes.tuned ? 1 : 0;
  return HPS_OK;
}

int hps_profile_enable(hps_handle* h, int on) {
  if (!h) {
    set_error("hps_profile_enable: NULL handle");
    return HPS_EINVAL;
  }
  h->prof.on = on != 0;
  return HPS_OK;
}

int hps_profile_read(hps_handle* h, hps_profile* out, int reset) {
  if (!h || !out) {
    set_error("hps_profile_read: bad arguments");
    return HPS_EINVAL;
  }
  HPS_CUDA_TRY(cudaSetDevice(h->dev));
  h->prof.flush();
  out->launches = h->prof.launches;
  for (int i = 0; i < HPS_NPHASES; ++i) {
    out->ms[i] = h->prof.ms[i];
    out->count[i] = h->prof.count[i];
  }
  if (reset) h->prof.reset();
  return HPS_OK;
}

size_t hps_memory_bytes(const hps_handle* h) { return h ? h->bytes + h->ks.bytes : 0; }

int hps_destroy(hps_handle* h) {
  free_handle(h);
  return HPS_OK;
}

}  // extern "C"
