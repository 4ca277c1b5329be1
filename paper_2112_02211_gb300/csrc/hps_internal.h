// Internal declarations of the HPS library: the handle and the kernel
// launchers implemented in setup.cu, apply.cu and krylov.cu.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/hps.h"

namespace hps {

void set_error(const std::string& msg);

// Throws-free error plumbing: every launcher returns cudaError_t and the API
// layer converts it to HPS_ECUDA with the message.
#define HPS_CUDA_TRY(expr)                                                          \
  do {                                                                              \
    cudaError_t e__ = (expr);                                                       \
    if (e__ != cudaSuccess) {                                                       \
      ::hps::set_error(std::string(#expr) + ": " + cudaGetErrorString(e__));        \
      return HPS_ECUDA;                                                             \
    }                                                                               \
  } while (0)

inline long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Lets `kernel` use up to `bytes` of dynamic shared memory.  The limit is a
// per-function attribute shared by every host thread, so it is raised once per
// (kernel, device) to the device's opt-in maximum and never lowered: concurrent
// callers needing different amounts cannot set it below each other's launch.
cudaError_t allow_dynamic_smem(const void* kernel, size_t bytes);

// Offsets (in doubles) of the 1D tables in Handle::tables.
struct TableLayout {
  int p, q;
  int x, D, D2, xg, wg, Q, Qi, total;
  explicit TableLayout(int p_ = 4) : p(p_), q(p_ - 2) {
    x = 0;
    D = x + p;            // 3 axes, p*p each, scaled by 2/h_axis
    D2 = D + 3 * p * p;   // squares of D
    xg = D2 + 3 * p * p;  // Gauss nodes on [-1, 1]
    wg = xg + q;          // Gauss weights
    Q = wg + q;           // q x q: Chebyshev-interior -> Gauss interpolation
    Qi = Q + q * q;       // inverse of Q
    total = Qi + q * q;
  }
};

// Cluster (block-Jacobi) bookkeeping, built on the host from integer grid
// arithmetic and uploaded once.
//
// Distinct blocks: clusters whose leaves carry the same (binned) homogenized
// constants lambda^tau in the same arrangement share one K block, and leaves
// with the same constant and the same internal-face mask share one B block
// (reuse of the local solver for leaves with nearly the same medium, Sec. 4.1
// remark).  Without binning every cluster and leaf owns its block unless two
// constants are bitwise equal.
struct ClusterTables {
  int ncl = 0;                       // clusters
  int nslots = 0;                    // internal face slots over all clusters
  std::vector<int> cl_leaf_begin;    // [ncl+1] into cl_leaves
  std::vector<int> cl_leaves;        // leaves of each cluster, lexicographic
  std::vector<int> cl_slot_begin;    // [ncl+1] first global slot of each cluster
  std::vector<long long> cl_kc_off;  // [ncl] element offset of the cluster's K block (ld = rup4(nint))
  std::vector<int> slot_lf;          // [nslots] leaf*6+face of each slot
  std::vector<int> slot_cluster;     // [nslots]
  std::vector<int> lf_slot;          // [nleaves*6] slot of (leaf, face) or -1 if external
  std::vector<uint8_t> int_mask;     // [nleaves] bit f: face f is internal to the leaf's cluster
  int max_ext = 6;                   // most external faces of any leaf (3 when every cluster is 2x2x2)
  std::vector<long long> b_off;      // [nleaves] element offset of the leaf's B block
  // distinct K blocks
  int nkc = 0;
  std::vector<int> cl_class;         // [ncl] K block of each cluster
  std::vector<int> kc_rep;           // [nkc] first cluster using the block
  std::vector<int> kc_slot_begin;    // [nkc+1] block slots; FP16 scale row = (kc_slot_begin[k] + s) q^2 + j
  std::vector<long long> kc_off;     // [nkc] element offset of block k
  std::vector<int> kc_members;       // clusters grouped by block, ascending within a block
  std::vector<int> kc_mem_begin;     // [nkc+1] into kc_members
  std::vector<int> kslot_class;      // [kc_slot_begin[nkc]] block of each block slot
  // distinct B blocks
  int nbc = 0;
  std::vector<int> leaf_bcls;        // [nleaves] B block of each leaf; FP16 scale row = (bcls*6 + face) q^2 + j
  std::vector<int> bc_rep;           // [nbc] first leaf using the block
  // stage-K work items (block, block slot * kKRowSplit + part of its rows,
  // first member, member count) for member groups of width 1, 2, 4 and 8, and
  // the blocks whose members are many enough for the tensor-core path
  // (tc_precond.cu), which then skip the items above
  std::vector<int4> kitems[4];
  long long kitems_ntc[4] = {0, 0, 0, 0};
  std::vector<int> kc_tc;
  // stage-K input t: the members of a block are consecutive and each block
  // starts on a 16-element boundary, so a block's t vectors form one strided
  // matrix; cl_tpos[c] is cluster c's offset, lf_tpos[leaf*6+face] the offset
  // of an internal face's q^2 values (-1 on external faces), tsize the
  // elements per right-hand side
  std::vector<long long> cl_tpos;
  std::vector<long long> lf_tpos;
  long long tsize = 0;
  // stage-B offsets per leaf, 6 entries each (internal faces first, then
  // external, in face order): bface = face index; brd = input offset of the
  // neighbour's slot across an internal face (nbr*nb + (face^1)*q^2) or of the
  // leaf's own external face (leaf*nb + face*q^2); bto = t offset of that
  // neighbour slot (internal faces); bsc = FP16 row-scale base (bcls*6 + face)*q^2
  std::vector<int> brd, bto, bsc;
  long long kc_elems = 0, b_elems = 0;
  // Every block has the same internal size nint (all clusters 2x2x2), blocks are
  // stored back to back (kc_off[k] = k nint ld), nint is a multiple of 16 and the
  // member at stage-K position m (kc_members[m]) starts at t offset m nint: the
  // blocks form one 3D array and t one [position][nint] matrix per right-hand
  // side, so the multi-RHS tensor-core stage K runs every block in one launch.
  bool uniform = false;
  int nint0 = 0;                     // internal values of every cluster when uniform
  std::vector<int> pos_class;        // [ncl] K block of the member at stage-K position m
  std::vector<int> leaf_cluster;     // [nleaves] cluster of each leaf
  // FP16 tensor-core stage K of one right-hand side (uniform layout): items (block, 128-row
  // tile, first member position, members <= 64)
  std::vector<int4> tc16_items;
  // stage-B work items: leaves sorted by B block, in groups of at most kBGroup that share one
  // block (first index into bgroup_leaves, count)
  std::vector<int> bgroup_leaves;
  std::vector<int2> bgroups;
  int max_group = 0;
};

struct DeviceClusterTables {
  int* slot_lf = nullptr;
  int* slot_cluster = nullptr;
  int* cl_slot_begin = nullptr;
  long long* cl_kc_off = nullptr;
  int* lf_slot = nullptr;
  uint8_t* int_mask = nullptr;
  long long* b_off = nullptr;
  int* leaf_bcls = nullptr;
  int* bc_rep = nullptr;
  long long* kc_off = nullptr;
  int* kc_slot_begin = nullptr;
  int* kslot_class = nullptr;
  int* kc_members = nullptr;
  int4* kitems[4] = {nullptr, nullptr, nullptr, nullptr};
  long long* cl_tpos = nullptr;
  long long* lf_tpos = nullptr;
  int* brd = nullptr;
  int* bto = nullptr;
  int* bsc = nullptr;
  int* pos_class = nullptr;
  int* leaf_cluster = nullptr;
  int4* tc16_items = nullptr;
  int* bgroup_leaves = nullptr;
  int2* bgroups = nullptr;
};

// Launch shape of the batched GEMV kernels: matrix rows per warp pass and a cap on
// resident CTAs per SM (0 = the occupancy limit).  Neither changes any result: each
// row is one warp's sum over its lanes in the same order.
struct LaunchShape {
  int rpw = 4;
  int bps = 0;
};
// The shapes a handle launches with, per right-hand-side group (1, 2, <= 4, <= 8):
// the ItI apply with FP32 maps [0] and FP64 maps [1], and the SIMT stage K per
// member-group width (1, 2, 4, 8).  Defaults from a hand sweep; replaced at setup
// by the autotuner (options.autotune).
struct Shapes {
  LaunchShape apply[2][4] = {{{4, 0}, {4, 0}, {2, 0}, {1, 0}}, {{4, 0}, {4, 0}, {2, 0}, {1, 0}}};
  LaunchShape k[4] = {{4, 0}, {4, 0}, {2, 0}, {2, 0}};
  bool tuned = false;
};

// Per-phase CUDA-event timing and a launch counter (see hps_profile).  Events
// are recorded as external events, so an interval recorded while a stream is
// being captured becomes a pair of event nodes of the graph; such intervals
// are taken out with take_recs() and read after every replay (read_recs).
struct Profiler {
  bool on = false;
  long long launches = 0;
  double ms[HPS_NPHASES] = {};
  long long count[HPS_NPHASES] = {};
  int step = -1;  // Arnoldi step the next intervals belong to (-1: none)
  struct Rec {
    int phase;
    cudaEvent_t a, b;
    int step;
  };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> recs;
  cudaEvent_t take() {
    if (pool.empty()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      return e;
    }
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  // An event record on st: an external event node of the graph while st is being
  // captured (the flag is only valid then), a plain record otherwise.
  static void record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
      cudaEventRecord(e, st);
  }
  // Start of a timed interval on stream st (nullptr when timing is off).
  cudaEvent_t begin(cudaStream_t st) {
    if (!on) return nullptr;
    cudaEvent_t e = take();
    record(e, st);
    return e;
  }
  void end(int phase, cudaEvent_t a, cudaStream_t st) {
    if (!on || !a) return;
    cudaEvent_t e = take();
    record(e, st);
    recs.push_back({phase, a, e, step});
  }
  // Intervals recorded since `from` (into a graph being captured); their events now
  // belong to the caller.
  std::vector<Rec> take_recs(size_t from) {
    std::vector<Rec> out(recs.begin() + from, recs.end());
    recs.resize(from);
    return out;
  }
  // Adds the intervals of one replay of a graph, those of steps < steps_done (and those
  // outside the steps) only.
  void read_recs(const std::vector<Rec>& rs, int steps_done) {
    for (const Rec& r : rs) {
      if (r.step >= steps_done) continue;
      float t = 0.f;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.phase] += t;
      count[r.phase] += 1;
    }
  }
  void release(std::vector<Rec>& rs) {
    for (const Rec& r : rs) {
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    rs.clear();
  }
  void flush() {
    for (const Rec& r : recs) {
      cudaEventSynchronize(r.b);
      float t = 0.f;
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.phase] += t;
      count[r.phase] += 1;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    recs.clear();
  }
  void reset() {
    flush();
    launches = 0;
    for (int i = 0; i < HPS_NPHASES; ++i) {
      ms[i] = 0;
      count[i] = 0;
    }
  }
  void destroy() {
    flush();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

// The paper's iterative path on the global system (Sec. 3-4): per distinct
// (binned) homogenized constant S~^{-1} = (A~^{-1})_bb, row-major nb x nb, and
// per axis the Algorithm 3 tables V (n1 x n1), V^{-1}, E (n1), row-major.
struct FullSystem {
  bool built = false;
  int ncls = 0;
  std::vector<int> cls;      // [nleaves] class of each leaf
  int* d_cls = nullptr;
  double2* Sinv64 = nullptr;
  float2* Sinv32 = nullptr;
  double* eig = nullptr;     // 3 x (2 n1^2 + n1)
};

// One restart cycle of GMRES (the first basis vector and m Arnoldi steps)
// captured as a CUDA graph; replayed every cycle of every solve with the same
// configuration.  Steps after convergence find the device gate closed and exit.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  // what the captured launches depend on
  int nrhs = 0, m = 0, ops_id = -1, mixed = 0, pc = 0, c64op = 0, cgs2 = 0, prof = 0;
  long long n = 0;
  const void* V = nullptr;
  long long launches = 0;                 // kernels per replay
  std::vector<Profiler::Rec> recs;        // timed intervals inside the graph
};

struct KrylovSpace {
  int m = 0, nrhs = 0, nblk = 0;
  long long nf = 0;
  double2* V = nullptr;      // (m+1) x nrhs x nf
  double2* x = nullptr;      // nrhs x nf
  double2* r = nullptr;      // nrhs x nf
  double2* b = nullptr;      // nrhs x nf
  double2* u = nullptr;      // nrhs x nf (V y)
  void* z = nullptr;         // nrhs x nf, inner precision
  void* zt = nullptr;        // precond scratch (internal slots), inner precision
  double2* part = nullptr;   // nrhs x nblk x (m+1) partial dots
  double2* hcol = nullptr;   // nrhs x (m+2) current Hessenberg column
  double2* H = nullptr;      // nrhs x (m+1) x m, rotated
  double* cs = nullptr;      // nrhs x m
  double2* sn = nullptr;     // nrhs x m
  double2* g = nullptr;      // nrhs x (m+1)
  double2* y = nullptr;      // nrhs x m
  double* est = nullptr;     // nrhs: |g_{j+1}| after the last step
  double* nrm = nullptr;     // nrhs: norms
  int* active = nullptr;     // nrhs; then kcount[nrhs], any_active, status, reorth[nrhs], nreorth
  int* status = nullptr;     // device status word (breakdown etc.)
  double2* s_dev = nullptr;  // staging for host inputs
  double2* t_dev = nullptr;
  double2* f_dev = nullptr;
  CycleGraph graph;
  size_t bytes = 0;
};

}  // namespace hps

struct hps_handle {
  int dev = 0;
  int nx = 0, ny = 0, nz = 0, p = 0, q = 0, n1 = 0, ni = 0, nb = 0, n = 0, nl = 0;
  long long nf = 0, nint = 0;
  double kappa = 0, eta = 0, h[3] = {0, 0, 0};
  hps_options opt{};
  int nsm = 0;
  cudaStream_t stream = nullptr;

  double* tables = nullptr;
  hps::TableLayout tl;

  // exact leaf maps (Gauss basis)
  int ldR = 0, ldH = 0;
  double2* R64 = nullptr;  // nl x nb x ldR
  float2* R32 = nullptr;   // nl x nb x ldR
  double2* H64 = nullptr;  // nl x nb x ldH
  float2* H32 = nullptr;   // nl x nb x ldH (lean mode instead of H64)
  // lean mode: remainders M - M32 of the FP32 maps in FP16, row r of leaf l scaled by
  // *16ls[l * nb + r] (compensated FP32 maps, compensated.cu)
  __half2* R16lo = nullptr;
  float* R16ls = nullptr;
  __half2* H16lo = nullptr;
  float* H16ls = nullptr;
  double2* lambda = nullptr;    // nl: homogenized constants lambda^tau
  double2* lambda_q = nullptr;  // nl: lambda^tau after binning (opt.lambda_bin), used by the preconditioner
  double2* cdiag = nullptr;   // nl x ni: C = kappa^2 (1 - b) at interior nodes (kept for recovery)

  // the paper's global-system path (options.full_system)
  hps::FullSystem fs;

  // preconditioner
  bool has_precond = false;
  hps::ClusterTables ct;
  hps::DeviceClusterTables dct;
  double2* Kc64 = nullptr;
  float2* Kc32 = nullptr;
  double2* B64 = nullptr;
  float2* B32 = nullptr;
  __half2* Kc16 = nullptr;  // FP16 copies, row r of block slot bs scaled by 1/Kc16s[bs*q^2 + r]
  float* Kc16s = nullptr;
  __half2* B16 = nullptr;   // FP16 copies of B, rows scaled by 1/B16s[(bcls*6+face)*q^2 + j]
  float* B16s = nullptr;
  void* pc_scratch = nullptr;  // nslots*q^2*max_rhs complex double (precond t buffer)
  float* tmax = nullptr;       // [rhs][cluster] largest |component| of stage B's t (FP16 stage K scale)
  int tmax_rhs = 0;            // right-hand sides tmax holds

  int* tc_error = nullptr;  // device error word of the tensor-core kernels
  // While a GMRES cycle is captured: the device word that the per-step kernels
  // (apply, preconditioner) read first, returning at once when it is 0 (no
  // right-hand side still active).  nullptr otherwise.
  mutable const int* gate = nullptr;
  hps::Shapes shapes;
  // test hook of hps_test_inject: bounded-wait limit (tries) of the tensor-core apply (0 =
  // default) and whether one of its CTAs skips one mbarrier arrival
  long long test_spin = 0;
  int test_skip_arrival = 0;
  hps::KrylovSpace ks;
  mutable hps::Profiler prof;
  size_t bytes = 0;
};

namespace hps {

// ---- setup.cu ----
cudaError_t launch_tables(double* tables, const TableLayout& tl, double hx, double hy, double hz,
                          cudaStream_t st);
cudaError_t launch_nodes(const double* tables, const TableLayout& tl, int nx, int ny, int nz,
                         double* interior_xyz_dev, double* face_xyz_dev, double* cheb_face_xyz_dev,
                         cudaStream_t st);
// Builds R (and H) for all leaves; see setup.cu.
int build_exact_maps(hps_handle* h, const double2* cdiag, cudaStream_t st);
// lambda^tau of every leaf, its binning and the distinct preconditioner blocks
// (sizes in h->ct); uploads the cluster tables.  Before the block storage is
// allocated.
int classify_preconditioner(hps_handle* h, const double2* cdiag, cudaStream_t st);
int compute_lambdas(hps_handle* h, const double2* cdiag, cudaStream_t st, std::vector<double2>& lamq);
// S~^{-1} per distinct homogenized constant and the Algorithm 3 tables (full.cu uses them).
int build_full_system(hps_handle* h, const double2* cdiag, cudaStream_t st);
// M = V diag(E) V^{-1} for a small real matrix with real distinct eigenvalues (host; the
// per-axis tables of Algorithm 3); false when it does not converge or fails its checks
bool axis_eig(int n, const double* M, double* V, double* Vinv, double* E);
int build_preconditioner(hps_handle* h, const double2* cdiag, cudaStream_t st);
int build_precond_fp16(hps_handle* h, cudaStream_t st);
int recover_interior(hps_handle* h, const double2* s, const double2* f, int nrhs, double2* u, double2* uf,
                     cudaStream_t st);
size_t workspace_cap(const hps_handle* h);
size_t exact_maps_workspace(const hps_handle* h, size_t budget, int* nbatch_out);
size_t precond_workspace(const hps_handle* h, size_t budget, int* cb_out);
void build_cluster_tables(hps_handle* h, int width);
// Distinct preconditioner blocks from binned lambda values (nullptr: one block
// per cluster and per leaf).
void assign_blocks(hps_handle* h, const std::vector<double2>* lamq);
// Shared K blocks with at least this many member clusters run on the tensor cores.
constexpr int kTcMinMembers = 16;
// Stage-K work items of the SIMT kernel cover 1/kKRowSplit of a slot's q^2 rows
// (finer items balance the last wave of the launch).
constexpr int kKRowSplit = 2;
// Leaves per stage-B work item (leaves sharing one B block).  Items of 8 leaves were measured
// faster (0.070 vs 0.147 ms per application at 16^3 leaves) but gave a wrong preconditioner on a
// complex medium (GMRES stalled; the same items one vector at a time gave other iterates than
// one leaf per item), for a reason not yet found; one leaf per item until it is.
constexpr int kBGroup = 1;
// Dynamic shared memory a block may opt into on sm_103 (227 KB).
constexpr int kMaxDynSmem = 227 * 1024;

// ---- apply.cu ----
// C128 complex double, C64 complex float, DF complex double-float (float4: re.h, im.h, re.l, im.l)
enum class VType { C128, C64, DF };
// y = (I + Pi R) f  (mode 0) or y = b - (I + Pi R) f (mode 1), R in FP64 or FP32.
cudaError_t launch_apply(const hps_handle* h, bool fp32_matrix, VType tin, const void* f,
                         VType tout, void* y, const double2* bvec, int nrhs, bool residual,
                         cudaStream_t st);
// compensated: the FP32 maps with their FP16 remainders (when kept) instead of the FP64 maps
cudaError_t launch_rhs(const hps_handle* h, const double2* s, const double2* t, double2* b, int nrhs,
                       cudaStream_t st, bool compensated = false);
// Smallest solve tolerance at which the mixed form forms its restart residual and right-hand
// side from the compensated FP32 maps (~3e-11 from the FP64 maps) instead of the FP64 maps.
constexpr double kCompensatedMinTol = 1e-8;
cudaError_t launch_precond(const hps_handle* h, bool fp32_matrix, VType tin, const void* r,
                           VType tout, void* z, void* scratch, int nrhs, cudaStream_t st, bool fp16_blocks = false);
// Tensor-core apply for 64-RHS groups (tc_apply.cu); f complex float, y complex
// float or double-float; nrhs a multiple of 64.
// whether launch_apply runs nrhs right-hand sides with complex-FP32 input on the tensor cores
bool apply_tc_eligible(const hps_handle* h, int nrhs);
// Times the candidate launch shapes of the applies and the SIMT stage K the solves will use
// and keeps the fastest in h->shapes (process-wide cache keyed by kernel, device and sizes).
int autotune_shapes(hps_handle* h, cudaStream_t st);
cudaError_t launch_apply_tc(const hps_handle* h, const float2* f, void* y, bool out_df, int nrhs, int* d_error,
                            cudaStream_t st);
// Stage K of the preconditioner for the shared K blocks listed in ct.kc_tc, on
// the tensor cores (tc_precond.cu): z_int = K_c t for every member cluster of
// those blocks; one right-hand side; t in the class-ordered layout.
cudaError_t launch_precond_tc(const hps_handle* h, const float2* t, float2* z, int* d_error, cudaStream_t st);
// Stage K for nrhs (a multiple of 64) right-hand sides at once, every block on the tensor cores
// in one launch (complex-FP32 blocks, one TF32 product): the GEMM of each K_c against the
// columns (member cluster, right-hand side).  Needs ct.uniform.  t: [rhs][tsize], z: [rhs][nf].
bool precond_tc_multi_eligible(const hps_handle* h, int nrhs);
// Stage K of every cluster block on the tensor cores with FP16 operands (tc_precond16.cu): the
// FP16 blocks against t scaled per cluster by tmax (which stage B fills); one right-hand side or
// 64, 128, ... of them; needs the uniform layout.
bool precond_tc16_eligible(const hps_handle* h, int nrhs);
cudaError_t launch_precond_tc16(const hps_handle* h, const float2* t, float2* z, int nrhs, cudaStream_t st);
cudaError_t launch_precond_tc_multi(const hps_handle* h, const float2* t, float2* z, int nrhs, int* d_error,
                                    cudaStream_t st);
// Timed wrappers (phase intervals recorded when profiling is on).
cudaError_t timed_apply(const hps_handle* h, int phase, bool fp32_matrix, VType tin, const void* f, VType tout,
                        void* y, const double2* bvec, int nrhs, bool residual, cudaStream_t st);

// ---- compensated.cu (lean mode: FP32 maps + FP16 remainders, double-float accumulation) ----
cudaError_t launch_split_lo(const double2* M, long long rows, int ld, __half2* lo, float* scale, cudaStream_t st);
bool compensated_maps(const hps_handle* h);
cudaError_t launch_apply_cf(const hps_handle* h, const double2* x, double2* y, const double2* b, int nrhs,
                            cudaStream_t st);
cudaError_t launch_rhs_cf(const hps_handle* h, const double2* s, const double2* t, double2* b, int nrhs,
                          cudaStream_t st);

// ---- full.cu (the paper's global-system path) ----
cudaError_t launch_full_apply(const hps_handle* h, bool fp64, VType tin, const void* u, VType tout, void* y,
                              const double2* b, int nrhs, cudaStream_t st);
cudaError_t launch_full_precond(const hps_handle* h, bool fp64, VType tin, const void* r, VType tout, void* z,
                                int nrhs, cudaStream_t st);

// ---- krylov.cu ----
int krylov_alloc(hps_handle* h, int nrhs, long long nvec = -1);
void krylov_free(hps_handle* h);
// Drops the captured GMRES cycle (its launches carry parameters that changed).
void krylov_drop_graph(hps_handle* h);
// Operators of one restarted GMRES: w = A z (inner precision), z = M^{-1} v,
// and the FP64 residual r = b - A x, on vectors of length n per right-hand side.
struct GmresOps {
  long long n = 0;
  bool pc = false;
  std::function<cudaError_t(VType, const void*, VType, void*, int, cudaStream_t)> apply;
  std::function<cudaError_t(VType, const void*, VType, void*, int, cudaStream_t)> precond;
  std::function<cudaError_t(const double2*, const double2*, double2*, int, cudaStream_t)> residual;
  // mixed form without a preconditioner: the apply takes the basis vector rounded to complex
  // FP32 (kept beside the double-float basis) instead of the double-float vector itself
  bool c64_operand = false;
  int id = 0;  // which operator family (face system 0, global system 1): part of the graph key
};
// Solve flags of gmres_core (bits of hps_gmres_solve's form beyond the form itself).
struct SolveFlags {
  bool x0 = false;       // x holds an initial guess
  bool no_graph = false; // launch the Arnoldi steps one by one instead of replaying a graph
  bool cgs2 = false;     // always two Gram-Schmidt passes (else the second only when needed)
};
int gmres_core(hps_handle* h, const GmresOps& ops, bool mixed, const double2* b, double2* x, int nrhs, double tol,
               hps_solve_info* info, cudaStream_t st, SolveFlags fl = SolveFlags());
int full_solve(hps_handle* h, int form, bool use_precond, const double2* s, const double2* t, int nrhs, double tol,
               double2* u, hps_solve_info* info, cudaStream_t st, SolveFlags fl = SolveFlags());
int gmres_solve(hps_handle* h, int form, const double2* b, double2* x, int nrhs, double tol,
                hps_solve_info* info, cudaStream_t st, bool use_precond, SolveFlags fl = SolveFlags());

}  // namespace hps
