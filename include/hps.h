/*
 * hps.h -- C ABI of the GB300 (sm_103a) library for the iterative HPS
 * Helmholtz solver of arXiv:2112.02211.
 *
 * Problem (1.1) of the paper, on the unit cube (0,1)^3:
 *
 *     -Lap u - kappa^2 (1 - b(x)) u = s(x)   in (0,1)^3,
 *     du/dn + i eta u              = t(x)   on the boundary,      Re(eta) != 0.
 *
 * The cube is split into nx x ny x nz equal leaf boxes (Sec. 2).  Each leaf
 * carries the modified Chebyshev collocation grid of order p (Sec. 2.1) and
 * q x q Gauss-Legendre points on each of its six faces, q = p - 2.  The
 * library solves the face form of the HPS system: the unknowns are the
 * incoming impedance data f = du/dn + i eta u on every leaf face (Definition
 * in Sec. 2.2), and
 *
 *     (I + Pi R) f = tbar - Pi h                                        (*)
 *
 * where R = blockdiag(R^tau) holds the leaf impedance-to-impedance (ItI)
 * maps, h^tau the leaf's outgoing response to the body load s, and Pi the
 * swap of outgoing data across shared faces (the interface condition
 * f^alpha = -g^beta, eq. (inter)); tbar is t on boundary faces, 0 elsewhere.
 * (*) is the exact reduction of the paper's global system (Sec. 3.1) onto
 * face data.  It is solved by restarted GMRES, right-preconditioned by a
 * block-Jacobi preconditioner over 2x2x2 leaf clusters built from locally
 * homogenized leaf maps (Sec. 4, Sec. 4.1).
 *
 * Layouts (all complex numbers are interleaved (re, im) pairs):
 *   leaf tau = ix + nx*(iy + ny*iz)                       (Fig. 4(a))
 *   face k in 0..5 = -x, +x, -y, +y, -z, +z               (Fig. 2, eq. (flux))
 *   face vector  [rhs][leaf][face][j2][j1], j1 fastest; in-face axes:
 *                +-x faces -> (y, z), +-y -> (x, z), +-z -> (x, y).
 *                N_f = nx*ny*nz*6*q*q complex values per right-hand side.
 *   interior     [rhs][leaf][k][j][i], i (x) fastest, n1 = p - 2 points per
 *                axis, i.e. nx*ny*nz*n1^3 values per right-hand side, at the
 *                interior Chebyshev nodes returned by hps_nodes.
 *
 * Errors: every entry point returns HPS_OK (0) or a negative HPS_E* code and
 * never throws; hps_last_error() gives a message for the calling thread.
 * Ownership: the handle owns all device state it allocates (leaf maps,
 * preconditioner blocks, Krylov workspace).  Callers own every buffer they
 * pass in.  A handle is used by one host thread at a time.
 */
#ifndef HPS_H
#define HPS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HPS_OK 0
#define HPS_EINVAL (-1)      /* bad argument: sizes, q != p-2, Re(eta) == 0, NaN/Inf input */
#define HPS_ENOMEM (-2)      /* device allocation failed or over the HBM budget */
#define HPS_ECUDA (-3)       /* a CUDA call failed (message in hps_last_error) */
#define HPS_ENOCONV (-4)     /* GMRES hit maxit; the best iterate and info are still written */
#define HPS_EBREAKDOWN (-5)  /* singular pivot or non-finite value in a kernel */
#define HPS_ETIMEOUT (-6)    /* a bounded device wait gave up */

/* Element types of device vectors passed to hps_apply / hps_precond. */
#define HPS_C128 0 /* complex double, 16 bytes */
#define HPS_C64 1  /* complex float, 8 bytes */
/* hps_precond only: complex float vectors, preconditioner blocks read from their
 * FP16 copies (one FP32 scale per row), as the mixed-form solve does. */
#define HPS_C64_H16 2

/* Solve forms (bit flags for hps_options.forms). */
#define HPS_FORM_FP64 1  /* everything in complex FP64 */
#define HPS_FORM_MIXED 2 /* complex-FP32 apply/preconditioner inside FP64 Krylov + FP64 outer residual */
/* Flags OR'd into the form argument of hps_gmres_solve and hps_full_solve: */
/* run GMRES without the preconditioner even when it was built (the solution is the same) */
#define HPS_SOLVE_NO_PRECOND 16
/* the output buffer holds an initial guess on entry (resume from a stored iterate): the
 * first residual is b - A x0 instead of b */
#define HPS_SOLVE_X0 32
/* launch each Arnoldi step's kernels from the host, with one synchronization per step,
 * instead of replaying the captured restart cycle (same arithmetic, same result bit for bit) */
#define HPS_SOLVE_NO_GRAPH 64
/* classical Gram-Schmidt twice at every step, instead of the second pass only where the
 * first cancelled most of the vector */
#define HPS_SOLVE_CGS2 128

typedef struct hps_handle hps_handle;

/* Leaves per axis and Chebyshev order; q must equal p - 2, 4 <= p <= 16. */
typedef struct {
  int nx, ny, nz;
  int p;
  int q;
} hps_grid;

typedef struct {
  int forms;          /* HPS_FORM_* flags: which operator precisions hps_setup builds */
  int restart;        /* GMRES restart length m (default 50) */
  int cluster;        /* block-Jacobi cluster width in leaves per axis: 2 (default) or 0 = none */
  int maxit;          /* maximum inner iterations per solve (default 5000) */
  int max_rhs;        /* maximum right-hand sides per solve (default 1) */
  size_t hbm_budget;  /* bytes the handle may allocate; 0 = no limit */
  int device;         /* CUDA device ordinal */
  int precond_fp16;   /* mixed form: also keep the preconditioner blocks in FP16 with one FP32
                         scale per row and use them in hps_gmres_solve (default 1) */
  int tc_apply;       /* tensor cores (three TF32 products, FP32 accumulation) for the
                         complex-FP32 apply of 64, 128, ... right-hand sides (inside an
                         unpreconditioned mixed solve the Krylov vectors are also kept rounded
                         to complex FP32 for it) and, with one TF32 product, for
                         preconditioner blocks shared by >= 16 clusters (complex-FP32
                         blocks; see lambda_bin); default 1 */
  int lean;           /* memory-lean mixed form (forms must be HPS_FORM_MIXED): the exact leaf
                         maps R, H are eliminated in FP64 but kept only in FP32, the cluster
                         inverses only in FP16 (plus complex-FP32 copies of blocks shared by
                         >= 16 clusters when they take <= 4 GiB, for the tensor-core path),
                         and the restart residual uses the FP32 maps with
                         FP64 vectors (about 1e-7 relative per apply, for tolerances >= 1e-5).
                         HPS_C128 applies are then unavailable.  Default 0. */
  double lambda_bin;  /* shared preconditioner blocks (Sec. 4.1 remark: one local solver for
                         leaves with nearly the same medium): each lambda^tau is rounded to the
                         nearest multiple of lambda_bin * max_tau |lambda^tau| (real and imaginary
                         parts separately, ties to even) before R~ and K_c are built, and clusters
                         whose leaves carry equal values in the same arrangement share one K_c
                         (leaves: one B block).  0 (default) keeps every lambda^tau; blocks are
                         still shared where values are bitwise equal.  Finite, >= 0.  Changes the
                         preconditioner only, never the converged solution. */
  int autotune;       /* time the candidate launch shapes (rows per warp, resident CTAs per SM)
                         of the ItI apply and of the preconditioner's stage K at setup and keep
                         the fastest (hps_launch_shapes); shapes never change results.
                         Default 1. */
  int full_system;    /* also build the paper's own iterative path on the global system
                         (Sec. 3-4; hps_full_apply, hps_full_precond, hps_full_solve): per
                         distinct homogenized constant the inverse Schur complement S~^{-1}, and
                         the Algorithm 3 eigen-tables.  Default 0. */
} hps_options;

typedef struct {
  int iterations;      /* inner GMRES iterations (max over right-hand sides) */
  int cycles;          /* restart cycles, each ending with an FP64 true residual */
  int converged;       /* 1 when every right-hand side met the tolerance */
  double rel_residual; /* max over RHS of ||b - A f||_2 / ||b||_2, FP64 operator */
  double seconds;      /* wall time of the solve (RHS build + GMRES), host clock */
  int reorth_steps;    /* Arnoldi steps (summed over right-hand sides) that took the second
                          Gram-Schmidt pass */
} hps_solve_info;

/* Fills *opt with the defaults listed above (forms = HPS_FORM_FP64|HPS_FORM_MIXED). */
void hps_default_options(hps_options* opt);

/*
 * Node coordinates of a grid, computed on the device (Sec. 2.1).
 * interior_xyz:   host, nx*ny*nz*n1^3*3 doubles (x,y,z per node, layout above),
 * face_xyz:       host, N_f*3 doubles, the Gauss points of every leaf face,
 * cheb_face_xyz:  host, N_f*3 doubles, the leaf's Chebyshev face nodes (the
 *                 n1 x n1 interior points of each face, face layout above
 *                 with j1/j2 indexing Chebyshev points) where hps_recover
 *                 returns face values.
 * Any pointer may be NULL.  Uses the current CUDA device.
 */
int hps_nodes(const hps_grid* grid, double* interior_xyz, double* face_xyz, double* cheb_face_xyz);

/*
 * Builds the leaf ItI maps R^tau (Gauss basis), the body-load maps H^tau and
 * the preconditioner for one medium.  Per leaf this assembles the leaf system
 * of eq. (leaf) and eliminates it with partial pivoting in FP64 on the
 * device: R_C = I - 2 i eta (A^{-1})_bb, H_C = -2 i eta (A^{-1})_bi, then
 * R = P R_C P^{-1}, H = P H_C with P the Chebyshev-to-Gauss face
 * interpolation.  The preconditioner uses the same construction with
 * C = kappa^2 (1 - b) replaced by lambda^tau = (max + min)/2 of C over the
 * leaf's interior nodes (Sec. 4.1, real and imaginary parts separately).
 *
 * b: host, nx*ny*nz*n1^3 complex (interleaved doubles), b at the interior
 *    nodes of hps_nodes.  kappa real, eta complex given as (eta, 0): the
 *    imaginary part of eta is 0 in this interface.  opt may be NULL.
 * On success *out owns all device state; free it with hps_destroy.
 */
int hps_setup(const hps_grid* grid, double kappa, double eta, const double* b,
              const hps_options* opt, hps_handle** out);

/*
 * Device bytes that hps_setup with these options would hold, plus the Krylov
 * workspace of one hps_gmres_solve with nrhs right-hand sides given as host
 * buffers, plus the largest transient setup workspace (taken at most
 * min(opt->hbm_budget, 24 GiB) when a budget is set).  For admission control
 * by an HBM budget.  Returns 0 for an invalid grid or options.  No device work.
 */
size_t hps_setup_bytes(const hps_grid* grid, const hps_options* opt, int nrhs);

/*
 * y = (I + Pi R) f for nrhs right-hand sides (the operator of (*); Sec. 2.2,
 * Sec. 3.1).  f, y: device, nrhs*N_f complex of the given dtype (HPS_C128
 * needs HPS_FORM_FP64 operators, HPS_C64 needs HPS_FORM_MIXED ones), must not
 * overlap.  stream: a cudaStream_t (NULL = legacy default stream).  The call
 * is asynchronous with respect to the host.
 */
int hps_apply(hps_handle* h, int dtype, const void* f, void* y, int nrhs, void* stream);

/*
 * z = J^{-1} r, the cluster block-Jacobi preconditioner (Sec. 4, Algorithm 4
 * in face form): on each cluster c of 2x2x2 leaves, z_c = (I + Pi_c R~)^{-1} r_c
 * where R~ are the homogenized leaf maps and Pi_c swaps only across faces
 * inside the cluster.  Same argument rules as hps_apply.  Uses a scratch
 * buffer owned by the handle, so calls on one handle must not overlap.
 */
int hps_precond(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream);

/*
 * The same preconditioner apply as hps_precond, for callers that must not
 * have the library allocate device memory during the call: processes that
 * hand the GPU's memory to their own pool at start-up, or that run inside a
 * fixed budget they do not control, where a cudaMalloc from a library could
 * fail, fragment the pool or stall the device.  (The paper has no
 * counterpart; this is an interface convenience.)  The scratch for the
 * cluster-internal right-hand sides lives in a static device array of
 * HPS_PRECOND_NOALLOC_MAX_BYTES bytes compiled into the library, held on
 * every device that loads it until the process exits.  A call needs
 * (internal face slots) * q^2 * nrhs * sizeof(element) bytes of it (for the
 * 16^3-leaf, p = 10 grid: 12.6 MB per complex-double right-hand side) and
 * returns HPS_EINVAL with a message when that exceeds the array.  nrhs is not
 * limited by options.max_rhs (the handle's scratch is not used), only by the
 * array.  Every call looks up the array's device address on the current device
 * (a host-side symbol lookup that allocates nothing); the first call on a
 * device may load the library's device code, so make it before any stream
 * capture begins.  The array keeps whatever the last call left in it; nothing
 * in it needs to start at zero, because every call overwrites the part it
 * reads.  All calls share the one array: calls that may overlap on the GPU
 * (other streams, other handles, other host threads) race on it and must be
 * serialized by the caller.  dtype: HPS_C128, HPS_C64 or HPS_C64_H16 with the
 * same operator choices as hps_precond (HPS_C64 reads the FP16 copies when the
 * handle keeps the cluster inverses in FP16 only).  Allocates no device memory.
 */
#define HPS_PRECOND_NOALLOC_MAX_BYTES ((size_t)16 << 20)
int hps_precond_noalloc(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream);

/*
 * Right-hand side of (*): b = tbar - Pi h with h^tau = H^tau s^tau.
 * s: nrhs interior vectors or NULL (s = 0); t: nrhs face vectors or NULL
 * (t = 0; only boundary-face entries are read).  s, t, b_out: device,
 * complex double.
 */
int hps_rhs(hps_handle* h, const double* s, const double* t, int nrhs, double* b_out,
            void* stream);

/*
 * Solves (*) for nrhs right-hand sides to ||b - A f||_2 <= tol ||b||_2 per
 * right-hand side, with the FP64 operator.  form: HPS_FORM_FP64 (restarted
 * GMRES in FP64) or HPS_FORM_MIXED (complex-FP32 apply and preconditioner
 * inside an FP64 Krylov basis, with the true residual recomputed in FP64 at
 * every restart, which restores FP64 accuracy), optionally OR'd with the
 * HPS_SOLVE_* flags.  s, t as in hps_rhs; f_out: nrhs*N_f complex doubles
 * (with HPS_SOLVE_X0 it holds the initial guess on entry).  Pointers may be
 * host or device memory (detected per pointer; host buffers are copied inside
 * the call).  info may be NULL.  The call returns after the result is in f_out.
 *
 * Each restart cycle (the first basis vector and `restart` Arnoldi steps:
 * preconditioner, apply, Gram-Schmidt, Givens rotation, normalization) runs
 * on the device without host synchronization: it is captured once per
 * configuration as a CUDA graph (on the handle's own stream) and replayed on
 * `stream`; a device flag written by each step's Givens kernel makes the
 * kernels of the following steps return at once after convergence.  The host
 * reads back once per cycle (residual norms and step counts).  Orthogonalization:
 * one classical Gram-Schmidt pass, and a second one at the steps where the
 * pass cancelled most of the vector (Rutishauser's criterion, ||w'|| <
 * ||w||/10, which bounds the loss of orthogonality per step by ~10 eps);
 * HPS_SOLVE_CGS2 forces the second pass everywhere.
 *
 * Errors: HPS_ENOCONV when maxit iterations did not reach tol (f_out holds
 * the last iterate, info the last residual); HPS_EBREAKDOWN when a residual
 * norm is not finite (NaN or Inf in the data or a non-finite intermediate),
 * found at the start or at a restart; HPS_ETIMEOUT when a tensor-core
 * kernel's bounded wait gave up; HPS_ECUDA for a CUDA error.
 */
int hps_gmres_solve(hps_handle* h, int form, const double* s, const double* t, int nrhs,
                    double tol, double* f_out, hps_solve_info* info, void* stream);

/*
 * Leaf solutions from face data (eq. (leaf)):
 * u^tau = A^{tau,-1} [s^tau; P^{-1} f^tau], P^{-1} moving the Gauss-point face
 * data to the leaf's Chebyshev face nodes.  s: nrhs interior vectors or NULL
 * (s = 0); f: nrhs face vectors (typically the output of hps_gmres_solve);
 * u_out: nrhs interior vectors (layout of hps_nodes' interior points);
 * u_face_out: NULL or nrhs face-layout vectors of u at the Chebyshev face
 * nodes (hps_nodes' cheb_face_xyz), the rest of the leaf's unknowns.  All
 * device pointers, complex double; one FP64 elimination per leaf and call
 * (cost comparable to hps_setup's).  Synchronous.
 */
int hps_recover(hps_handle* h, const double* s, const double* f, int nrhs, double* u_out,
                double* u_face_out, void* stream);

/*
 * The paper's own iterative path on the global system (Sec. 3-4), built with
 * options.full_system.  Vectors hold u at every node of every leaf:
 * [rhs][leaf][n] with n = n1^3 + 6 n1^2, the leaf's interior nodes (layout
 * above) followed by its six faces' n1 x n1 Chebyshev nodes (face layout,
 * hps_nodes' cheb_face_xyz).  Device pointers; p <= 14 for HPS_C128.
 *
 * hps_full_apply:   y = A u, A the global matrix of eq. (2x2): per leaf the
 *                   collocated operator of eq. (leaf) (interior rows by 1D
 *                   products along the three lines, Algorithm 1; face rows
 *                   F = N + i eta I) plus the neighbour's outgoing rows
 *                   G = N - i eta I across each shared face (Algorithm 2).
 * hps_full_precond: z = blockdiag(A~^tau)^{-1} r, the per-leaf block-Jacobi
 *                   preconditioner with homogenized leaf matrices (Sec. 4,
 *                   eq. (block_pc), Algorithms 3 and 4): Algorithm 3 for
 *                   A~_ii^{-1} and S~^{-1} = (A~^{-1})_bb per distinct (binned,
 *                   options.lambda_bin) constant.
 * hps_full_solve:   restarted GMRES on A u = [s; t; 0] with that preconditioner
 *                   (right preconditioning; form HPS_FORM_FP64 or HPS_FORM_MIXED,
 *                   optionally | HPS_SOLVE_NO_PRECOND), stopping on the FP64 true
 *                   relative residual <= tol.  s: nrhs interior vectors or NULL;
 *                   t: nrhs face vectors at Gauss points (moved to the Chebyshev
 *                   face nodes by P^{-1}) or NULL; u_out: nrhs global vectors.
 *                   Synchronous.  Errors as hps_gmres_solve.
 * The face system above is the production path; this one is the paper's own
 * design, kept for comparison.
 */
int hps_full_apply(hps_handle* h, int dtype, const void* u, void* y, int nrhs, void* stream);
int hps_full_precond(hps_handle* h, int dtype, const void* r, void* z, int nrhs, void* stream);
int hps_full_solve(hps_handle* h, int form, const double* s, const double* t, int nrhs, double tol, double* u_out,
                   hps_solve_info* info, void* stream);

/*
 * Distinct preconditioner blocks of the handle: clusters, distinct K_c blocks
 * and distinct B blocks (see hps_options.lambda_bin).  Any pointer may be NULL.
 * HPS_EINVAL when the handle has no preconditioner.
 */
int hps_precond_info(const hps_handle* h, int* clusters, int* k_blocks, int* b_blocks);

/*
 * Host-only planning of the shared preconditioner blocks that hps_setup does
 * after binning (Sec. 4.1 remark; no device work, no GPU needed).  lambda_q:
 * the binned constants of every leaf, nx*ny*nz complex doubles (interleaved,
 * leaf order ix + nx*(iy + ny*iz)).  Clusters are the 2x2x2 blocks of leaves
 * (1-wide at the end of an odd axis), numbered x fastest.  A leaf's B block is
 * keyed by (lambda_q, internal-face mask); a cluster's K_c block by the
 * sequence of its leaves' keys; -0 and +0 are one key.  Blocks are numbered in
 * order of first appearance.  Writes leaf_b_block[nx*ny*nz] and
 * cluster_k_block[*clusters] (either may be NULL; the cluster count is
 * ceil(nx/2)*ceil(ny/2)*ceil(nz/2)) and the counts (any may be NULL).
 * HPS_EINVAL for an invalid grid, a NULL lambda_q or a non-finite constant.
 */
int hps_plan_blocks(const hps_grid* grid, const double* lambda_q, int* leaf_b_block, int* cluster_k_block,
                    int* clusters, int* k_blocks, int* b_blocks);

/*
 * Host-only: M = V diag(E) V^{-1} for a small real n x n matrix M with real,
 * distinct eigenvalues -- the per-axis factorization L1 = V E V^{-1} that
 * Algorithm 3 (Sec. 4.1) needs and hps_setup computes when full_system is set
 * (no device work).  Shifted QR iteration with deflation for E, inverse
 * iteration for the columns of V, Gauss-Jordan with partial pivoting for
 * V^{-1}.  M, V, Vinv: host row-major n x n; E: host n; 1 <= n <= 64.
 * HPS_EBREAKDOWN when the iteration does not converge (e.g. a complex pair)
 * or when max|M V - V E| > 1e-9 max|M| or max|V V^{-1} - I| > 1e-9;
 * HPS_EINVAL for bad arguments or a non-finite entry.
 */
int hps_axis_eig(int n, const double* M, double* V, double* Vinv, double* E);

/* What hps_export copies out (host doubles, interleaved complex). */
#define HPS_EXPORT_R 0      /* R^index, 6q^2 x 6q^2 row-major, FP64 */
#define HPS_EXPORT_H 1      /* H^index, 6q^2 x n1^3 row-major */
#define HPS_EXPORT_LAMBDA 2 /* lambda^index: one complex value */
#define HPS_EXPORT_KC 3     /* K_c of cluster index, n_int x n_int row-major */
#define HPS_EXPORT_B 4      /* B^index: leaf index's (internal rows x external cols) block of R~ */
/* Copies one leaf's (or cluster's) operator to host memory for inspection.
 * Returns the number of doubles written (>0) or a negative error code;
 * with host_out == NULL only the size is returned. */
long long hps_export(hps_handle* h, int what, int index, double* host_out);

/* Replaces the stored ItI map R^index of one leaf (Definition in Sec. 2.2: the
 * map from incoming to outgoing impedance data on the leaf's six faces, Gauss
 * basis) with a map supplied by the caller: host_in holds 6q^2 x 6q^2 complex
 * doubles, row-major, interleaved, the layout hps_export writes.  The FP64
 * copy is overwritten as given and the complex-FP32 copy with the values
 * rounded to nearest.  Only what = HPS_EXPORT_R is accepted.  Use: checking
 * the apply kernels against an independent operator, or a leaf map computed
 * by another discretization of the same leaf.  The preconditioner and H are
 * not changed.  Synchronous; HPS_EINVAL for a bad index, what or a
 * non-finite entry. */
int hps_import_map(hps_handle* h, int what, int index, const double* host_in);

/*
 * Test hook for the bounded device waits (no counterpart in the paper).  Every
 * wait of the tensor-core kernels on an mbarrier is bounded: after a limit the
 * CTA sets the handle's error word, stops issuing work, waits (bounded) for its
 * own copies and tensor-core operations, frees its tensor memory and returns,
 * and the solve returns HPS_ETIMEOUT with the GPU context intact.  With
 * what = HPS_INJECT_SKIP_ARRIVAL, one warp of CTA 0 of the multi-RHS
 * tensor-core apply leaves out one arrival, so that the MMA-issuing thread's
 * wait runs out; spin_limit (> 0) replaces the wait limit (tries of
 * mbarrier.try_wait) of that kernel, 0 keeps the default.  HPS_INJECT_NONE
 * with spin_limit 0 restores normal operation.  Drops the handle's captured
 * GMRES cycle.  For tests of the time-out path only.
 */
#define HPS_INJECT_NONE 0
#define HPS_INJECT_SKIP_ARRIVAL 1
int hps_test_inject(hps_handle* h, int what, long long spin_limit);

/* Launch shapes of a handle's batched GEMV kernels, per right-hand-side group
 * (1, 2, <= 4, <= 8 per launch): matrix rows per warp pass (1, 2, 4, 8) and a
 * cap on resident CTAs per SM (0 = the occupancy limit). */
typedef struct {
  int apply_rows_per_warp[2][4];   /* ItI apply with FP32 maps [0], FP64 maps [1] */
  int apply_ctas_per_sm[2][4];
  int stage_k_rows_per_warp[4];    /* preconditioner stage K, member groups of 1, 2, 4, 8 */
  int stage_k_ctas_per_sm[4];
  int tuned;                       /* 1 when chosen by the autotuner at setup */
} hps_launch_shapes;
int hps_get_launch_shapes(const hps_handle* h, hps_launch_shapes* out);

/* Phases timed by the profiler (indices into hps_profile.ms / count). */
#define HPS_PHASE_APPLY 0     /* w = A z inside the Arnoldi loop (working precision) */
#define HPS_PHASE_PRECOND_B 1 /* preconditioner stage B: z_ext = r_ext, t = r_int - B r_ext */
#define HPS_PHASE_PRECOND_K 2 /* preconditioner stage K: z_int = K_c t */
#define HPS_PHASE_ARNOLDI 3   /* CGS2 dots/updates, norm, Givens, scaling */
#define HPS_PHASE_RESIDUAL 4  /* FP64 true residual b - A x at each restart */
#define HPS_PHASE_RHS 5       /* right-hand side b = tbar - Pi H s */
#define HPS_PHASE_UPDATE 6    /* least squares, x += M^{-1} V y */
#define HPS_NPHASES 8

typedef struct {
  long long launches;        /* kernels launched by hps_gmres_solve / hps_apply / hps_precond */
  double ms[HPS_NPHASES];    /* device time per phase (CUDA events on the call's stream) */
  long long count[HPS_NPHASES]; /* timed intervals per phase */
} hps_profile;

/* Turns per-phase CUDA-event timing on (1) or off (0).  The launch counter
 * always runs.  Timing adds two event records per timed interval. */
int hps_profile_enable(hps_handle* h, int on);

/* Copies the counters accumulated since the last reset into *out (waiting for
 * the recorded events), and resets them when reset != 0. */
int hps_profile_read(hps_handle* h, hps_profile* out, int reset);

/* Device bytes held by the handle. */
size_t hps_memory_bytes(const hps_handle* h);

/* Frees all device state of the handle (NULL is accepted). */
int hps_destroy(hps_handle* h);

/* Message of the last failure on the calling thread ("" when none). */
const char* hps_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HPS_H */
