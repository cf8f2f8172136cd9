/*
 * topo.h -- C ABI of the GB300 (sm_103a) AARMR topology-optimisation library.
 *
 * The library solves the equilibrium equation K(rho~) u = f of minimum-
 * compliance topology optimisation (Eq. 3) on a regular grid of unit Q4
 * (plane stress) or hex8 elements with the modified SIMP law (Eq. 1), by
 *   - MGCG: conjugate gradients preconditioned by a Galerkin V-cycle
 *     (Algorithm 2), which also maintains the PARM (Eq. 27-28), and
 *   - the CARM reduced model built from the PARM (Eq. 15-29),
 * and provides the compliance sensitivity (Eq. 6, 34), the density filter
 * and its transpose (Eq. 31-33) and the optimality-criteria update (Eq. 3
 * constraint, update rule of the paper's ref. [31]).  Algorithm 1 (the
 * choice between CARM and MGCG) is driven by the caller from these calls.
 *
 * Conventions (all sizes in elements of the stated type):
 *   nel  = nelx*nely (2D) or nelx*nely*nelz (3D)        -- elements
 *   nn   = (nelx+1)*(nely+1)(*(nelz+1))                  -- nodes
 *   n    = dim*nn                                         -- DOFs
 *   node (i,j,k) = i + (nelx+1)*(j + (nely+1)*k); DOF c of a node = dim*node+c;
 *   element (ex,ey,ez) = ex + nelx*(ey + nely*ez).
 *   Vectors are float64, contiguous, in that DOF order.  Multi-vector blocks
 *   are column-major (column i starts at i*n).
 *
 * Ownership: the caller owns every buffer.  Device memory for the solver
 * state is one caller-allocated workspace whose size to_workspace_bytes()
 * reports; the library never allocates device memory.  Pointer arguments
 * marked (dev) are device pointers borrowed for the duration of the call;
 * (host) are host pointers.  Every call is enqueued on the CUDA stream given
 * to to_mesh_init and returns without synchronising unless stated.
 *
 * Errors: every call returns a to_status.  Invalid sizes, null pointers or
 * non-finite scalars return TO_E_INVALID before any launch.  A failed CUDA
 * launch returns TO_E_CUDA.  to_last_error() gives a message.  No call
 * aborts the process.
 */
#ifndef TOPO_H_
#define TOPO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t to_status;

enum {
  TO_OK = 0,
  TO_E_INVALID = 1,        /* bad argument; nothing launched */
  TO_E_STATE = 2,          /* call out of order (e.g. CARM before the PARM is full) */
  TO_E_OOM = 3,            /* workspace smaller than to_workspace_bytes() */
  TO_E_CUDA = 4,           /* a CUDA runtime call or launch failed */
  TO_E_NOT_CONVERGED = 5,  /* iteration limit reached; result still written */
  TO_E_SINGULAR = 6,       /* a factorisation met a non-positive pivot */
  TO_E_TIMEOUT = 7         /* a bounded device wait expired */
};

enum { TO_FP64 = 0, TO_MIXED = 1 };
enum { TO_FILTER_DENSITY = 0, TO_FILTER_SENS = 1 };
enum { TO_SOLVE_WARM_START = 1, TO_SOLVE_PUSH_PARM = 2 };
enum { TO_OP_K = 0, TO_OP_KREF = 1, TO_OP_DK = 2 };
enum { TO_PREC_NATIVE = 0, TO_PREC_FP64 = 1, TO_PREC_FP32 = 2, TO_PREC_DF = 3 };

typedef struct to_ctx to_ctx;

/* Problem description.  dim is 2 (Q4, plane stress) or 3 (hex8); nel[2] is
 * ignored in 2D.  E0, Emin, penal: SIMP law of Eq. 1; nu: Poisson ratio;
 * rmin: density-filter radius of Eq. 32 in element lengths.  mg_levels
 * counts all grids including the finest; every nel[i] must be divisible by
 * 2^(mg_levels-1).  precision: TO_FP64 (all arithmetic in float64) or
 * TO_MIXED (stiffness apply, V-cycle and smoother in float32; CG vectors,
 * dot products, reduced solves, Gram-Schmidt, compliance and OC in
 * float64).  n_parm = N_s columns of the PARM, n_carm = N_m columns of the
 * CARM (each 1..16). */
typedef struct to_mesh_desc {
  int32_t dim;
  int32_t nel[3];
  double E0, Emin, nu, penal, rmin;
  int32_t mg_levels;
  int32_t precision;
  int32_t n_parm, n_carm;
} to_mesh_desc;

/* Bytes of device workspace needed for a problem (host-only query). */
to_status to_workspace_bytes(const to_mesh_desc* desc, int64_t* bytes);

/* Create a solver context.
 * fixed_mask (dev, uint8, n): 1 = the DOF is prescribed zero (copied).
 * f (dev, float64, n): nodal load vector (copied); f must be zero on fixed
 *   DOFs and not identically zero.
 * workspace (dev), ws_bytes: caller allocation of to_workspace_bytes() bytes,
 *   256-byte aligned; owned by the caller and used until to_destroy.
 * stream: cudaStream_t (as void*) on which every call of this context runs.
 * Supports must be closed under coarse-grid interpolation (every fixed fine
 * DOF is interpolated only from fixed coarse DOFs); otherwise TO_E_INVALID.
 * The Galerkin coarse operators rely on it. */
to_status to_mesh_init(const to_mesh_desc* desc, const uint8_t* fixed_mask, const double* f,
                       void* workspace, int64_t ws_bytes, void* stream, to_ctx** out);

/* Set the physical densities rho~ (dev, float64, nel) of this design
 * iteration: E_e = Emin + (E0-Emin) rho~_e^penal (Eq. 1).  The previous E
 * becomes the reference stiffness K_ref of the reanalysis (Eq. 8); the first
 * call sets both.  Invalidates the multigrid hierarchy (rebuilt lazily). */
to_status to_set_density(to_ctx* ctx, const double* rho_phys);

/* MGCG (Algorithm 2 as preconditioner of CG) for K(E) u = f.
 * u (dev, float64, n): in: initial guess if flags has TO_SOLVE_WARM_START
 *   (else ignored and zero is used; its entries on fixed DOFs are taken as
 *   zero, as in the solution); out: the solution.
 * rtol: stop when ||f - K u|| / ||f|| < rtol.  In TO_FP64 the CG recursive
 *   residual is tested; in TO_MIXED (float32 operator inside CG) the
 *   recursive residual is replaced by the float64 true residual f - K u
 *   whenever it has dropped 100x since the last replacement, and
 *   convergence is declared on the true residual; where the true residual
 *   exceeds the recursive one by more than 1.5x, CG restarts from it.
 * maxit: CG iteration cap (>= 1).  On the cap the last iterate is returned
 *   with TO_E_NOT_CONVERGED.
 * flags & TO_SOLVE_PUSH_PARM: append u/||u|| to the PARM (Eq. 28), dropping
 *   the oldest column when full (Sec. 3.1).
 * iters (host, may be NULL): CG iterations taken; relres (host, may be
 *   NULL): final relative residual.  This call synchronises the stream.
 * The host reads |r|^2 once per CG iteration; the read is enqueued before
 * the next preconditioner application and waited on after it, so the
 * V-cycle runs during the round trip (its result is discarded on the
 * iteration that stops).  The first call on a context allocates 64 bytes of
 * pinned host memory for that read (released by to_destroy).
 * The first solve after to_set_density rebuilds the multigrid hierarchy; in
 * TO_MIXED the coarsest matrix's explicit inverse is formed in float32 and
 * checked (one small synchronising read), and a context whose float32
 * factorisation meets a non-positive pivot (near-void designs) factors in
 * float64 from then on. */
to_status to_mgcg_solve(to_ctx* ctx, double rtol, int32_t maxit, int32_t flags, double* u,
                        int32_t* iters, double* relres);

/* Append u/||u|| (u: dev, float64, n) to the PARM, FIFO (Eq. 27-28). */
to_status to_parm_push(to_ctx* ctx, const double* u);
/* Number of PARM columns currently held (host query, no sync). */
to_status to_parm_count(to_ctx* ctx, int32_t* count);
/* Remove all PARM columns. */
to_status to_parm_reset(to_ctx* ctx);

/* Truncation of the CARM basis (Eq. 21, which states no rule): with the
 * basis columns scaled to unit length, singular directions with
 * sigma_i <= TO_CARM_SVD_TOL * sigma_1 are dropped.  The value sits well
 * above the rounding level of the basis in either precision (both build it
 * with float64-accurate products) and below every direction that changes
 * the reduced solution measurably. */
#define TO_CARM_SVD_TOL 1e-6
/* A basis column keeping <= TO_QR_DEPENDENT_TOL of its norm after being
 * orthogonalised twice against the earlier ones is numerically dependent on
 * them: it adds no column to the orthonormal factor (its projections stay
 * in the triangular factor, so the SVD still sees it). */
#define TO_QR_DEPENDENT_TOL 1e-10

/* Build the CARM basis R~ from u_last (dev, float64, n): K_Phi = Phi^T K_ref
 * Phi (Eq. 15), r_1 = u_last, r_i = -Phi K_Phi^{-1} Phi^T dK r_{i-1}
 * (Eq. 18-20, 26), with float64-accurate products in both precisions; then
 * Eq. 21: R (columns scaled to unit length) = R~ Sigma V^T truncated at
 * TO_CARM_SVD_TOL, computed as a QR factorisation of R (classical
 * Gram-Schmidt, two passes per column) followed by the SVD of the small
 * triangular factor on the device.  R~ has the kept left singular vectors
 * as columns, in descending order of sigma.  Needs a full PARM (else
 * TO_E_STATE); TO_E_SINGULAR if nothing is kept (u_last = 0).
 * Synchronises once (reads the kept count). */
to_status to_carm_build(to_ctx* ctx, const double* u_last);

/* Autotuner of the launch shapes of the column-streaming 3D operators.
 * Their free parameter is the number of node layers a block streams along
 * z (each chunk recomputes one element layer below it, so fewer, longer
 * chunks do less redundant work but fill fewer SMs).  to_autotune times,
 * with CUDA events on the context stream, every distinct chunk length of
 * each kernel the context's solver runs on this grid:
 *   TO_TUNE_OP_APPLY / _RESID / _SMOOTH: the finest-grid operator of the
 *     solver (float32 in TO_MIXED, float64 in TO_FP64) as K p, as the
 *     V-cycle's residual and as its post-smoother;
 *   TO_TUNE_GAL1_RESID / _SMOOTH: the level-1 Galerkin operator applied
 *     from the finest moduli (3D, >= 3 levels);
 *   TO_TUNE_ACC_APPLY / _RESID: the double-float operator (TO_MIXED).
 * For the float32 finest-grid kernels it also times the 16-row tile
 * variant (TO_OPERATOR_TALL_TILES) and the work-list launch of either tile
 * (TO_OPERATOR_WORK_LIST).
 * It keeps the fastest (the occupancy heuristic's own shape when within 1 %
 * of it), applies it to every later launch of that kernel on this context,
 * drops the captured V-cycle graphs so that they are recaptured with it, and
 * caches it for the process under (device, kernel, grid), so later
 * contexts of the same grid take it without timing.  Results do not depend
 * on the chunking (every node sums its element contributions in the same
 * order).  reps: timed launches per candidate (>= 1); results (host, may be
 * NULL): up to cap entries, one per kernel; *count (host): entries written.
 * Needs to_set_density first (TO_E_STATE); synchronises; do not call during
 * stream capture.  2D contexts have nothing to tune (*count = 0). */
enum { TO_TUNE_OP_APPLY = 0, TO_TUNE_OP_RESID = 1, TO_TUNE_OP_SMOOTH = 2, TO_TUNE_GAL1_RESID = 3,
       TO_TUNE_GAL1_SMOOTH = 4, TO_TUNE_ACC_APPLY = 5, TO_TUNE_ACC_RESID = 6, TO_TUNE_N = 7 };
typedef struct {
  int32_t kernel;        /* TO_TUNE_* */
  int32_t candidates;    /* chunk lengths timed (0: taken from the process cache) */
  int32_t chunk_layers;  /* chosen node layers per chunk (0: the heuristic's shape) */
  double chosen_us;      /* average launch time of the chosen shape (0 when cached) */
  double heuristic_us;   /* average launch time of the heuristic's shape (0 when cached) */
  int32_t variant;       /* float32 finest-grid kernels (TO_TUNE_OP_*): bit 0 the tile,
                            0 = 8-row tiles, 1 = 16-row tiles (TO_OPERATOR_TALL_TILES);
                            bit 1 the work-list launch (TO_OPERATOR_WORK_LIST) */
} to_tune_result;
to_status to_autotune(to_ctx* ctx, int32_t reps, to_tune_result* results, int32_t cap,
                      int32_t* count);

/* Continuous batching of design iterations.  A serving loop advances every
 * active job by one design iteration per round (Fig. 1): the density phase
 * of all jobs, each job's solve (MGCG or CARM, on its own stream), then the
 * update phase of all jobs; jobs join and leave between rounds.
 * to_batch_step runs one phase of n jobs as ONE CUDA graph launch on
 * `stream` (a cudaStream_t as void*):
 *   TO_PHASE_DENSITY: rho_phys = H(rho)/Hs (Eq. 31-32), then
 *     to_set_density(ctx, rho_phys) (Eq. 1);
 *   TO_PHASE_UPDATE: C and dc of u (Eq. 3, 6/34) into compliance_dev and
 *     dc, dc_f = H^T(dc/Hs) (Eq. 33), and the OC update of rho (ref. [31] of
 *     the paper), its change into change_dev (may be NULL).
 * Each job's kernels are one branch of the graph, captured from the job's
 * context stream with its own buffers in the order the single-job calls
 * use, so every job computes bitwise what the single-job calls compute; the
 * branches run concurrently.  The graph is captured on the first call for a
 * job table and cached (up to 64 tables, least recently used dropped; a
 * table holding a destroyed context is dropped) and replayed while the
 * table repeats (including which of each job's two modulus buffers is the
 * current one, so a steady set of jobs alternates between two cached graphs
 * per phase).  The call enqueues and returns; `stream`
 * waits for nothing else, so order it after each job's previous work (for
 * example by making `stream` one of the jobs' context streams, or with
 * events).  No other thread may use the jobs' context streams during the
 * call.  n in [1, TO_BATCH_MAX_JOBS]; a context appearing twice, NULL
 * arrays, a context without a density (update phase) or bad volfrac/move
 * give TO_E_INVALID with nothing launched; errors are read with
 * to_last_error(NULL).  The paper runs one design loop; the batching is an
 * extension for serving several. */
#define TO_BATCH_MAX_JOBS 256
enum { TO_PHASE_DENSITY = 0, TO_PHASE_UPDATE = 1 };
typedef struct {
  to_ctx* ctx;
  double* rho;              /* design variables (dev, nel): read; written by the update */
  double* rho_phys;         /* physical densities (dev, nel): written by the density phase */
  const double* u;          /* displacement (dev, n): read by the update */
  double* dc;               /* compliance sensitivity (dev, nel): written by the update */
  double* dc_f;             /* filtered sensitivity (dev, nel): written by the update */
  const double* dv_f;       /* filtered volume sensitivity (dev, nel): read by the update */
  double* compliance_dev;   /* dev, 1 double: written by the update */
  double* change_dev;       /* dev, 1 double, or NULL */
  double volfrac, move;     /* OC parameters (update) */
} to_batch_job;
to_status to_batch_step(const to_batch_job* jobs, int32_t n, int32_t phase, void* stream);

/* Operator and multigrid options of a context (default 0).
 * TO_OPERATOR_TENSOR_CORES (3D TO_MIXED only): the float32 finest-grid
 * operator's products (K p of CG, the
 * V-cycle's finest residual and smoother) run on the tensor cores (tcgen05,
 * TF32 split into two parts per operand, three products, float32
 * accumulation: about 2^-21 relative per element product) instead of the
 * CUDA cores.  Results then differ from the default at that rounding level.
 * Drops the captured V-cycle graphs and the autotuned launch shapes (tune
 * again).  A device wait that expires in these kernels makes the next
 * to_mgcg_solve return TO_E_TIMEOUT.  TO_E_INVALID for unknown bits or a
 * 2D context. */
#define TO_OPERATOR_TENSOR_CORES 1
/* TO_OPERATOR_FUSED_COARSE: the coarse end of the V-cycle (Algorithm 2) --
 * the stored levels whose assembled stencil is at most a few MB, down to
 * the coarsest grid and back -- runs as one launch of one thread-block
 * cluster with hardware cluster barriers between the steps, instead of one
 * kernel per step (the default).  The results are bit for bit the same.
 * Measured at 192 x 96 x 96 it is slower (each step then runs on the
 * cluster's 8-16 SMs with one memory round trip or more per step, where the
 * one-kernel steps use the whole GPU and overlap their launches), so it is
 * off by default.  Changing it drops the captured V-cycle graphs. */
#define TO_OPERATOR_FUSED_COARSE 2
/* TO_OPERATOR_TALL_TILES: the float32 finest-grid operator (3D TO_MIXED)
 * runs its 256-thread variant with 16-row tiles (16 element rows computed
 * for 15 owned node rows instead of 8 for 7) in every launch; to_autotune
 * also times that variant and may select it for a kernel on its own.  The
 * results are bit for bit the same.  Changing it drops the captured
 * V-cycle graphs. */
#define TO_OPERATOR_TALL_TILES 4
/* TO_OPERATOR_WORK_LIST: the float32 finest-grid operator (3D TO_MIXED) is
 * launched as a work list in every launch: one CTA per resident block slot,
 * each taking the next (tile, z-chunk) item from a device counter until
 * none is left (the last CTA resets the counter), instead of one block per
 * item; to_autotune also times this launch and may select it for a kernel
 * on its own.  The results are bit for bit the same.  Changing it drops the
 * captured V-cycle graphs. */
#define TO_OPERATOR_WORK_LIST 8
to_status to_operator_options(to_ctx* ctx, int32_t flags);

/* Options of to_carm_build (default 0).  TO_CARM_R1_PROJECTED_LOAD: the
 * first basis vector is the load multiplied by the approximate inverse of
 * Eq. 18, r_1 = Phi K_Phi^{-1} Phi^T f, instead of u_last (the alternative
 * the paper compares in Fig. 2 and finds to change little); u_last is then
 * still required but unused.  Unknown bits give TO_E_INVALID. */
#define TO_CARM_R1_PROJECTED_LOAD 1
to_status to_carm_options(to_ctx* ctx, int32_t flags);

/* Test hook on the last CARM basis: *kq (host) = columns of the QR factor,
 * *k (host) = directions kept by Eq. 21, sigma (host, may be NULL, n_carm
 * doubles) = singular values of the unit-column basis, descending
 * (synchronises when sigma is given).  TO_E_STATE before to_carm_build. */
to_status to_carm_info(to_ctx* ctx, int32_t* kq, int32_t* k, double* sigma);

/* Test hook: column j (0 <= j < k) of the last CARM basis R~, widened to
 * float64 into out (dev, n).  TO_E_INVALID for j out of range. */
to_status to_carm_basis_column(to_ctx* ctx, int32_t j, double* out);

/* Test hook: *err (host) = max_ij |(R~^T R~)_ij - delta_ij| over the last
 * CARM basis (synchronises).  Overwrites the reduced matrix, so call
 * to_carm_solve afterwards, not before. */
to_status to_carm_basis_error(to_ctx* ctx, double* err);

/* Reduced solve on the last CARM basis (K R~ is always formed with the
 * float64 operator, also in TO_MIXED): K_R = R~^T K R~, f_R = R~^T f,
 * y = K_R^{-1} f_R (Eq. 23-24), u = R~ y (Eq. 25, dev float64 n, out) and
 * eps = ||K R~ y - f|| / ||f|| (Eq. 29) written to eps (host, may be NULL;
 * synchronises when given) and to eps_dev (dev, may be NULL). */
to_status to_carm_solve(to_ctx* ctx, double* u, double* eps, double* eps_dev);

/* Compliance and its sensitivity for displacement u (dev, n):
 * C = sum_e E_e u_e^T KE u_e (Eq. 3) -> compliance_dev (dev, 1 double) and
 * dc_e = -penal (E0-Emin) rho~_e^(penal-1) u_e^T KE u_e (Eq. 6 / 34) -> dc
 * (dev, nel). */
to_status to_sensitivity(to_ctx* ctx, const double* u, double* compliance_dev, double* dc);

/* Compliant mechanisms (Sec. 4.3, the displacement inverter).
 *
 * to_mesh_springs: linear springs to ground on free finest-grid DOFs (2D
 * contexts): every product with K and K_ref (TO_OP_K, TO_OP_KREF, the CG,
 * the V-cycle's finest level, the CARM's K_ref Phi and K R~) becomes
 * (K + S) x with S diagonal, k[q] at dofs[q]; dK is unchanged (the springs
 * do not depend on the design); the multigrid hierarchy includes P^T S P.
 * dofs (host int64, n) and k (host float64 >= 0, n) are copied; n <=
 * TO_MAX_SPRINGS; n = 0 removes them.  Takes effect at the next
 * to_set_density.  Synchronises (reads the DOFs' masks).  TO_E_INVALID for
 * a 3D context, a DOF out of range, repeated or fixed, or a bad k. */
#define TO_MAX_SPRINGS 4
to_status to_mesh_springs(to_ctx* ctx, int32_t n, const int64_t* dofs, const double* k);

/* Sensitivity of an output displacement u_out = l^T u through the adjoint
 * field lam (K lam = l): dc_e = -penal (E0-Emin) rho~_e^(penal-1)
 * lam_e^T KE u_e -> dc (dev, nel), the prescribed DOFs taken as zero in
 * both fields; sum_e E_e lam_e^T KE u_e -> mutual_dev (dev, 1 double).
 * u, lam: dev float64 n.  Uses the density of the last to_set_density. */
to_status to_sensitivity_adjoint(to_ctx* ctx, const double* u, const double* lam,
                                 double* mutual_dev, double* dc);

/* Damping exponent eta of the OC update (default 1/2, the compliance rule):
 * rho_new = clamp(rho max(0, -dc / (lambda dv))^eta) within the move limit
 * (0.3 for the mechanism problem).  Applies to to_oc_update and the batched
 * update phase (not to the no-allocation entry point).  TO_E_INVALID
 * unless 0 < eta <= 1. */
to_status to_oc_options(to_ctx* ctx, double eta);

/* Density filter (Eq. 31-32), mode TO_FILTER_DENSITY: out = (H in) / Hs;
 * or its transpose for sensitivities (Eq. 33), mode TO_FILTER_SENS:
 * out = H^T (in / Hs).  in, out: dev float64 nel, must not alias. */
to_status to_filter(to_ctx* ctx, int32_t mode, const double* in, double* out);

/* Optimality-criteria update of the design rho (dev, float64, nel, in/out):
 * rho_new = clamp(rho sqrt(max(0, -dc_f/(lam dv_f))), max(0, rho-move),
 * min(1, rho+move)) with lam chosen by bisection on [0, 1e9] to a relative
 * bracket of 1e-13 so that sum_e dv_f,e rho_new,e = volfrac*nel (the
 * filtered volume when dv_f = H^T(1/Hs), Eq. 3).  dc_f, dv_f: dev nel.
 * change_dev (dev, 1 double, may be NULL): max |rho_new - rho|. */
to_status to_oc_update(to_ctx* ctx, double volfrac, double move, const double* dc_f,
                       const double* dv_f, double* rho, double* change_dev);

/* The optimality-criteria update of to_oc_update for callers that cannot
 * allocate device memory (code running inside another runtime's memory pool
 * or allocator hook, plugins whose host application owns all device
 * allocations): it needs no context and no workspace and allocates nothing.
 * The paper has no counterpart; this is an interface variant.
 * nel: element count, 1 <= nel <= 2,097,152 (else TO_E_INVALID, nothing
 *   launched).  volfrac, move, dc_f, dv_f, rho, change_dev: as for
 *   to_oc_update (dev pointers; change_dev may be NULL).  stream: a
 *   cudaStream_t (as void*) on which the kernels are enqueued; the call does
 *   not synchronise.
 * Scratch: a ~16 MiB file-scope device array of the library, which every GPU
 * that loads libtopo.so holds until the process exits.  Its device address
 * belongs to the CUDA context current when the call is made: the first call
 * in each context (the primary context of a device, a context the caller
 * created and made current, or the new primary context after a
 * cudaDeviceReset) looks the address up (cudaGetSymbolAddress) and caches
 * it under the context's unique ID; make that first call before any stream
 * capture.  All calls in one context share the array: calls that overlap on
 * the GPU (different streams) race and must be serialised by the caller.
 * Errors are reported by the return code and to_last_error(NULL). */
to_status to_oc_update_noalloc(int64_t nel, double volfrac, double move, const double* dc_f,
                               const double* dv_f, double* rho, double* change_dev,
                               void* stream);

/* y = op(x) for x, y dev float64 n (no aliasing).  op: TO_OP_K (current
 * stiffness with BCs, Eq. 7), TO_OP_KREF (reference stiffness, Eq. 8) or
 * TO_OP_DK (dK = K - K_ref, zero on fixed DOFs).  prec: TO_PREC_NATIVE
 * (the context's apply precision), TO_PREC_FP64, TO_PREC_FP32 (3D: x is
 * rounded to float32 and the float32-storage operator of the mixed solver
 * runs; y is its result widened) or
 * TO_PREC_DF (3D: double-float arithmetic on the FP32 pipe, ~2^-48
 * relative; elsewhere float64).  TO_MIXED uses TO_PREC_DF for the products
 * that must be float64-accurate (true CG residuals, K R~). */
to_status to_apply(to_ctx* ctx, int32_t op, int32_t prec, const double* x, double* y);

/* One V-cycle of the current hierarchy (Algorithm 2): z ~= K^{-1} r, with
 * r, z dev float64 n (builds the hierarchy if stale). */
to_status to_vcycle(to_ctx* ctx, const double* r, double* z);

/* Galerkin operator of level l >= 1 (coarse grid l of the hierarchy):
 * y = A_l x with x, y dev float64 of that level's DOF count (see
 * to_level_info).  For tests of the coarse operators. */
to_status to_level_apply(to_ctx* ctx, int32_t level, const double* x, double* y);
/* Element counts per axis and DOF count of level l. */
to_status to_level_info(to_ctx* ctx, int32_t level, int32_t nel_out[3], int64_t* ndof);

/* Profiling: launches of the kinds selected by the bit mask `kinds` (bit k
 * = kind k; 0 turns profiling off) are bracketed by CUDA events on the
 * context stream.  kind 0 = finest-grid operator with float32 storage and
 * arithmetic (the operator of the mixed solver), 1 = coarse-grid Galerkin
 * operator, 2 = whole V-cycle, 3 = finest-grid operator in the other
 * precisions (float64, double-float, float32 arithmetic on float64 storage).
 * Inside MGCG the V-cycle runs as a captured CUDA graph: its inner launches
 * are timed only through kind 2.  to_profile_read synchronises,
 * returns the number of timed launches, their summed milliseconds and
 * (bytes, may be NULL) their summed algorithmic DRAM bytes (each input and
 * output array counted once), and forgets them.  to_launch_count returns
 * the number of kernels launched by this context since the last reset. */
to_status to_profile_enable(to_ctx* ctx, int32_t kinds);
to_status to_profile_read(to_ctx* ctx, int32_t kind, int64_t* count, double* ms, double* bytes);
to_status to_launch_count(to_ctx* ctx, int64_t* count, int32_t reset);

/* Message of the last error of ctx (or of the last context-less call when
 * ctx is NULL).  The string is owned by the library. */
const char* to_last_error(const to_ctx* ctx);

/* Release host-side state (the workspace stays the caller's). */
void to_destroy(to_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TOPO_H_ */
