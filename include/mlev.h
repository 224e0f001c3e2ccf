/*
 * mlev - multilevel local and parallel P1 finite element eigensolver on one GPU.
 *
 * Computes the smallest eigenpair (lambda_{h_n}, u_{h_n}) of
 *     a(u, v) = lambda b(u, v)  for all v in V_{0h}(Omega),   b(u, u) = 1,
 * with a(u, v) = (kappa grad u, grad v) and b(u, v) = (u, v) (paper Section 3,
 * Eq. Weak_Eigenvalue_Problem), by Algorithm 4.2 of Li, Han, Xie, You ("Local and
 * parallel finite element algorithm based on multilevel discretization for
 * eigenvalue problem"): an eigenproblem on V_{0h_1}, then n-1 applications of the
 * one correction step of Algorithm 4.1 (local auxiliary problems on Omega_j,
 * gluing with the G_{m+1} boundary value problem, Rayleigh-Ritz on
 * V_{0H} + span{u~}).
 *
 * Geometry: T_H is a grid of ncx x ncy square cells of side H (origin x0, y0), a
 * cell mask selects Omega, and every cell is split by its SW-NE diagonal. Level k
 * has mesh size h_k = H / 2^k (T_{h_1} is one regular refinement of T_H,
 * Section 4.2). All nodal arrays are row-major with x fastest; a level-k lattice
 * has (ncy*2^k + 1) rows of (ncx*2^k + 1) nodes.
 *
 * Conventions for every call:
 *  - Return value: MLEV_OK (0) or a negative MLEV_E* code; mlev_last_error()
 *    gives a message. No C++ exception crosses this interface.
 *  - Host arrays passed to mlev_set_* are copied before the call returns.
 *  - Device buffers (workspace, kappa when kappa_on_device, outputs) are owned by
 *    the caller. The library never allocates device memory; mlev_solve works only
 *    inside the caller's workspace and launches on the caller's stream.
 *  - One context must not be used from two host threads at once.
 */
#ifndef MLEV_H
#define MLEV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MLEV_OK 0
#define MLEV_EINVAL (-1)        /* bad argument or inconsistent setup */
#define MLEV_ENOMEM (-2)        /* workspace too small / host allocation failed */
#define MLEV_ECUDA (-3)         /* a CUDA runtime call failed */
#define MLEV_ENOCONV (-4)       /* an iteration hit its cap before its tolerance */
#define MLEV_ETIMEOUT (-5)      /* a bounded device-side wait gave up */
#define MLEV_EUNSUPPORTED (-6)  /* valid input outside what this build implements */
#define MLEV_ESTATE (-7)        /* call order violated (e.g. solve before setup) */

#define MLEV_KAPPA_ONE 0             /* kappa == 1 (the Laplacian of Example 1) */
#define MLEV_KAPPA_PER_COARSE_CELL 1 /* kappa[b][cj][ci], constant on each cell of T_H */
#define MLEV_KAPPA_PER_FINE_ELEM 2   /* kappa[b][cj][ci][t] on triangles of T_{h_n}; t=0 lower, t=1 upper */

#define MLEV_GLUE_PAPER 0  /* Algorithm 4.1 step 2: u~ = u~^j on closed G_j, G_{m+1} problem elsewhere */

#define MLEV_PREC_FP64 0   /* every kernel in FP64 (the plain method) */
#define MLEV_PREC_MIXED 1  /* FP32 multigrid for local/strip solves + FP64 residual refinement */

#define MLEV_MAX_LEVELS 10
#define MLEV_MAX_EIGENPAIRS 8

typedef struct mlev_ctx mlev_ctx;

/* Solver options. Fill with mlev_opts_default() and override fields. */
typedef struct mlev_opts {
  int precision;        /* MLEV_PREC_MIXED or MLEV_PREC_FP64 */
  int vcycles;          /* V-cycles per solve pass of each auxiliary problem (Eq. Aux_Problem) */
  int refine_passes;    /* solve passes; passes after the first start from an FP64 residual */
  int strip_vcycles;    /* V-cycles per pass for the G_{m+1} problem (Eq. G_m+1_Problem) */
  int pre_smooth;       /* red-black Gauss-Seidel sweeps before restriction */
  int post_smooth;      /* sweeps after prolongation */
  int coarse_sweeps;    /* sweeps on the coarsest grid of each multigrid hierarchy */
  int level1_max_iter;  /* iteration cap of the level-1 eigensolver (Algorithm 4.2 step 1) */
  double level1_tol;    /* relative eigen-residual target of the level-1 eigensolver; the
                           correction steps contract its error, so the autotuner may loosen
                           it (mlev_grad_kappa's forward pass uses at most 1e-10) */
  int rr_max_iter;      /* Newton/bisection cap of the Rayleigh-Ritz step */
  int use_graph;        /* 1: capture the launch sequence in a CUDA graph and replay it */
  double omega;         /* over-relaxation of the red-black Gauss-Seidel smoother (1 = plain GS) */
  int check_residuals;  /* 1: measure the final relative residual of every local / G_{m+1} solve */
  int profile;          /* 1: time every launch with CUDA events (no graph); read with mlev_profile_read */
  int fused;            /* 1: fused multigrid kernels (down / up / shared-memory tail); 0: one launch per
                           operation; 2: one launch per operation on the large grids, the shared-memory
                           tail for the small ones (see tail_nodes) */
  int tail_nodes;       /* largest grid (nodes) the in-block tail of a fused V-cycle takes on; 0 = as many
                           levels as fit in shared memory */
  int reg_depths;       /* fused = 2 only: the first reg_depths depths (finest first) run the
                           register-blocked fused down / up legs instead of one launch per operation,
                           where those legs apply (FP32, plain Gauss-Seidel with omega = 1, 1 or 2
                           sweeps, kappa = 1 or per coarse cell on levels >= 3); 0 = none */
  int reserved;
} mlev_opts;

/* Per-solve diagnostics (batch member 0 unless noted). */
typedef struct mlev_report {
  int levels;                          /* n */
  int batch;                           /* B */
  double lambda[MLEV_MAX_LEVELS + 1];  /* lambda_{h_k} for k = 1..n (index k) */
  int level1_iters;                    /* max over the batch */
  double level1_residual;              /* max over the batch */
  int rr_iters[MLEV_MAX_LEVELS + 1];   /* max over the batch */
  double local_residual[MLEV_MAX_LEVELS + 1];  /* max over jobs of ||f - A e|| / ||f|| (check_residuals) */
  double strip_residual[MLEV_MAX_LEVELS + 1];  /* same for the G_{m+1} problem (check_residuals) */
  long long n_fine;                    /* interior nodes of T_{h_n} (unknowns per problem) */
  long long n_local_fine;              /* sum over j of unknowns of Omega_j on T_{h_n} */
  long long n_strip_fine;              /* unknowns of the G_{m+1} problem on T_{h_n} */
  int n_coarse;                        /* interior nodes of T_H */
  int kernel_launches;                 /* launches issued by the last mlev_solve (graph nodes if replayed) */
  int status_flags;                    /* device-side status bits (0 = clean) */
  long long h2d_bytes;                 /* host-to-device bytes copied by this call */
  long long d2h_bytes;                 /* device-to-host bytes copied by this call (outputs only) */
} mlev_report;

/* Per-kernel-family timing of the last solve run with opts.profile = 1. */
typedef struct mlev_kernel_stat {
  char name[32];   /* kernel family, e.g. "mg_smooth" */
  int launches;    /* launches in that solve */
  double ms;       /* summed CUDA-event durations of those launches (events on the solve's stream) */
  double bytes;    /* algorithmic bytes those launches must move (the library's traffic model) */
} mlev_kernel_stat;

/* Fill opts with the defaults of this build. */
void mlev_opts_default(mlev_opts* opts);

/* Create a context bound to CUDA device `device`. *out is NULL on failure.
 * device == -1 creates a planning-only context: every mlev_set_*, mlev_workspace_size
 * and mlev_problem_info works (no GPU needed); mlev_solve* return MLEV_ESTATE. */
int mlev_create(mlev_ctx** out, int device);

/* Destroy a context (NULL is ignored). Does not touch caller-owned device memory. */
void mlev_destroy(mlev_ctx* ctx);

/* Message of the last failing call on ctx ("" if none); valid until the next call. */
const char* mlev_last_error(const mlev_ctx* ctx);

/*
 * Coarse triangulation T_H (Section 2.1; Section 4 "coarsest triangulation"):
 * ncx x ncy cells of side H from (x0, y0); cell_in[cj*ncx + ci] != 0 marks cells of
 * Omega. Each cell is split by its SW-NE diagonal. Requires 2 <= ncx, ncy <= 64.
 */
int mlev_set_domain(mlev_ctx* ctx, int ncx, int ncy, double x0, double y0, double H,
                    const uint8_t* cell_in);

/*
 * Domain decomposition (Section 4, before Algorithm 4.1): cell_owner[cj*ncx+ci] = j
 * in [0, m) for the disjoint D_j (-1 on cells outside Omega); overlap[j] = number
 * of coarse cells by which D_j is enlarged (Chebyshev distance) to Omega_j; delta =
 * inset defining the closed G_j = { x in closure(D_j) : dist_inf(x, dD_j \ dOmega) >= delta },
 * a positive multiple of H/4. Every D_j must be a rectangle of cells (else
 * MLEV_EUNSUPPORTED); the closed G_j must be pairwise disjoint (else MLEV_EINVAL).
 * glue_mode must be MLEV_GLUE_PAPER.
 */
int mlev_set_partition(mlev_ctx* ctx, int m, const int32_t* cell_owner, const int32_t* overlap,
                       double delta, int glue_mode);

/* Number of levels n >= 2 (h_k = H / 2^k, k = 1..n; Section 4.2, Algorithm 4.2). */
int mlev_set_levels(mlev_ctx* ctx, int n);

/*
 * Bilinear forms (Section 2.2, Section 3): a(u,v) = (kappa grad u, grad v),
 * b(u,v) = (u,v), for `batch` independent problems sharing the geometry.
 * kappa layout by kind: ONE -> kappa ignored (may be NULL); PER_COARSE_CELL ->
 * [batch][ncy][ncx]; PER_FINE_ELEM -> [batch][ncy*2^n][ncx*2^n][2]. Values must be
 * positive on cells of Omega. If kappa_on_device != 0 the pointer is a device
 * buffer the caller keeps alive and unchanged-in-layout while solving (it is read
 * at every mlev_solve); otherwise it is copied now (call mlev_set_levels first
 * for PER_FINE_ELEM).
 */
int mlev_set_forms(mlev_ctx* ctx, int batch, int kappa_kind, const double* kappa, int kappa_on_device);

/*
 * Number q of smallest eigenpairs to compute (default 1), 1 <= q <= MLEV_MAX_EIGENPAIRS.
 * Section 4 states the correction step for one simple eigenvalue and says the version for
 * several (and multiple) eigenvalues follows in the same way; Section 6 (Table 1) computes
 * the first five. With q > 1 level 1 gives the q smallest eigenpairs of the pencil on
 * V_{0h_1} (Algorithm 4.2 step 1), every correction step runs steps 1 and 2 of Algorithm 4.1
 * for each pair with its own lambda_i, and step 3 is one Rayleigh-Ritz problem on
 * V_{0H} + span{u~_1, ..., u~_q}; each u_i is b-normalised with b(u_i, W) > 0 for the T_H
 * function W whose nodal value at the coarse node (X, Y) is 1 + frac(0.6180339887498949 k),
 * k = Y (ncx + 1) + X (a positive, irregular weight). Outputs of mlev_solve / mlev_solve_host / mlev_solve_noalloc become
 * lambda [batch][q] (ascending) and u [batch][q][grid]; mlev_report describes pair 1 of
 * member 0. q > 1 needs a coefficient given on the host (kappa_on_device = 0), a coarse grid
 * of at most 16 cells per side, and no gradient (mlev_grad_kappa returns MLEV_EUNSUPPORTED);
 * otherwise MLEV_EUNSUPPORTED at the next solve. Call before mlev_workspace_size.
 */
int mlev_set_eigenpairs(mlev_ctx* ctx, int q);

/* Bytes of device workspace mlev_solve needs for the current setup and opts. */
int mlev_workspace_size(mlev_ctx* ctx, const mlev_opts* opts, size_t* bytes);

/* Unknown counts of the current setup (any pointer may be NULL). */
int mlev_problem_info(mlev_ctx* ctx, long long* n_fine, long long* n_local_fine, long long* n_strip_fine,
                      int* n_coarse);

/*
 * Run Algorithm 4.2 for every batch member on `stream` (a cudaStream_t; NULL =
 * legacy default stream).
 *  workspace  : device buffer of >= mlev_workspace_size() bytes, 256-byte aligned,
 *               owned by the caller. The first solve with a given workspace
 *               uploads the plan tables into it (issue that first call before
 *               any stream capture).
 *  lambda_out : device array [batch] receiving lambda_{h_n}.
 *  u_out      : NULL or device array [batch][(ncy*2^n+1)*(ncx*2^n+1)] receiving
 *               u_{h_n} with b(u,u) = 1 and int u > 0, zero on and outside dOmega.
 *  rep        : NULL or host report; non-NULL makes the call synchronize `stream`.
 * Asynchronous when rep == NULL: errors found on the device then surface in the
 * next call that synchronizes (a non-NULL rep).
 */
int mlev_solve(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
               double* lambda_out, double* u_out, mlev_report* rep);

/*
 * Same as mlev_solve with HOST buffers: copies kappa_host (layout of
 * mlev_set_forms, may be NULL to keep the current coefficients) to the device,
 * solves, and copies lambda (and u if u_host != NULL) back, synchronizing stream.
 * The kappa staging area is part of the workspace (mlev_workspace_size counts it).
 * opts.use_graph applies as in mlev_solve (the plan tables and kappa are copied before
 * the graph launch, the results after it). Host buffers in pinned memory make the copies
 * direct transfers.
 */
int mlev_solve_host(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
                    const double* kappa_host, double* lambda_host, double* u_host, mlev_report* rep);

/*
 * Same computation as mlev_solve, for callers that cannot allocate device memory: for
 * example a plugin inside a host application whose own memory pool must own every
 * device allocation, or a latency-critical loop that may never enter the CUDA
 * allocator (cudaMalloc can block and synchronize the device). No device memory is
 * allocated for data: the workspace is a fixed array of MLEV_NOALLOC_WORKSPACE_BYTES
 * (32 MiB) compiled into the library, which every GPU that loads the library keeps until
 * the process exits. The paper has no counterpart; this is an interface convenience.
 *  - Problems whose mlev_workspace_size exceeds MLEV_NOALLOC_WORKSPACE_BYTES are
 *    rejected with MLEV_ENOMEM and a message giving both sizes.
 *  - The first call on a device looks up the array's device address (a one-time
 *    set-up with that device current); make that first call before any stream capture.
 *    The address is kept for the life of the process, so resetting the device
 *    (cudaDeviceReset) after that first call is not supported.
 *  - A call copies the plan tables (and host kappa) into the array and synchronizes
 *    `stream` only when the array does not already hold this context's tables for its
 *    current setup (first call, another context used the array since, or a mlev_set_*
 *    call changed the setup); otherwise it only enqueues the solve.
 *  - All calls share the one array, so calls whose GPU work overlaps in time (other
 *    streams, other threads or contexts on the same device) race and give wrong results.
 *  - opts.use_graph = 1 and opts.profile = 1 create driver objects on first use, as in
 *    mlev_solve (a private capture stream and a graph executable; CUDA events).
 *  - Outputs and the meaning of every argument are as in mlev_solve.
 */
#define MLEV_NOALLOC_WORKSPACE_BYTES (32u << 20)
int mlev_solve_noalloc(mlev_ctx* ctx, const mlev_opts* opts, void* stream, double* lambda_out, double* u_out,
                       mlev_report* rep);

/*
 * Copy the per-family statistics of the last profiled solve (opts.profile = 1) into
 * out[0 .. min(capacity, families) - 1]; *count receives the number of families.
 * Returns MLEV_ESTATE if no profiled solve has completed on ctx.
 */
int mlev_profile_read(mlev_ctx* ctx, mlev_kernel_stat* out, int capacity, int* count);

/*
 * Derivative of the final eigenvalue lambda_{h_n} of Algorithm 4.2 (with the correction
 * step of Algorithm 4.1) with respect to the coefficient kappa of a(u, v) = int kappa
 * grad u . grad v (Section 2.2), by the adjoint (reverse) method.
 *
 * The map differentiated is the algorithm itself, every local and G_{m+1} solve
 * (Eqs. Aux_Problem, G_m+1_Problem) and both eigenproblems (Algorithm 4.2 step 1,
 * Eq. Eigen_Augment_Problem) taken as exact; the discrete solves use the same
 * multigrid, precision and cycle counts as mlev_solve with the same opts, except that
 * level 1 is solved to a relative residual of at most 1e-10 (opts.level1_tol is capped
 * there, since the level-1 adjoint needs the exact level-1 eigenpair). The call
 * runs the forward solve again (keeping u~_k, lambda_k and the Rayleigh-Ritz
 * coefficients of every level), then the reverse sweep, in which the local solutions
 * e^j of each level are recomputed rather than stored.
 *
 *   dlambda   [batch] device: upstream weights w_b; the result is w_b * dlambda_b/dkappa
 *   layout    MLEV_GRAD_FINE_ELEM: dkappa[b][cj][ci][t] per triangle of T_{h_n}
 *             (t = 0 lower, 1 upper; the derivative with respect to a coefficient given
 *             per finest triangle, whatever kappa_kind is);
 *             MLEV_GRAD_COARSE_CELL: dkappa[b][cj][ci] per T_H cell (a coefficient
 *             constant on each coarse cell)
 *   dkappa    device output, overwritten; zero outside Omega
 *   lambda_out  nullable [batch] device: lambda_{h_n} of the forward pass
 *   rep         nullable host report, as in mlev_solve
 *
 * The workspace must hold mlev_grad_workspace_size bytes (more than mlev_solve's: level
 * checkpoints and adjoint fields). Errors as in mlev_solve; MLEV_ENOCONV also when the
 * level-1 adjoint solve reaches its cap (4 * level1_max_iter iterations). Not captured
 * in a CUDA graph (opts.use_graph is ignored); opts.profile times its launches.
 */
#define MLEV_GRAD_FINE_ELEM 0
#define MLEV_GRAD_COARSE_CELL 1
int mlev_grad_workspace_size(mlev_ctx* ctx, const mlev_opts* opts, size_t* bytes);
int mlev_grad_kappa(mlev_ctx* ctx, const mlev_opts* opts, void* workspace, size_t ws_bytes, void* stream,
                    const double* dlambda, int layout, double* dkappa, double* lambda_out, mlev_report* rep);

#ifdef __cplusplus
}
#endif

#endif /* MLEV_H */
