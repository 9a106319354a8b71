/*
 * ipm.h -- C ABI of the GB300 (sm_103a) primal-dual interior point method for convex QPs
 *
 *     min 0.5 x^T H x + c^T x   s.t.   A x <= b,   l <= x <= u            (1)
 *
 * This is the paper's QP (Section 3.1, eq:qp) with the variable bounds kept apart from A, as
 * Section 4 does before eq:2x2_reduced; the paper's two-sided rows l_A <= A x <= u_A are
 * taken as its stack B = [A; -A] of one-sided rows (ipm_qp.bl).  Each Newton
 * step (eq:newton_system) is reduced to the normal-equations system
 *
 *     (H + A^T Theta A + Sigma) dx = r,  Theta = diag(y / s),  Sigma = diag(z_l/t_l + z_u/t_u)
 *
 * (the Schur complement of eq:2x2_reduced) and solved matrix-free by preconditioned
 * conjugate gradients (Section 4.1; the linear solve of Algorithm 1), on the device.
 *
 * Conventions for every entry point:
 *   - Return value: an ipm_status code; functions never abort and never print.
 *     ipm_last_error(h) gives a one-line description of the last failure on a handle.
 *   - Pointers are host or device memory as the `mem` argument says (IPM_MEM_HOST /
 *     IPM_MEM_DEVICE).  Device pointers must be readable from the current CUDA device.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  The library orders its
 *     work after everything already queued on `stream` and makes `stream` wait for it before
 *     returning; calls that return data to host memory synchronise before returning.
 *   - The library owns every device buffer it allocates (one arena per handle, allocated by
 *     ipm_set_qp and freed by ipm_set_qp / ipm_destroy).  Inputs are deep-copied.
 *   - Vectors are dense float64 arrays; sparse matrices are CSR with int64 row pointers and
 *     int32 column indices (indices within a row in any order, no duplicates).
 *   - A handle is not thread safe; different handles may be used concurrently.
 */
#ifndef IPM_H_
#define IPM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
enum ipm_status {
  IPM_OK = 0,
  IPM_ERR_ARG = 1,               /* invalid argument (sizes, NULL, non-finite data, bad layout) */
  IPM_ERR_OOM = 2,               /* device allocation failed or exceeds options.mem_budget      */
  IPM_MAX_ITER = 3,              /* options.max_ipm iterations without reaching tol_kkt         */
  IPM_CG_STALL = 4,              /* PCG hit options.max_cg with its residual above 1e-2 of the  */
                                 /* right-hand side in two consecutive Newton steps (the solve */
                                 /* stops there)                                               */
  IPM_NUMERICAL = 5,             /* NaN/Inf in an iterate, PCG breakdown or step length -> 0    */
  IPM_INFEASIBLE_SUSPECTED = 6,  /* the multipliers diverge along a Farkas certificate of primal */
                                 /* infeasibility (y, z >= 0, A^T y - z_l + z_u ~ 0,            */
                                 /* b^T y - l^T z_l + u^T z_u < 0 after scaling)               */
  IPM_ERR_TIMEOUT = 7,           /* host wall-clock limit options.timeout_ms exceeded: the     */
                                 /* solve keeps running on the device; collect it with         */
                                 /* ipm_solve_wait (ipm_solve_query polls) before the handle's */
                                 /* next call, which is refused with IPM_ERR_STATE until then  */
  IPM_ERR_CUDA = 8,              /* a CUDA runtime call failed (see ipm_last_error)             */
  IPM_ERR_STATE = 9,             /* call out of order (e.g. ipm_solve before ipm_set_qp)        */
  IPM_ERR_TOO_LARGE = 10,        /* size beyond the fixed scratch of ipm_apply_operator_static  */
  IPM_BUSY = 11                  /* ipm_solve_query: the solve is still running                 */
};

enum ipm_mem_space { IPM_MEM_HOST = 0, IPM_MEM_DEVICE = 1 };

/* Preconditioner of the PCG solve (Section 4.1.2 computes the Jacobi diagonal).
 *  JACOBI    : M = diag(H + A^T Theta A + Sigma), the paper's choice.
 *  BLOCK32   : M = the 32 x 32 diagonal blocks of H + A^T Theta A + Sigma (blocks of consecutive
 *              variables), each Cholesky-factored on the device every IPM iteration; the part of
 *              the blocks that does not change with the iterate is formed once per QP.  Needs
 *              the columns of every row of F and A in increasing order and F64 storage
 *              (IPM_ERR_ARG otherwise).
 *  JACOBI_LR : Jacobi on the rows whose theta is moderate, plus an exact low-rank correction
 *              (Woodbury) for the "stiff" rows whose theta_i sum_j a_ij^2 / M0_j > stiff_gamma;
 *              keeps PCG iteration counts bounded as mu -> 0 (default).
 *  DENSE     : the whole matrix, formed and Cholesky-factored on the device (one diagonal
 *              block of size n); for n <= dense_max_n and FP64 storage.                      */
enum ipm_precond { IPM_PRECOND_JACOBI = 0, IPM_PRECOND_JACOBI_LR = 1, IPM_PRECOND_DENSE = 2,
                   IPM_PRECOND_AUTO = 3, IPM_PRECOND_BLOCK32 = 4 };

/* Storage of the matrix values inside PCG.  F64 (default): the FP64 operator throughout.
 * F32 / BF16 / FP8_E4M3: a second copy of the values of R = [F; A] and R^T in that type with
 * one FP32 scale per row, an FP32-accumulating operator inside PCG, and FP64 iterative
 * refinement of every Newton step against the FP64 operator (residuals and reductions stay
 * FP64).  Not part of the paper, which is FP64 throughout. */
/* The linear system PCG solves for each Newton step (Section 4): the condensed (Schur
 * complement) form (H + A^T Theta A + Sigma) dx = r, or the paper's doubly augmented form
 * eq:2x2_augmented in (dx, dy) with its Jacobi preconditioner. */
enum ipm_system { IPM_SYSTEM_CONDENSED = 0, IPM_SYSTEM_AUGMENTED = 1 };

enum ipm_storage { IPM_STORAGE_F64 = 0, IPM_STORAGE_F32 = 1, IPM_STORAGE_BF16 = 2, IPM_STORAGE_FP8_E4M3 = 3 };

/* Arithmetic of the PCG operator with F64 storage (not part of the paper, which uses FP64).
 *  F64  : float64 multiply-adds (GB300 issues two per SM per clock, which bounds the passes).
 *  MIXED: half of every lane's products as float64 multiply-adds, half in double-float (as
 *         DF32), so the float64 and float32 pipes work at once; each entry is still read once.
 *         Keeps both copies of R and R^T; the same range condition as DF32.  Rows as CSR.
 *  DF32 : double-float: every value of R, R^T and of the vectors the operator reads is carried
 *         as a (hi, lo) pair of float32 (48 significant bits, the same 8 bytes), products and
 *         sums by error-free transformations on the float32 pipe; row sums within about 1e-13
 *         of sum |a x|.  Residuals, reductions and the rest of the iteration stay float64.
 *         Needs the non-zero values of R within [2^-90, 2^90]; otherwise ipm_set_qp keeps F64
 *         (ipm_info.op_arith tells which ran).  An extra copy of R and R^T (8 bytes per entry
 *         each) is stored. */
enum ipm_arith { IPM_ARITH_F64 = 0, IPM_ARITH_DF32 = 1, IPM_ARITH_MIXED = 2 };

/* Format of R's rows in the PCG rows pass.  CSR: one int32 column index per entry.  RUNS: the
 * maximal stretches of consecutive entries with consecutive columns (a dose row's contiguous
 * spot bands), cut into pieces of at most 32 entries with one 8-byte descriptor each, so no
 * per-entry index is read.  AUTO: RUNS for the reduced storages when R has at least 8 entries
 * per run on average (the row order is the caller's), CSR otherwise (with float64 or
 * double-float arithmetic the CSR pass measured as fast or faster on the RT workload). */
enum ipm_rows_format { IPM_ROWS_AUTO = 0, IPM_ROWS_CSR = 1, IPM_ROWS_RUNS = 2 };

/* ipm_solve flags. */
enum ipm_solve_flags { IPM_COLD = 0, IPM_WARM = 1 };

typedef struct ipm_options {
  double tol_kkt;        /* stop when the relative KKT residual <= tol_kkt (default 1e-6)      */
  double tau;            /* fraction-to-boundary factor of the step lengths (0.995)            */
  int max_ipm;           /* IPM iteration limit (200)                                          */
  int max_cg;            /* PCG iteration limit per Newton step (2000)                         */
  double cg_eta_max;     /* PCG relative tolerance eta = clamp(cg_eta_factor * relKKT, ...)    */
  double cg_eta_min;     /*   ... between cg_eta_min (1e-10) and cg_eta_max (1e-2)            */
  double cg_eta_factor;  /*   (0.3)                                                            */
  int precond;           /* enum ipm_precond (IPM_PRECOND_AUTO: DENSE if n <= 1024 and storage */
                         /* is F64, else JACOBI_LR); DENSE needs storage F64 (IPM_ERR_ARG)     */
  double stiff_gamma;    /* JACOBI_LR threshold (1.0)                                          */
  int stiff_max;         /* JACOBI_LR: at most this many stiff rows (256, <= 1024)             */
  int dense_max_n;       /* DENSE allowed up to this n (2048, the maximum)                      */
  double timeout_ms;     /* host wall-clock limit per ipm_solve, 0 = none                       */
  double mem_budget;     /* bytes of device memory a handle may allocate, 0 = unlimited        */
  int equal_steps;       /* 1: alpha_p = alpha_d = min of both (default 0: separate, Alg. 1)   */
  int autotune;          /* 1: ipm_set_qp times the operator kernels for 4/8/16/32 lanes per   */
                         /* row on the loaded matrices and keeps the fastest (kept per matrix  */
                         /* signature for the process).  0 (default): lanes from the average   */
                         /* row length, so results are bitwise reproducible across processes  */
  int use_graphs;        /* 1: the whole solve as one CUDA graph, the IPM and PCG loops as      */
                         /* nested conditional-while nodes (default); 0: the same kernels      */
                         /* launched one by one from host loops (for per-kernel profilers)     */
  int storage;           /* enum ipm_storage (default IPM_STORAGE_F64)                          */
  int refine_max;        /* reduced precision: at most this many refinement passes per step (8) */
  double refine_eta;     /* reduced precision: the factor by which the residual falls between  */
                         /* two FP64 residual evaluations: refine_mode 1 replaces the PCG      */
                         /* residual then, refine_mode 0 ends a refinement pass there; 0      */
                         /* (default) = 0.01 with replacement, 0.1 with passes                 */
  int lanes_rows;        /* lanes per row of the kernels over R (4, 8, 16, 32; 0 = automatic)   */
  int lanes_cols;        /* lanes per row of the kernels over R^T (same; overrides autotune)    */
  double warm_rho;       /* IPM_WARM: complementarity pairs raised to >= warm_rho * mu0 of the  */
                         /* last cold start (1e-5); 0 keeps the previous point as it is        */
  int u_cap;             /* columns reserved for the low-rank Hessian term U diag(u_w) U^T      */
                         /* (0: as many as the loaded QP has); ipm_set_lowrank may use up to   */
                         /* max(u_cap, u_cols of the QP)                                       */
  int ingest_host;       /* 1: ipm_set_qp builds R^T on the host (multi-threaded) instead of    */
                         /* on the device; both give the same bytes (0)                        */
  int system;            /* enum ipm_system (IPM_SYSTEM_CONDENSED); AUGMENTED needs storage F64 */
                         /* and precond JACOBI or AUTO (it always runs the Jacobi PCG)         */
  int lanes_at;          /* lanes per row of the kernels over the stored A^T alone (right-hand  */
                         /* side with the Jacobi diagonal, Jacobi diagonal): 4, 8, 16, 32; 0 =  */
                         /* from its average row length                                        */
  int op_arith;          /* enum ipm_arith: PCG operator arithmetic with F64 storage (F64)      */
  int rows_format;       /* enum ipm_rows_format of the PCG rows pass (AUTO)                    */
  int rows_stage;        /* 1: with RUNS and double-float or reduced storage, the rows pass     */
                         /* streams R's values, piece descriptors and row pointers into shared  */
                         /* memory by bulk copies (TMA), one three-stage pipeline per SM;       */
                         /* 0 (default): it reads global memory (measured faster on the RT     */
                         /* workload)                                                           */
  double wait_limit_ms;  /* limit of every device-side wait (1000): when one runs out the solve */
                         /* stops with IPM_ERR_TIMEOUT (the iterate is then not meaningful)     */
  int wait_test;         /* test of the device watchdog (0): 1 arms the first staged tile's     */
                         /* barrier for 16 bytes more than is copied, so its wait runs out      */
                         /* (needs rows_stage = 1)                                              */
  int cols_format;       /* reduced storages: 0 (default) the column pass reads R^T's int32     */
                         /* row indices (CSR); 1: as 16-bit gaps (a base row per column, filler */
                         /* slots for wider gaps, columns padded to 8 slots: 2 index bytes an   */
                         /* entry instead of 4, measured slower on the RT workload: the decode  */
                         /* costs more than the bytes it saves)                                 */
  int refine_mode;       /* reduced storages: 1 one PCG per Newton step whose recursive         */
                         /* residual is replaced by the FP64 residual rhs - K dx each time it   */
                         /* falls by refine_eta (the search direction is kept), ending when a   */
                         /* replaced residual meets the step's tolerance; 0 refinement passes,  */
                         /* each a PCG restarted on the current FP64 residual; 2 (default) = 1  */
                         /* for F32 and BF16, 0 for FP8 (whose coarse values make the kept      */
                         /* direction drift: 688 against 240 PCG iterations on an RT QP)        */
} ipm_options;

/* Fills *opt with the defaults listed above. */
void ipm_default_options(ipm_options* opt);

/* The QP (1).  H = diag(h0) + H_dense + F^T diag(f_w) F + U diag(u_w) U^T, each term optional
 * (the last is the quasi-Newton Hessian of Section 3.3, eq:bfgs_hessian, applied matrix-free).
 * Constraint rows come either from F (a_rows: row indices into F, the dose-matrix case where
 * A is a subset of D's rows) or from a CSR matrix A; not both.  m = 0 is allowed (bounds only).
 *
 * Two-sided rows bl <= A x <= b (the paper's l_A <= A x <= u_A, Section 4 before
 * eq:2x2_reduced) are given by bl.  The solver stores them as the paper's stack B = [A; -A]:
 * the "stored rows" are first A_k x <= b_k for every k with finite b_k, in order, then
 * -A_k x <= -bl_k for every k with finite bl_k, in order (a_rows rows with a lower side get a
 * negated copy in the matrix store).  ipm_get_xyz reports per caller row k the signed
 * multiplier y_k = y_upper - y_lower and the slack b_k - A_k x (A_k x - bl_k where b_k is
 * +inf; +inf for a row with neither side); the step-level entry points work on the stored
 * rows, whose count ipm_get_sizes gives.  Without bl the stored rows are the caller's rows. */
typedef struct ipm_qp {
  int64_t n;                 /* variables, >= 1                                            */
  int64_t m;                 /* linear inequality rows, >= 0                               */
  int mem;                   /* ipm_mem_space of every pointer in this struct              */
  const double* c;           /* n, linear cost (the paper's p)                             */
  const double* b;           /* m, right-hand side of A x <= b (NULL iff m == 0)           */
  const double* l;           /* n, lower bounds, -inf allowed; NULL = all -inf             */
  const double* u;           /* n, upper bounds, +inf allowed; NULL = all +inf; l < u      */
  const double* h0;          /* n, diagonal part of H (>= 0); NULL = 0                     */
  const double* H_dense;     /* n*n row-major symmetric block of H; NULL = none            */
  int64_t f_rows;            /* rows r of the factor F (0 = no factor term)                */
  const int64_t* F_indptr;   /* r+1                                                        */
  const int32_t* F_indices;  /* nnz(F), column indices in [0, n)                           */
  const double* F_data;      /* nnz(F)                                                     */
  const double* f_w;         /* r, weights >= 0                                            */
  const int32_t* a_rows;     /* m row indices into F (or NULL)                             */
  const int64_t* A_indptr;   /* m+1 (or NULL)                                              */
  const int32_t* A_indices;  /* nnz(A)                                                     */
  const double* A_data;      /* nnz(A)                                                     */
  int64_t u_cols;            /* columns of U in the low-rank term U diag(u_w) U^T of H     */
                             /* (eq:bfgs_hessian; 0 = none, at most 65536)                  */
  const double* U;           /* n x u_cols, row-major: variable j's u_cols values adjacent */
  const double* u_w;         /* u_cols weights; may be negative (BFGS), H must stay PSD    */
  const double* bl;          /* m, lower sides of the rows (-inf = none); NULL = one-sided */
                             /* rows A x <= b.  With bl, b may hold +inf; bl < b           */
} ipm_qp;

typedef struct ipm_info {
  int status;                /* ipm_status of the last ipm_solve                           */
  int ipm_iters;             /* IPM iterations taken                                       */
  int64_t cg_iters;          /* PCG iterations summed over all Newton steps                */
  int max_cg_step;           /* most PCG iterations in one Newton step                     */
  int max_stiff_rows;        /* most stiff rows in the JACOBI_LR correction                */
  int precond;               /* preconditioner actually used                               */
  double rel_kkt;            /* relative KKT residual of the returned point                */
  double primal_res;         /* its primal, dual and gap parts                             */
  double dual_res;
  double gap_res;
  double primal_obj;         /* 0.5 x^T H x + c^T x                                        */
  double dual_obj;
  double mu;                 /* final barrier parameter                                    */
  double solve_ms;           /* wall time of the last ipm_solve                            */
  int64_t kernel_launches;   /* kernels of this library launched by the last ipm_solve     */
  int lanes_rows;            /* lanes per row of the kernels over R and over R^T (chosen   */
  int lanes_cols;            /* by the autotuner at ipm_set_qp)                            */
  int64_t refine_passes;     /* FP64 refinement passes summed over the Newton steps        */
  int64_t fallback_steps;    /* Newton steps finished by FP64 PCG after refinement stalled */
  int op_arith;              /* enum ipm_arith the F64-storage PCG operator ran in         */
  int rows_runs;             /* 1 if the PCG rows pass read R's rows as runs               */
  int cols_gap;              /* 1 if the reduced-precision column pass reads 16-bit gaps   */
} ipm_info;

/* Per-step result of ipm_newton_direction. */
typedef struct ipm_cg_report {
  int iters;                 /* PCG iterations                                             */
  int converged;             /* 1 if ||r|| <= eta ||rhs|| was met                          */
  int stiff_rows;            /* rows in the low-rank correction                            */
  double rel_res;            /* final ||r|| / ||rhs||                                      */
  double eta;                /* tolerance used                                             */
} ipm_cg_report;

typedef struct ipm_handle ipm_handle;

/* Creates a solver handle on the current CUDA device.  opt may be NULL (defaults).
 * Allocates no device memory.  Errors: IPM_ERR_ARG (out == NULL or invalid options). */
int ipm_create(const ipm_options* opt, ipm_handle** out);

/* Loads the QP (1) (deep copy into solver-owned device memory) and builds, on the device, the
 * stored transposes R^T and A^T used by the matrix-free operator (rows ascending within each
 * column, so every product is a deterministic gather), the diagonal of H (computed once, as
 * in Section 4.1.2) and the workspace.  Replaces any earlier QP on the handle.
 * Errors: IPM_ERR_ARG (inconsistent sizes, index out of range, non-finite data, l >= u,
 * bl >= b, both or neither of a_rows/A given with m > 0), IPM_ERR_OOM, IPM_ERR_CUDA. */
int ipm_set_qp(ipm_handle* h, const ipm_qp* qp, void* stream);

/* Sizes of the loaded QP: n, the caller's rows m and the stored rows m_rows (equal to m
 * unless bl was given; see ipm_qp).  Any output may be NULL.  Errors: IPM_ERR_STATE (no QP). */
int ipm_get_sizes(const ipm_handle* h, int64_t* n, int64_t* m, int64_t* m_rows);

/* Runs Algorithm 1 on the device from the start point (IPM_COLD) or from the last iterate
 * (IPM_WARM: the previous solution, or one given by ipm_set_iterate).  Returns the solve
 * status: IPM_OK when rel KKT <= tol_kkt; IPM_MAX_ITER, IPM_INFEASIBLE_SUSPECTED,
 * IPM_NUMERICAL or IPM_ERR_TIMEOUT otherwise (the iterate is kept either way). */
int ipm_solve(ipm_handle* h, void* stream, int flags);

/* Asynchronous form of ipm_solve: queues the whole solve (one CUDA graph launch) behind the
 * work already on `stream` and returns at once; `stream` is made to wait for the solve.  At
 * most one solve per handle is in flight.  Needs use_graphs = 1. */
int ipm_solve_async(ipm_handle* h, void* stream, int flags);

/* Waits for the solve started by ipm_solve_async (bounded by options.timeout_ms), returns its
 * status and fills *info if non-NULL. */
int ipm_solve_wait(ipm_handle* h, ipm_info* info);

/* IPM_BUSY while the solve started by ipm_solve_async is running, IPM_OK when it has finished
 * (or none is in flight); does not block. */
int ipm_solve_query(ipm_handle* h);

/* Batched solve (the uneven many-QP workload): every handle's whole solve captured as one
 * branch of a single CUDA graph, so one launch runs all of them concurrently on the device;
 * each handle keeps its own data, schedule and scalars.  ipm_batch_create captures the graph
 * (after ipm_set_qp on every handle); ipm_batch_solve launches it behind `stream`, waits, and
 * stores each handle's result (read it with ipm_get_xyz); statuses (count ints) may be NULL.
 * A batch is invalidated by ipm_set_qp, ipm_share_qp, ipm_set_lowrank or ipm_destroy on any of
 * its handles: after the first three ipm_batch_solve returns IPM_ERR_STATE without launching
 * anything (each handle carries a generation count that the batch checks); after
 * ipm_destroy of a member the batch must not be used at all. */
typedef struct ipm_batch ipm_batch;
int ipm_batch_create(ipm_handle* const* handles, int count, int flags, ipm_batch** out);
int ipm_batch_solve(ipm_batch* b, void* stream, int* statuses);
int ipm_batch_destroy(ipm_batch* b);

/* Fills *info: the last solve's results (zero before the first solve) and the operator
 * configuration chosen at ipm_set_qp (op_arith, rows_runs, lanes_rows, lanes_cols).
 * Errors: IPM_ERR_ARG (NULL), IPM_ERR_STATE (no QP loaded). */
int ipm_get_info(ipm_handle* h, ipm_info* info);

/* Copies the current iterate to caller memory (any pointer may be NULL to skip it):
 * x, z_l, z_u (n), y, s (m: the caller's rows; for two-sided rows the signed multiplier and
 * slack described at ipm_qp); fills *info if non-NULL. */
int ipm_get_xyz(ipm_handle* h, double* x, double* y, double* z_l, double* z_u, double* s,
                ipm_info* info, int mem, void* stream);

/* Replaces the factor weights f_w (f_rows values) and/or the linear cost c (n values) of the
 * loaded QP (NULL keeps the current one) without re-ingesting any matrix; diag(H) is updated.
 * For SQP-like chains of related QPs (Section 3.2: each SQP iteration changes the QP's
 * Hessian and cost, the constraints stay), followed by ipm_solve(..., IPM_WARM). */
int ipm_update_costs(ipm_handle* h, const double* f_w, const double* c, int mem, void* stream);

/* Replaces the low-rank Hessian term U diag(u_w) U^T of the loaded QP (Section 3.3: each SQP
 * iteration appends two BFGS columns; u_cols = 0 drops the term, as the paper's reset after
 * spot filtering does).  U is n x u_cols row-major, u_cols at most the capacity reserved at
 * ipm_set_qp (IPM_ERR_TOO_LARGE otherwise).  diag(H) is recomputed; the handle's captured
 * solve graphs are rebuilt at the next solve (a batch that contains the handle must be
 * created again).  The iterate is kept, so IPM_WARM continues from the last solution. */
int ipm_set_lowrank(ipm_handle* h, int64_t u_cols, const double* U, const double* u_w, int mem, void* stream);

/* Loads into h the QP already loaded on src without copying its matrices: h references src's
 * device copy of R, R^T (and its reduced-precision copies and dense H block), which stays
 * alive until the last handle that uses it is destroyed or reloaded, and allocates only its
 * own state (problem vectors, iterate, PCG and preconditioner work space; sizes in
 * ipm_device_bytes).  c, f_w, b, l, u start as copies of src's and may then be changed with
 * ipm_update_costs on either handle independently.  Both handles may solve at the same time.
 * No counterpart in the paper: it lets several solves of one plan run concurrently (serving).
 * Errors: IPM_ERR_STATE (src has no QP, or h has a solve in flight), IPM_ERR_ARG (different
 * devices, or h's storage option differs from src's), IPM_ERR_OOM. */
int ipm_share_qp(ipm_handle* h, ipm_handle* src, void* stream);

/* Device bytes held by the handle: the matrix store (possibly shared; matrix_refs = number of
 * handles referencing it) and the handle's own state.  Any output may be NULL. */
int ipm_device_bytes(const ipm_handle* h, int64_t* matrix_bytes, int64_t* state_bytes, int* matrix_refs);

/* Sizes in bytes of the interface structs as this library was compiled (ipm_options,
 * ipm_qp, ipm_info, ipm_cg_report), for bindings to check their own layouts.  Any pointer
 * may be NULL.  No counterpart in the paper. */
int ipm_abi_sizes(int64_t* options, int64_t* qp, int64_t* info, int64_t* cg_report);

/* Forgets the lane widths the autotuner (options.autotune) chose per matrix signature in this
 * process, so that the next ipm_set_qp with autotune = 1 times the kernels again (a cold start,
 * as in a fresh process).  Handles already loaded keep their widths.  No counterpart in the
 * paper. */
int ipm_autotune_reset(void);

/* Frees the handle and its device memory.  NULL-safe. */
int ipm_destroy(ipm_handle* h);

/* Static description of a status code. */
const char* ipm_status_str(int status);

/* Last error message recorded on h ("" if none). */
const char* ipm_last_error(const ipm_handle* h);

/* ---- Step-level entry points: one step of Algorithm 1 each, on the current iterate ---- */

/* Sets the iterate (x, s, y, z_l, z_u) and mu; used for warm starts and to evaluate single
 * steps.  x must lie strictly inside finite bounds; s, y, z_l, z_u > 0 where they apply.
 * Here and in the step-level calls below, s, y, r_p, r_s, ds and dy have one value per
 * stored row (ipm_get_sizes' m_rows). */
int ipm_set_iterate(ipm_handle* h, const double* x, const double* s, const double* y,
                    const double* z_l, const double* z_u, double mu, int mem, void* stream);

/* Perturbed KKT residuals at the current iterate (Section 3.1, eq:perturbed_KKT, restated for
 * (1)): r_d = Hx + c + A^T y - z_l + z_u (n), r_p = Ax + s - b (m), r_s = s o y - mu (m),
 * r_l = t_l o z_l - mu, r_u = t_u o z_u - mu (n; 0 at infinite bounds).  NULL skips a vector.
 * kkt (optional, 4 doubles) receives the relative KKT residual and its primal, dual and gap
 * parts as defined for ipm_info. */
int ipm_residuals(ipm_handle* h, double* r_d, double* r_p, double* r_s, double* r_l, double* r_u,
                  double* kkt, int mem, void* stream);

/* q = (H + A^T Theta A + Sigma) p at the current iterate: one matrix-free operator apply of
 * the PCG (Section 4.1.1; the condensed counterpart of the operator of Listing 1).  p, q: n.
 * With options.system = IPM_SYSTEM_AUGMENTED it applies that system's (1,1) block,
 * H + Sigma + 2 A^T Theta A. */
int ipm_apply_kkt(ipm_handle* h, const double* p, double* q, int mem, void* stream);

/* Jacobi diagonal diag(H + A^T Theta A + Sigma) at the current iterate (Section 4.1.2). */
int ipm_precond_diag(ipm_handle* h, double* diag, int mem, void* stream);

/* Newton direction at the current iterate and mu (Algorithm 1: the PCG solve, then the
 * recovery of the full direction): dx, dz_l, dz_u (n), ds, dy (m).  eta <= 0 selects the solver's own rule;
 * otherwise PCG stops at ||r|| <= eta ||rhs||.  rep may be NULL. */
int ipm_newton_direction(ipm_handle* h, double eta, double* dx, double* ds, double* dy,
                         double* dz_l, double* dz_u, ipm_cg_report* rep, int mem, void* stream);

/* Fraction-to-boundary step lengths for the given direction at the current iterate (Section
 * 3.1 line search; Algorithm 1's step lengths):
 *   alpha_p = min(1, tau max{a: s + a ds >= 0, t_l + a dx >= 0, t_u - a dx >= 0}),
 *   alpha_d = min(1, tau max{a: y + a dy >= 0, z_l + a dz_l >= 0, z_u + a dz_u >= 0}). */
int ipm_step_lengths(ipm_handle* h, const double* dx, const double* ds, const double* dy,
                     const double* dz_l, const double* dz_u, double tau, double* alpha_p,
                     double* alpha_d, int mem, void* stream);

/* Per-iteration trace of the last ipm_solve (metrics only): row k holds
 *   {k+1, mu, rel_kkt, primal, dual, gap, alpha_p, alpha_d, pcg_iters, pcg_converged,
 *    stiff_rows, pcg_rel_residual, eta, refine_passes}  (IPM_TRACE_COLS doubles).
 * Copies at most max_rows rows into buf (host memory) and returns the number of rows the last
 * solve recorded (so buf == NULL queries the count). */
#define IPM_TRACE_COLS 14
int ipm_get_trace(const ipm_handle* h, double* buf, int max_rows);

/* Measurement hook for the PCG operator (Section 4.1.1's matvec, the loop that Section 5.1.2
 * finds to take most of the run time): at the current iterate, launches the row-gather kernel
 * over R and the gather over the stored transpose `reps` times each on the library's stream,
 * timed with CUDA events around every launch: the FP64 kernels for IPM_STORAGE_F64, else the
 * reduced-precision kernels of the handle's storage.  Returns the mean milliseconds per launch
 * and the algorithmic bytes and flops of one launch of each kernel (bytes: every matrix value,
 * index and row pointer once at its stored width, every dense vector once; flops: 2 per
 * stored non-zero).
 * Any output pointer may be NULL. */
int ipm_profile_operator(ipm_handle* h, int reps, double* ms_rows, double* ms_cols, double* bytes_rows,
                         double* bytes_cols, double* flops_rows, double* flops_cols);

/* ---- Allocation-free operator apply (the paper has no counterpart) ----
 * For callers that cannot call cudaMalloc (an application that owns and budgets all device
 * memory itself, a custom allocator that must not recurse into the CUDA allocator, a hook
 * that may not allocate): computes, with no allocation of any kind,
 *     q = R^T diag(omega) (R p) + dg o p
 * -- the condensed PCG operator when R = [F; A], omega = f_w (+ theta on constraint rows) and
 * dg = h0 + sigma -- from caller-owned device arrays: R (nR x n CSR), its transpose RT
 * (n x nR CSR), omega (nR), dg, p and q (n).  The intermediate R p lives in a file-scope
 * device array of IPM_STATIC_SCRATCH_ROWS doubles (2 MiB, held by every GPU that loads the
 * library until the process exits); nR > IPM_STATIC_SCRATCH_ROWS returns IPM_ERR_TOO_LARGE
 * before any work.  The first call on a device looks up the array's device address (with
 * that device current); make that first call before any stream capture.  All calls share
 * the array: calls that overlap on the GPU race, so serialise them.  Work is queued on
 * `stream` (device pointers only).  IPM_ERR_ARG for n < 1, nR < 0 or any NULL pointer (R's three
 * arrays and omega may be NULL only when nR = 0), checked before the size limit, so no call
 * with a NULL pointer launches anything. */
#define IPM_STATIC_SCRATCH_ROWS 262144
int ipm_apply_operator_static(int64_t n, int64_t nR, const int64_t* R_indptr, const int32_t* R_indices,
                              const double* R_data, const int64_t* RT_indptr, const int32_t* RT_indices,
                              const double* RT_data, const double* omega, const double* dg,
                              const double* p, double* q, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* IPM_H_ */
