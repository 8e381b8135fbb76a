/*
 * molt.h - C ABI of the GB300 (sm_103a) MOL^T Cahn-Hilliard library.
 *
 * The library implements the hot path of arXiv 1611.04214 (Causley, Cho, Christlieb,
 * "Method of lines transpose: energy gradient flows using direct operator inversion for
 * phase field models"): the O(N) inversion of the 1D modified Helmholtz operator
 * L = I - c d_xx by fast convolution (Sec. 3.2), applied line by line in x and y
 * (Sec. 5), inside the lagged fixed-point stage solve of the Cahn-Hilliard equation
 * u_t = -Lap(eps^2 Lap u - f(u)), f(u) = u^3 - u (Eq. CahnHilliard), stepped by BE,
 * BDF2, SDIRK2, SDIRK3 or SDC2 (Sec. 3-4).
 *
 * Conventions for every entry point:
 *  - C linkage; every call returns a molt_status (0 = MOLT_OK, negative = error) and never
 *    throws.  After an error, molt_last_error(solver) returns a message (static lifetime
 *    until the next call on that solver).
 *  - Handles are opaque and owned by the library; create/destroy pairs free everything.
 *  - Field buffers passed as "device" pointers are caller-owned device memory of nx*ny
 *    elements, row-major [ny][nx] with x contiguous (1D problems: ny = 1), of the
 *    solver's precision (float for MOLT_FP32, double for MOLT_FP64).  Device pointers must
 *    be aligned to the element size.  "host" pointers are caller-owned host memory of the
 *    same layout (pinned or pageable).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *    work of a call is ordered on that stream; calls that return a number read it back and
 *    synchronize that stream.
 *  - One solver per stream at a time: a solver owns device workspace and time history and
 *    is not safe for concurrent calls.
 *  - Grid convention: a periodic line of n stored nodes has h = L/n (node n is node 0); a
 *    Neumann or Dirichlet line of n stored nodes has both walls as nodes and h = L/(n-1).
 *  - Dirichlet lines hold u = -1 on the walls (v = u + 1 = 0 per inversion, the wall value
 *    compatible with Remark Laplacian).
 */
#ifndef MOLT_H
#define MOLT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MOLT_OK = 0,
    MOLT_ERR_ARG = -1,            /* bad size, parameter or pointer */
    MOLT_ERR_NOT_CONVERGED = -2,  /* a stage hit max_iter; the field holds the last iterate */
    MOLT_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    MOLT_ERR_OOM = -4,            /* device workspace could not be allocated */
    MOLT_ERR_UNSUPPORTED = -5     /* valid request this build does not implement */
} molt_status;

typedef enum { MOLT_BC_PERIODIC = 0, MOLT_BC_NEUMANN = 1, MOLT_BC_DIRICHLET = 2 } molt_bc;
typedef enum { MOLT_FP32 = 0, MOLT_FP64 = 1 } molt_precision;
typedef enum {
    MOLT_BE = 0,      /* Eq. CH_BE: one stage, tau = dt */
    MOLT_BDF2 = 1,    /* Eq. BDF2: tau = 2dt/3; first step (and after a dt change) is BE */
    MOLT_SDIRK2 = 2,  /* Sec. 4.2: two stages, eta = 1 - sqrt(2)/2 */
    MOLT_SDIRK3 = 3,  /* Sec. 4.4: Alexander's three-stage method, eta = 0.43587 */
    MOLT_SDC2 = 4,    /* Sec. 4.3 Eq. SDC_fixed: BE level [0] + trapezoid level [1] */
    MOLT_BDF3 = 5     /* Eq. BDF3: tau = 6dt/11; its two starting steps (and two after a dt change)
                         are SDIRK2 steps (Sec. 4.4) */
} molt_scheme;

typedef struct molt_grid molt_grid;
typedef struct molt_solver molt_solver;

/* Solver parameters (Sec. 3-4, Eq. parameters). */
typedef struct {
    double eps;        /* interface width epsilon > 0 */
    int quad_order;    /* spatial quadrature order M in {2, 4, 6} (Sec. 3.2) */
    int precision;     /* molt_precision of fields and sweeps */
    double tol;        /* fixed-point tolerance on ||v^{k+1} - v^k||_inf (Sec. 4.4) */
    int max_iter;      /* fixed-point iteration cap per stage (N_maxit, Sec. 6) */
} molt_params;

/* Per-step report. */
typedef struct {
    int status;          /* MOLT_OK or MOLT_ERR_NOT_CONVERGED */
    int stages;          /* stage solves run by this step */
    int iters[4];        /* fixed-point iterations of each stage (first 4) */
    int total_iters;     /* sum over all stages */
    double residual;     /* largest final ||v^{k+1} - v^k||_inf over the stages (FP64) */
    double tol_used;     /* tolerance actually applied (FP32 runs: see molt_step) */
} molt_step_info;

/* Create a grid description (host only, no device work).
 * dim = 1: an nx-node line, ny must be 1.  dim = 2: an ny-by-nx grid.  Lx, Ly > 0 are the
 * domain lengths; bc is a molt_bc used in both directions.  Each direction needs at least
 * 8 nodes.  Errors: MOLT_ERR_ARG. */
molt_status molt_grid_create(molt_grid** grid, int dim, int nx, int ny, double Lx, double Ly, int bc);
void molt_grid_destroy(molt_grid* grid);

/* Create a solver on the current CUDA device for `grid` with parameters `p` (copied).
 * Allocates the device workspace (15 fields of the grid's size).
 * Errors: MOLT_ERR_ARG (eps <= 0, M not in {2,4,6}, tol <= 0, max_iter < 1,
 * line shorter than M+2, or x lines longer than the row kernels support: 16384 nodes),
 * MOLT_ERR_OOM, MOLT_ERR_CUDA.  2D time steps additionally need nx <= 8192
 * (their row passes sweep two fields); molt_step returns MOLT_ERR_UNSUPPORTED otherwise. */
molt_status molt_solver_create(molt_solver** solver, const molt_grid* grid, const molt_params* p);
void molt_solver_destroy(molt_solver* solver);

/* Replace the parameters (the precision cannot change).  Clears the time history. */
molt_status molt_set_params(molt_solver* solver, const molt_params* p);

/* Change the boundary condition of both directions.  Clears the time history. */
molt_status molt_set_bc(molt_solver* solver, int bc);

/* How a stage's fixed-point loop is driven.
 * MOLT_EXEC_GRAPH (default): the loop is a CUDA graph with a conditional WHILE node whose
 *   body launches one iteration and a one-thread check kernel that applies the stopping rule on
 *   the device; the host reads the loop state back once per stage.  Graphs are built on first
 *   use per stage coefficient and reused while parameters, boundary condition and dt are
 *   unchanged.  If a graph cannot be built, the host-driven loop runs instead (counted by
 *   molt_graph_fallbacks).
 * MOLT_EXEC_HOST_LOOP: the host launches each iteration and reads the residual back after it
 *   (also used while profiling is enabled). */
typedef enum { MOLT_EXEC_HOST_LOOP = 0, MOLT_EXEC_GRAPH = 1 } molt_execution;
/* mode: a molt_execution value.  Errors: MOLT_ERR_ARG (null solver or unknown mode). */
molt_status molt_set_execution(molt_solver* solver, int mode);
/* Stages that ran the host-driven loop because their graph could not be built (0 for NULL). */
long long molt_graph_fallbacks(const molt_solver* solver);

/* Forget the time history (BDF2 previous level, SDC2 level-[0] state). */
molt_status molt_reset_history(molt_solver* solver);

/* Advance the physical field u (device, in place) by one time step dt > 0 of `scheme`.
 * Every stage solves v - tau F(v) = r with the lagged fixed-point iteration of
 * Eq. CH_BE_fixed2_factor (tau >= eps^2) or Eq. CH_BE_fixed_complete (tau < eps^2),
 * in 2D with the splitting error lagged as in Sec. 5.1.  The sweeps run in the solver's
 * precision; the residual max-norm is exact (Sterbenz) and compared in FP64.  FP32 fields
 * cannot resolve a change below a few units in the last place of the stored variable w
 * (w = u on periodic/Neumann grids, w = u + 1 on Dirichlet grids), so for FP32 solvers the
 * tolerance applied is max(tol, 2 * 2^-24 * max|w|), and an iteration whose residual is below
 * 64 * 2^-24 * max|w| and has not reached a new minimum for 6 iterations is accepted as
 * converged at FP32 precision (the rounding noise floor); `info->tol_used` reports the tolerance (or residual) that ended the stage.  BDF2 and SDC2 keep history between calls made
 * with the same dt.  Returns MOLT_ERR_NOT_CONVERGED (field = last iterate, history
 * updated) when a stage hits max_iter; `info` may be NULL. */
molt_status molt_step(molt_solver* solver, void* u_dev, double dt, int scheme, void* stream,
                      molt_step_info* info);

/* End-to-end variant of molt_step on a HOST buffer: copies u_host to the device, runs
 * `nsteps` steps, copies the result back into u_host and synchronizes `stream`.
 * `info` (may be NULL) reports the last step. */
molt_status molt_run_host(molt_solver* solver, void* u_host, double dt, int scheme, int nsteps,
                          void* stream, molt_step_info* info);

/* Discrete free energy (Eq. EnergyFunctional) of the physical field u (device):
 * h_x h_y [ sum over grid edges of eps^2/2 (difference/h)^2 weighted by the trapezoid
 * weight across the edge + sum over nodes of trapezoid-weighted (u^2-1)^2/4 ], accumulated
 * in FP64 with a fixed summation order.  Synchronizes `stream`. */
molt_status molt_energy(molt_solver* solver, const void* u_dev, double* energy, void* stream);

/* Trapezoid-weighted integral of u (device), FP64, fixed summation order.  Synchronizes. */
molt_status molt_mass(molt_solver* solver, const void* u_dev, double* mass, void* stream);

/* One application of H_c = (I - c d^2)^{-1} (Eq. L_Inverse with alpha = c^{-1/2}) along
 * `axis` (0 = x: every row; 1 = y: every column) to every line of `in_dev`, written to
 * `out_dev` (device; may equal in_dev only for axis 0).  Local quadrature of order M
 * (Sec. 3.2), left/right exponential recurrences (Eq. IL, IR), and the boundary
 * correction of the solver's bc (Eq. homogeneous and its Neumann/Dirichlet analogues).
 * The boundary condition is homogeneous in the values passed in.  c > 0. */
molt_status molt_helmholtz_apply(molt_solver* solver, int axis, double c, const void* in_dev,
                                 void* out_dev, void* stream);

/* The same H_c along x (every row) computed on the tensor cores: the chunked form of the
 * recurrences of Eq. IL / IR as products of 128 x (128 + M) decay-times-quadrature matrices with one
 * window of 128 + M node values per 128-node chunk, on FP16 high / low splits of both operands
 * (three products, FP32 accumulation), followed by an FP32 carry scan per line with the FP64
 * periodic boundary correction (Eq. homogeneous).  An experiment on the split-precision
 * chunked-recurrence variant; molt_helmholtz_apply remains the production sweep.
 * Needs an FP32 solver on a periodic grid with nx a power of two in [1024, 8192] and ny a multiple
 * of 8192 / nx; in_dev and out_dev distinct.  Allocates about 0.45 MB of operand workspace on
 * first use and rebuilds the operands (host FP64, one synchronizing upload) whenever c changes.
 * Errors: MOLT_ERR_ARG, MOLT_ERR_UNSUPPORTED, MOLT_ERR_OOM, MOLT_ERR_CUDA (including a product
 * that did not complete within its one-second wait, reported through the solver's status word
 * at its next step). */
molt_status molt_helmholtz_rows_tc(molt_solver* solver, double c, const void* in_dev, void* out_dev, void* stream);

/* ---- Autotuner (no counterpart in the paper) ------------------------------------------------
 * Each sweep of a step can run on several kernel families; molt_autotune times every one that is
 * available for the solver's grid and keeps the fastest for the solver's later sweeps.
 *   rows:    MOLT_LAUNCH_ROWS_ONE_BLOCK (the pipelined kernel, one block per line),
 *            MOLT_LAUNCH_ROWS_CLUSTER2 (the pipelined kernel on a two-block cluster per line),
 *            MOLT_LAUNCH_ROWS_GENERAL (the general row kernel),
 *            MOLT_LAUNCH_ROWS_TENSOR_CORE (single H_c sweeps only: the chunked recurrence on the
 *            tensor cores of molt_helmholtz_rows_tc; eligible only when its largest difference from
 *            the FP32 sweep on the tuning data is within 1e-6 of the result's largest magnitude);
 *   columns: MOLT_LAUNCH_COLS_TMA (TMA tiles), MOLT_LAUNCH_COLS_CP_ASYNC (cp.async tiles),
 *            MOLT_LAUNCH_COLS_GENERAL (the general column kernels).
 * The scan-versus-chunk choice of the row sweeps is the ROWS_* against ROWS_TENSOR_CORE choice. */
enum {
    MOLT_LAUNCH_DEFAULT = 0,
    MOLT_LAUNCH_ROWS_ONE_BLOCK = 1,
    MOLT_LAUNCH_ROWS_CLUSTER2 = 2,
    MOLT_LAUNCH_ROWS_GENERAL = 3,
    MOLT_LAUNCH_COLS_TMA = 4,
    MOLT_LAUNCH_COLS_CP_ASYNC = 5,
    MOLT_LAUNCH_COLS_GENERAL = 6,
    MOLT_LAUNCH_ROWS_TENSOR_CORE = 7
};

typedef struct {
    int pass;          /* 0 = single H_c sweeps (rhs inverses), 1..4 = 2D iteration passes, 5, 6 = 1D passes,
                          7, 8 = vector-model 2D passes 1 and 2, 9 = vector-model 1D pass a */
    int axis;          /* 0 = rows (x), 1 = columns (y) */
    int chosen;        /* MOLT_LAUNCH_* kept for this sweep (0: none available; the default stays) */
    int candidates;    /* entries of launch[] and ms[] filled */
    int launch[4];     /* the MOLT_LAUNCH_* timed */
    double ms[4];      /* device ms per sweep; -1 = not available for this grid; negative = not eligible */
    double tc_rel_diff; /* tensor-core candidate: largest difference from the FP32 sweep / largest |H f| */
} molt_tuning;

/* Time the candidates of every sweep of a step (FP32 solvers; FP64 solvers keep their one kernel
 * family and report no entries) on hash-uniform test data in the solver's own work fields, and keep
 * the fastest.  Up to `capacity` entries go to `entries` (may be NULL); *count (may be NULL)
 * receives the number of sweeps tuned.  The solver's time history is cleared (its work fields were
 * overwritten) and its cached loop graphs are rebuilt on next use.  Synchronizes `stream`.  Errors:
 * MOLT_ERR_ARG, MOLT_ERR_CUDA. */
molt_status molt_autotune(molt_solver* solver, void* stream, molt_tuning* entries, int capacity, int* count);

/* Host-only diagnostic: the local quadrature weights of Sec. 3.2 for one stencil.
 * Writes M+1 weights of J^L (side = 0) or J^R (side = 1) for node offsets
 * offsets[0..M] (integers relative to the node) at nu = alpha*h > 0, including the
 * factor 1/2 of Eq. IL.  No device work. */
molt_status molt_quadrature_weights(double nu, int M, const int* offsets, int side, double* weights);

/* FP32 column sweep that allocates nothing (no counterpart in the paper; a deployment aid).
 * For callers that cannot call cudaMalloc - code under a memory manager that owns all device
 * memory, or in a latency-critical loop where an allocation could synchronize the device.
 * Applies H_c along y (every column) of the ny-by-nx FP32 field in_dev, writing out_dev (both
 * caller-owned device buffers, row-major [ny][nx], distinct).  The grid convention, bc and
 * quadrature order are those of molt_grid_create / molt_params, with Ly the column length.
 * The scan's scratch is a 4 MiB file-scope device array, held by every GPU that loads the
 * library until the process exits; grids need ceil(ny/128) * nx <= 262144, otherwise
 * MOLT_ERR_ARG.  Outside stream capture every call looks up the array's device address
 * (cudaGetSymbolAddress) in the current context; a call made while `stream` is capturing reuses
 * the address of the last uncaptured call on that device, so make the first call on each device
 * before any stream capture.  All calls share the array: each call writes the scratch before
 * reading it, and calls that overlap on the GPU race on it.  Each call also clears, on `stream`,
 * a device status word that its column kernels set when a bounded wait for a tile copy ran out
 * of time (read it with molt_helmholtz_columns_noalloc_status).  Errors are reported by
 * molt_last_error(NULL). */
molt_status molt_helmholtz_columns_noalloc(int nx, int ny, double Ly, int bc, int quad_order, double c,
                                           const float* in_dev, float* out_dev, void* stream);

/* Status of the last molt_helmholtz_columns_noalloc call (no counterpart in the paper).
 * Synchronizes `stream` and writes the device status word to *status: 0 when every column
 * kernel of that call completed its tiles; bit 0 set when a tile copy did not arrive within its
 * one-second wait, in which case that call's output is incomplete and must not be used.
 * Allocates nothing.  Errors: MOLT_ERR_ARG (null status), MOLT_ERR_CUDA. */
molt_status molt_helmholtz_columns_noalloc_status(void* stream, unsigned* status);

/* ---- Vector Cahn-Hilliard (Sec. 5.2, Eq. CH_vector) -----------------------------------------
 * One step of the three-phase vector model u_t = -Lap[eps^2 Lap u - grad W(u)], u = (u1, u2),
 * W = |z^3 - 1|^2 with z = u1 + i u2, in place on two distinct device fields of the solver's grid
 * and precision (row-major like molt_step).  The state is translated about
 * z3 = (-1/2, -sqrt(3)/2) (Eq. CH_vector_linearize).  Each component's stage solve is the scalar
 * one with 18 in place of 2:
 *   - tau >= eps^2/81: Eq. CH_vector_fixed1, c = 9 tau +- sqrt(81 tau^2 - eps^2 tau);
 *   - otherwise: Eq. CH_vector_fixed2, c = sqrt(eps^2 tau).
 * The lagged term of component j is G_j = [grad W(v + z3)]_j - ((c1 + c2)/tau) v_j.  Both
 * components' lagged terms come from the previous iterate.  The iteration stops on the larger
 * of the two components' changes, as in molt_step.  Boundary conditions apply to v = u - z3, so
 * Dirichlet walls hold u = z3.
 * scheme: MOLT_BE, or MOLT_BDF2 (BE start, and a BE step again after any dt change).
 * The BDF2 history is the state before the previous vector step.  molt_reset_history,
 * molt_set_params and molt_set_bc clear it.
 * Allocates nine work fields on first use.
 * Errors:
 *   MOLT_ERR_ARG: null, equal fields, or a bad dt.
 *   MOLT_ERR_UNSUPPORTED: another scheme, or 2D x lines longer than the two-field row kernels
 *     allow.
 *   MOLT_ERR_NOT_CONVERGED: the fields hold the last iterate.
 *   MOLT_ERR_CUDA, MOLT_ERR_OOM. */
molt_status molt_vch_step(molt_solver* solver, void* u1_dev, void* u2_dev, double dt, int scheme, void* stream,
                          molt_step_info* info);

/* ---- Adaptive step size (Sec. 5, Algorithm 1) ---------------------------------------------
 * One call advances u by one accepted step whose local truncation error estimate eta meets
 * lte_tol.  Two estimators of Sec. 5 (params.estimator):
 *   MOLT_LTE_RICHARDSON: Backward Euler by Richardson extrapolation.  One BE step of size dt and
 *     two of size dt/2, eta = (1/2) max|u_dt - u_dt/2|; the two-half-step solution is kept.
 *   MOLT_LTE_SDC2: BE-SDC2.  One SDC2 step from a fresh start, eta = max|u^[1] - u^[0]| over its
 *     BE level [0] and its second-order level [1]; level [1] is kept.
 *   MOLT_LTE_BDF2: BE-BDF2.  One BE step and one variable-step BDF2 step over the same interval,
 *     from the state before the previous accepted adaptive step (u^{n-1}, step size dt_prev):
 *     with omega = dt/dt_prev, v - tau F(v) = a_n u^n + a_prev u^{n-1}, tau = dt(1+omega)/(1+2omega),
 *     a_n = (1+omega)^2/(1+2omega), a_prev = -omega^2/(1+2omega); eta = max|u_BDF2 - u_BE|, the
 *     BDF2 solution is kept.  The solver keeps u^{n-1} after each accepted BE-BDF2 step; a call
 *     without it (the first, or after molt_step, molt_run_host, molt_reset_history,
 *     molt_set_params, molt_set_bc or an adaptive step with another estimator) uses BE-SDC2.
 * With N_it the largest fixed-point iteration count of the attempt's stage solves and
 * N_maxit = params.max_iter:
 *   eta <= lte_tol and N_it/N_maxit < 0.7: accept, next dt = dt min(theta sqrt(lte_tol/eta), gamma)
 *   eta <= lte_tol and N_it/N_maxit < 1:   accept, next dt = dt min(theta sqrt(lte_tol/eta), 1)
 *   eta <= lte_tol and N_it >= N_maxit:    reject, dt = dt / gamma
 *   eta > 2 lte_tol:                       reject, dt = dt / gamma
 *   lte_tol < eta <= 2 lte_tol:            reject, dt = dt theta sqrt(lte_tol/eta)
 * and the retried / proposed dt is clipped to [dt_min, dt_max]. */
typedef struct {
    double lte_tol;    /* LTE tolerance sigma_tol (> 0) */
    double dt_min;     /* smallest step (> 0); a rejection at dt_min is an error */
    double dt_max;     /* largest step proposed (>= dt_min) */
    double theta;      /* safety factor (paper: 0.8) */
    double gamma;      /* growth / shrink factor (paper: 1.3) */
    int estimator;     /* MOLT_LTE_RICHARDSON (0), MOLT_LTE_SDC2 (1) or MOLT_LTE_BDF2 (2) */
} molt_adaptive;

enum { MOLT_LTE_RICHARDSON = 0, MOLT_LTE_SDC2 = 1, MOLT_LTE_BDF2 = 2 };

typedef struct {
    double dt_used;    /* size of the accepted step */
    double dt_next;    /* proposed size of the next step */
    double eta;        /* LTE estimate of the accepted step */
    int rejections;    /* rejected attempts before it */
    int max_iters;     /* N_it of the accepted attempt */
} molt_adaptive_info;

/* One adaptive step in place on the device field u (FP32 or FP64 as the solver), starting with
 * a trial size dt.  Allocates up to three work fields on first use.  The multistep history (BDF2/BDF3/
 * SDC2) is reset.  Errors: MOLT_ERR_ARG (bad parameters or estimator), MOLT_ERR_NOT_CONVERGED (dt_min
 * reached without meeting lte_tol; u unchanged), MOLT_ERR_CUDA, MOLT_ERR_OOM. */
molt_status molt_step_adaptive(molt_solver* solver, void* u_dev, double dt, const molt_adaptive* params,
                               void* stream, molt_adaptive_info* info);

/* One adaptive step of the vector model (Sec. 5.2) under Algorithm 1 as Sec. 6.2.2 runs it, in
 * place on the two device fields u1, u2 (distinct, the solver's grid and precision), starting
 * with a trial size dt.  Estimators (params.estimator):
 *   MOLT_LTE_RICHARDSON: one vector BE step of dt and two of dt/2, eta = (1/2) max over both
 *     components of |u_dt - u_dt/2|; the two-half-step state is kept.
 *   MOLT_LTE_BDF2: one vector BE step and one variable-step BDF2 step (the formula of
 *     molt_step_adaptive) over the same interval from the state before the previous accepted
 *     step; eta = max over both components of |u_BDF2 - u_BE|; the BDF2 state is kept.  Without
 *     that history (the first call, or after molt_vch_step, molt_reset_history, molt_set_params,
 *     molt_set_bc) the Richardson estimate is used.
 * Accept / reject and the next step size follow the rule documented at molt_step_adaptive.
 * Allocates six more work fields on first use.  Errors: MOLT_ERR_ARG, MOLT_ERR_UNSUPPORTED (another
 * estimator), MOLT_ERR_NOT_CONVERGED (dt_min reached; the fields are unchanged), MOLT_ERR_CUDA,
 * MOLT_ERR_OOM. */
molt_status molt_vch_step_adaptive(molt_solver* solver, void* u1_dev, void* u2_dev, double dt,
                                   const molt_adaptive* params, void* stream, molt_adaptive_info* info);

/* ---- Batched instances ----------------------------------------------------------------
 * Many independent 2D problems, each with its own grid size, eps and time step, stepped
 * together in FP32.  Every instance follows Sec. 2-5 exactly as molt_step does (stage
 * coefficients of Sec. 2.2 / 2.3 from its own tau and eps, the 2D fixed-point iteration of
 * Sec. 5, the stopping rule documented at molt_params).  Each pass of the stage solve is one
 * launch over all instances.  Errors of the batch calls are reported by molt_last_error(NULL). */
typedef struct molt_batch molt_batch;

typedef struct {
    int nx, ny;      /* grid nodes of the instance, each in [quad_order + 2, 1024] */
    double Lx, Ly;   /* domain lengths (> 0) */
    double eps;      /* interface parameter (> 0) */
} molt_instance;

/* Create a batch of `count` >= 1 instances sharing the boundary condition, the quadrature
 * order M (2, 4 or 6), the fixed-point tolerance and max_iter.  The batch owns its device
 * workspace (ten packed fields plus scan scratch).  A packed field stores the instances back to
 * back: instance i occupies ny_i * nx_i floats, row-major with x fastest, from
 * molt_batch_offsets()[i].  Errors: MOLT_ERR_ARG, MOLT_ERR_OOM, MOLT_ERR_CUDA. */
molt_status molt_batch_create(molt_batch** batch, int count, const molt_instance* instances, molt_bc bc,
                              int quad_order, double tol, int max_iter);
molt_status molt_batch_destroy(molt_batch* batch);

/* Floats in one packed field (sum of ny_i * nx_i); 0 for NULL. */
long long molt_batch_points(const molt_batch* batch);

/* Offsets (in floats) of the `count` instances in a packed field. */
molt_status molt_batch_offsets(const molt_batch* batch, long long* offsets);

/* Graph (default) or host-driven stage loop; both give bit-identical fields. */
molt_status molt_batch_set_execution(molt_batch* batch, molt_execution mode);

/* One time step of every instance, in place on the packed device field u_dev (FP32, u of the
 * paper).  dt: host array of `count` steps (> 0).  scheme: MOLT_BE or MOLT_BDF2 (BDF2 starts
 * with one BE step, again whenever any dt changes).  The step's stage (rhs inverse and the
 * fixed-point loop) runs as one CUDA graph with a conditional WHILE node; each instance stops
 * on its own rule and skips later iterations.  iters / residual / status: host arrays of
 * `count` entries (each may be NULL) receiving each instance's iterations, last residual
 * max|w_new - w| and MOLT_OK or MOLT_ERR_NOT_CONVERGED.  Returns MOLT_ERR_NOT_CONVERGED when any
 * instance reached max_iter (the fields hold the last iterates), MOLT_ERR_UNSUPPORTED for other
 * schemes, MOLT_ERR_ARG, MOLT_ERR_CUDA. */
molt_status molt_batch_step(molt_batch* batch, float* u_dev, const double* dt, molt_scheme scheme, void* stream,
                            int* iters, double* residual, int* status);

/* One line inversion H_c (Sec. 3.2, Eq. IL/IR with the boundary correction of Sec. 3.3) of every
 * instance of the batch along one axis (0 = x, each row; 1 = y, each column), in one launch
 * sequence over all instances: out = H_{c_i} in, instance by instance, with the batch's boundary
 * condition and M.  c: host array of `count` values (> 0; alpha = c^(-1/2)); in, out: packed
 * device fields (FP32, layout of molt_batch_create), not aliased.  Per axis the batch keeps the
 * line parameters of the last two arrays c it swept with; another c is built on the host and
 * uploaded (the call then synchronizes `stream`).  Later steps reload their own parameters.
 * Asynchronous otherwise.  Errors: MOLT_ERR_ARG, MOLT_ERR_CUDA. */
molt_status molt_batch_helmholtz_apply(molt_batch* batch, int axis, const double* c, const float* in_dev,
                                       float* out_dev, void* stream);

/* Schedule autotuner of the batched passes (no counterpart in the paper).  Every batched kernel
 * walks its work list (row items, column tiles, carry items) from its block index in steps of the
 * grid size, so one launch runs either one block per work item or a persistent grid of a few
 * blocks per SM looping over the items.  This call times one fixed-point iteration of every
 * instance under each of 4 x 4 schedules (rows x columns: one block per item, 2, 4 or 8 blocks per
 * SM), with the stage parameters of the steps dt (host array of `count`), and keeps the fastest
 * for later steps.  ms_table (16 entries, row schedule major; may be NULL) receives the times,
 * grid_rows / grid_cols (may be NULL) the chosen grids (0 = one block per item).  It overwrites
 * the batch's work fields and forgets the BDF2 history; synchronizes `stream`.  Errors:
 * MOLT_ERR_ARG, MOLT_ERR_CUDA. */
molt_status molt_batch_autotune(molt_batch* batch, const double* dt, void* stream, double* ms_table, int* grid_rows,
                                int* grid_cols);

/* Set the schedule of the batched passes directly: grid_rows / grid_cols blocks per row / column
 * launch (0 = one block per work item).  Results do not depend on it.  Errors: MOLT_ERR_ARG. */
molt_status molt_batch_set_schedule(molt_batch* batch, int grid_rows, int grid_cols);

/* ---- Three-dimensional split stage (the extension of Sec. 5's splitting to 3D) ------------
 * The paper only remarks that its dimensional splitting extends to three dimensions.  The
 * reading implemented here: with L_a = I - c d_aa per axis, I - c Lap = L_x L_y L_z - P, and with
 * H_a = L_a^{-1}, D_a = I - H_a, M^{-1} = H_x H_y H_z, the splitting remainder is
 * M^{-1} P = X = D_x D_y + D_x D_z + D_y D_z - 2 D_x D_y D_z (X = D_x D_y in 2D, Eq.
 * CH_2D_Doperator1); the 2D fixed-point iteration of Sec. 5.1 then holds with X in place of
 * D_x D_y.  FP32 fields of nz * ny * nx floats, row-major with x fastest, periodic or Neumann
 * lines (the grid conventions of molt_grid_create per axis).  Each iteration is a sequence of
 * single line sweeps over the whole field (not fused).  Errors of these calls are reported by
 * molt_last_error(NULL). */
typedef struct molt_solver3d molt_solver3d;

/* nx, ny in [M + 2, 1024] (the y lines run as a batch of nz slabs, molt_batch_create), nz in
 * [M + 2, 2^20];
 * params: precision must be MOLT_FP32; eps, M, tol and max_iter as molt_solver_create.  The
 * solver owns 14 fields of workspace, the column scan scratch of the z lines and an internal
 * batch of nz slabs.  Errors: MOLT_ERR_ARG, MOLT_ERR_UNSUPPORTED (Dirichlet, FP64),
 * MOLT_ERR_OOM, MOLT_ERR_CUDA. */
molt_status molt_solver3d_create(molt_solver3d** solver, int nx, int ny, int nz, double Lx, double Ly,
                                 double Lz, molt_bc bc, const molt_params* params);
molt_status molt_solver3d_destroy(molt_solver3d* solver);

/* One time step in place on the device field u_dev (u of the paper): MOLT_BE, or MOLT_BDF2 with a
 * BE start repeated whenever dt changes.  The stage's stopping rule is molt_step's (FP32 floor
 * and stall rule); info (may be NULL) receives iterations, residual and tolerance used.
 * Synchronizes `stream` once per iteration (host-driven loop).  Errors: MOLT_ERR_ARG,
 * MOLT_ERR_UNSUPPORTED (other schemes), MOLT_ERR_NOT_CONVERGED (the field holds the last
 * iterate), MOLT_ERR_CUDA. */
molt_status molt_solver3d_step(molt_solver3d* solver, float* u_dev, double dt, molt_scheme scheme, void* stream,
                               molt_step_info* info);

/* One line inversion H_c (Sec. 3) of every line along axis 0 (x), 1 (y) or 2 (z); in_dev and
 * out_dev distinct.  Synchronizes `stream` to read the column kernels' wait status.  Errors:
 * MOLT_ERR_ARG, MOLT_ERR_CUDA (also when a bounded wait for a tile copy ran out). */
molt_status molt_solver3d_apply(molt_solver3d* solver, int axis, double c, const float* in_dev, float* out_dev,
                                void* stream);

/* Kernels this 3D solver has launched (its internal batch's sweeps counted as 3 each). */
long long molt_solver3d_launches(const molt_solver3d* solver);

/* ---- Sixth-order (functionalized) Cahn-Hilliard model on independent 1D lines ----------------
 * Eq. FCH0 in v = u + 1 (Eq. FCH): v_t = Lap[(eps^2 Lap - f'(v) + eta eps^2)(eps^2 Lap v - f(v))],
 * f(v) = v^3 - 3v^2 + 2v, BE steps with the cube completed (the paper's last section).  The
 * reading implemented: BE keeps the PDE's signs (Eq. FCH_BE prints the last four bracket terms
 * with the opposite ones); with a = (dt eps^4)^(1/3), H = (I - a Lap)^{-1} (the line inverse of
 * Sec. 3 with c = a) and D = H - I the lagged iteration is v^{k+1} = H z,
 *   z = H^2 v^n + (3 + c_eta) D^2 v - 3 H D v - c_f D^2 f + c_p H D p,
 *   p = -eps^2 f' Lap v + f f' - eta eps^2 f,
 * c_eta = dt eta eps^4 / a^2, c_f = dt eps^2 / a^2, c_p = dt / a, and Lap v^{k+1} = (v^{k+1} - z)/a
 * carried with the iterate (across steps; the first step takes (H v^n - v^n)/a).  About the
 * wells a mode x = a k^2 is multiplied per iteration by m(x) = h[(3 + c_eta - 2c_f) x^2 h^2 + 3x h^2
 * - c_p x h^2 (2 eps^2 x / a + 4 - 2 eta eps^2)], h = 1/(1 + x): the iteration diverges where
 * |m| > 1 (eps = 0.18, eta = 1: dt = 0.1 does, dt <= 0.07 does not).  Fields are `lines`
 * independent lines of nx nodes, [lines][nx] row-major, FP32 or FP64 per params->precision.
 * Each iteration runs 7 line sweeps, one pointwise kernel and 6 linear combinations, and
 * synchronizes `stream` to read the residual.  Errors of these calls are reported by
 * molt_last_error(NULL). */
typedef struct molt_fch1d molt_fch1d;

/* nx in [M + 2, the one-field row kernel's limit (molt_solver_create's 1D limit)], lines in
 * [1, 2^24], L > 0 the line length (the grid conventions of molt_grid_create), bc periodic or
 * Neumann, eta finite; params: precision, eps, M, tol, max_iter as molt_solver_create.  The
 * solver owns 16 fields of nx * lines values.  Errors: MOLT_ERR_ARG, MOLT_ERR_UNSUPPORTED
 * (Dirichlet), MOLT_ERR_OOM. */
molt_status molt_fch1d_create(molt_fch1d** solver, int nx, int lines, double L, molt_bc bc, double eta,
                              const molt_params* params);
molt_status molt_fch1d_destroy(molt_fch1d* solver);

/* One BE step in place on the device field u_dev (u of the paper; float* or double* per the
 * precision).  The stopping rule is molt_step's: ||v^{k+1} - v^k||_inf < tol (Sec. 4.4) over all
 * lines, in FP32 floored at 2 ulp of max|v| with the stall rule below 64 ulp.  info (may be NULL)
 * receives the iterations, residual and tolerance used.  Errors: MOLT_ERR_ARG (null, dt <= 0),
 * MOLT_ERR_NOT_CONVERGED (the field holds the last iterate), MOLT_ERR_CUDA. */
molt_status molt_fch1d_step(molt_fch1d* solver, void* u_dev, double dt, void* stream, molt_step_info* info);

/* Kernels launched by this solver so far (host counter). */
long long molt_fch1d_launches(const molt_fch1d* solver);

/* ---- Sixth-order model on a 2D grid (the paper's case) -----------------------------------------
 * Eq. FCH0 / FCH with BE and the cube completed as for molt_fch1d_*, split as in Sec. 5.1: with
 * M^{-1} = H_x H_y (line inverses of I - a d_xx, I - a d_yy, a = (dt eps^4)^(1/3)) and
 * X = D_x D_y, I - a Lap = M (I - X), and the lagged iteration is v <- M^{-3} R(v) + (1 - (1-X)^3) v
 * (R as in 1D).  With K = M^{-1} a Lap = 2 M^{-1} - H_x - H_y the iterate is kept as v = M^{-1} W,
 *   W <- M^{-2} v^n - 3 M^{-1} K v + (3 + c_eta) K^2 v - c_f K^2 f + c_p M^{-1} K p
 *        + (3X - 3X^2 + X^3) W,
 * so that Lap v = K W / a exactly (the first step starts from W = v^n; later steps carry W).
 * Fields [ny][nx] row-major, x fastest, FP32 or FP64 per params->precision, periodic or Neumann
 * (the grid conventions of molt_grid_create).  Regrouped by linearity, each iteration runs 14
 * one-field line sweeps, one pointwise kernel and 11 linear combinations, and synchronizes
 * `stream` to read the residual.
 * Errors are reported by molt_last_error(NULL). */
typedef struct molt_fch2d molt_fch2d;

/* nx in [M + 2, the one-field row kernel's limit], ny >= M + 2, nx * ny < 2^31, Lx, Ly > 0, bc
 * periodic or Neumann, eta finite; params as molt_solver_create.  The solver owns 23 fields of
 * nx * ny values and the column scan scratch.  Errors: MOLT_ERR_ARG, MOLT_ERR_UNSUPPORTED
 * (Dirichlet), MOLT_ERR_OOM. */
molt_status molt_fch2d_create(molt_fch2d** solver, int nx, int ny, double Lx, double Ly, molt_bc bc, double eta,
                              const molt_params* params);
molt_status molt_fch2d_destroy(molt_fch2d* solver);

/* One BE step in place on the device field u_dev (float* or double* per the precision), with
 * molt_fch1d_step's stopping rule and info.  Errors: MOLT_ERR_ARG, MOLT_ERR_NOT_CONVERGED (the
 * field holds the last iterate), MOLT_ERR_CUDA (also when a column kernel's bounded wait for a
 * tile copy ran out). */
molt_status molt_fch2d_step(molt_fch2d* solver, void* u_dev, double dt, void* stream, molt_step_info* info);

/* Kernels launched by this solver so far (host counter). */
long long molt_fch2d_launches(const molt_fch2d* solver);


/* Last error message of `solver` (or of the last failed create/ABI call when NULL). */
const char* molt_last_error(const molt_solver* solver);

/* Number of kernels this solver has launched so far (all entry points), for reporting. */
long long molt_kernel_launches(const molt_solver* solver);

/* Diagnostics (no counterpart in the paper): number of FP32 column-sweep kernels launched with
 * tensor-memory-accelerator tile loads since the library was loaded, over all solvers and
 * entry points.  Eligible column sweeps (FP32, lines a multiple of 32, length >= 256, 16-byte
 * aligned fields) use these kernels unless the environment variable MOLT_COLS_TMA is "0" when
 * the sweep is launched or captured; both kernel families give bit-identical results. */
long long molt_column_tma_launches(void);

/* Diagnostics (no counterpart in the paper): checks on the GPU that a device-side wait gives up
 * instead of hanging.  Launches one block whose mbarrier wait can never complete, through the
 * same bounded wait the TMA column kernels use for their tile copies (limit: 1 s of GPU time).
 * On return *timed_out = 1 if the wait gave up and set the status word, *waited_seconds = how
 * long it waited.  Synchronizes the device; allocates two small device words.  Errors:
 * MOLT_ERR_ARG (null output), MOLT_ERR_CUDA. */
molt_status molt_selftest_bounded_wait(int* timed_out, double* waited_seconds);

/* Diagnostics (no counterpart in the paper): the fused multiply-add throughput the current GPU
 * sustains in `precision` (MOLT_FP32 or MOLT_FP64), in TFLOP/s (one FMA = 2 flops): independent
 * FMA chains in registers, 8 blocks of 256 threads per SM, timed with CUDA events after one
 * warm-up launch.  The ceiling of the FP64 line sweeps, which are arithmetic-bound on this part.
 * Synchronizes the device; allocates a small result buffer.  Errors: MOLT_ERR_ARG, MOLT_ERR_CUDA. */
molt_status molt_fma_throughput_probe(int precision, double* tflops);

/* Diagnostic timing (not part of the method; off by default).  While enabled, every sweep
 * kernel launch is bracketed by two CUDA events on its stream. */
molt_status molt_profile_enable(molt_solver* solver, int enable);

/* Wait for the recorded events and write, per kernel slot (MOLT_PROFILE_SLOTS entries), the
 * summed device milliseconds and launch counts since the last collect; then forget them.
 * Slots: row kernel of fused pass k = k, column aggregate kernel of pass k = 8 + k, column
 * carry kernel = 16, column final kernel of pass k = 17 + k, with k = 0 plain H_c, 1 pass 1,
 * 2 pass 2, 3 pass 3, 4 pass 4, 5 and 6 the two 1D passes. */
#define MOLT_PROFILE_SLOTS 32
molt_status molt_profile_collect(molt_solver* solver, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* MOLT_H */
