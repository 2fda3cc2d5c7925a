/*
 * kkt.h -- C ABI of the GB300 KKT refactorization library.
 *
 * The library solves the sequence of sparse symmetric indefinite systems
 * K_k x_k = b_k, k = 1..M, that an interior-point ACOPF solver produces
 * (Eq. 11; Alg. 1). All K_k share one sparsity pattern (Sec. II), so the
 * work splits into the three stages of a sparse direct solver (Sec. II):
 *
 *   kkt_analyze   once per pattern, on the host: equilibration plan,
 *                 fill-reducing ordering, frozen pivot sequence, symbolic
 *                 factorization, supernodal assembly tree and its level
 *                 schedule; uploaded to the GPU once (Alg. 1 setup).
 *   kkt_refactor  per K_k, on the GPU: equilibrate, load the new values
 *                 into the frozen factor pattern and refactor without
 *                 pivoting (Alg. 1).
 *   kkt_solve     triangular solves with the current factors (Alg. 1).
 *   kkt_refine    solve followed by iterative refinement to a backward-error
 *                 tolerance (Alg. 1 refines every solve; Sec. V calls for a
 *                 better refinement: FGMRES here).
 *
 * Conventions
 *   - Matrices are full symmetric CSR (both triangles), 0-based int32 row
 *     pointers and column indices, columns sorted and unique within a row,
 *     every diagonal entry stored. Values are FP64.
 *   - Pointers named h_* are host memory, d_* are device memory of the
 *     current CUDA device. The caller owns every array it passes; device
 *     arrays must stay valid until the work on `stream` has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls taking a stream are asynchronous and stream-ordered
 *     unless stated otherwise; none allocates device memory (all memory is
 *     allocated by kkt_analyze).
 *   - A kkt_ctx is not thread-safe: use one context per session / thread.
 *   - No C++ exception crosses this interface; errors are kkt_status codes.
 */
#ifndef KKT_GB300_H
#define KKT_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kkt_ctx kkt_ctx;
typedef struct kkt_model kkt_model;
typedef struct kkt_group kkt_group;

typedef enum {
    KKT_OK = 0,
    KKT_E_ARG = 1,        /* invalid argument (null pointer, bad size, bad option) */
    KKT_E_CUDA = 2,       /* a CUDA runtime call failed */
    KKT_E_NOMEM = 3,      /* device or host allocation failed, or over the memory budget */
    KKT_E_STATE = 4,      /* call out of order (solve before refactor, ...) */
    KKT_E_STRUCT = 5,     /* pattern not symmetric / unsorted / missing diagonal */
    KKT_E_NOCONV = 6,     /* refinement did not reach the tolerance */
    KKT_E_TIMEOUT = 7,    /* a bounded device wait gave up */
    KKT_E_NUMERIC = 8     /* NaN or Inf met in the factorization or the residual */
} kkt_status;

enum { KKT_FP64 = 0,      /* factors and triangular solves in FP64 */
       KKT_FP32_IR = 1 }; /* factors and triangular solves in FP32 (FP32 accumulation);
                             scaling, residual and FGMRES stay FP64 */

enum { KKT_PRECOND_LU = 0,       /* refinement preconditioned by the exact triangular solves */
       KKT_PRECOND_JACOBI = 1,    /* ... by Jacobi sweeps with the factors (approximate, Sec. V) */
       KKT_PRECOND_BLOCK_JACOBI = 2 };  /* ... by block-Jacobi sweeps, each front's pivots a block
                                           solved exactly inside the sweep (Gauss-Seidel within it) */

enum { KKT_ORDER_MINDEG = 0,  /* the library's quotient-graph minimum degree */
       KKT_ORDER_USER = 1,    /* kkt_options.user_perm */
       KKT_ORDER_NATURAL = 2 };

typedef struct {
    int precision;              /* KKT_FP64 (default) or KKT_FP32_IR */
    int ordering;               /* KKT_ORDER_* (default KKT_ORDER_MINDEG) */
    const int32_t *user_perm;   /* host, n entries: user_perm[k] = original row/column
                                   eliminated k-th; read only during kkt_analyze */
    double static_pivot_eps;    /* a pivot u_jj with |u_jj| < eps * max|D K D| is replaced by
                                   sign(u_jj) * eps * max|D K D| (sign(0) = +1) and counted.
                                   <= 0 selects the default: 1e-14 (FP64), 1e-7 (FP32);
                                   NaN or >= 1: KKT_E_ARG */
    int ruiz_iters;             /* equilibration iterations per refactor (default 10) */
    int restart;                /* FGMRES restart length m (default 30, max 64) */
    int max_cycles;             /* FGMRES restart cycles (default 10) */
    int relax_pivots;           /* supernode amalgamation: max pivots of a merged front
                                   for the "small front" rule (default 16) */
    double relax_zeros;         /* amalgamation: max share of explicit zeros (default 0.15;
                                   outside [0, 1] or NaN: KKT_E_ARG) */
    int max_pivots;             /* pivots per supernode: merges stop and larger supernodes
                                   are split into chains at this size (default 16, max 64) */
    int no_graphs;              /* 1: launch every kernel from the host instead of replaying
                                   the captured CUDA graphs of the level loops (default 0) */
    int tree_min_fronts;        /* the top levels of the assembly tree that hold fewer fronts
                                   than this (fronts x instances for a batched context; every
                                   level above them included) are refactored and
                                   solved by persistent, dependency-driven kernels instead of
                                   one launch per level (default 2432; 0 = one launch per level
                                   everywhere). Both schedules give bitwise identical results */
    long long spin_limit;       /* polls (about 100 ns each) of a bounded device wait of those
                                   kernels before it gives up and the call reports
                                   KKT_E_TIMEOUT (default 1 << 23, about a second) */
    int precond;                /* KKT_PRECOND_* for kkt_refine and kkt_precondition
                                   (default KKT_PRECOND_LU) */
    int jacobi_sweeps;          /* sweeps per triangular factor with KKT_PRECOND_JACOBI or
                                   KKT_PRECOND_BLOCK_JACOBI (default 4, 1..1000000) */
} kkt_options;

typedef struct {
    int n_perturbed;            /* static pivot perturbations in the last refactor */
    int iters;                  /* FGMRES inner iterations of the last refine */
    double backward_err;        /* omega = ||b-Kx||_inf / (||K||_inf ||x||_inf + ||b||_inf), FP64 */
    double rel_resid2;          /* ||b-Kx||_2 / ||b||_2 */
    int refactor_count;         /* refactorizations since analyze */
    int status;                 /* kkt_status of the last numeric call (device-side checks) */
    long long launches;         /* CUDA kernels this context has launched since analyze */
    int batch;                  /* numeric instances of the context (kkt_get_info) */
} kkt_info;

/* Per-kernel timing of a context in profiling mode (see kkt_set_profiling). */
typedef struct {
    const char *name;           /* kernel (or kernel family) name, static storage */
    long long launches;         /* kernels launched */
    double ms;                  /* summed CUDA-event time of their launch groups */
} kkt_kernel_stat;

/* Sizes of an analysis: what a context will hold in device memory. */
typedef struct {
    int n;
    int64_t nnz;                /* nonzeros of K */
    int64_t nnz_lu;             /* structural nonzeros of L + U (diagonal once) */
    int64_t stored_factor;      /* factor values stored (incl. amalgamation zeros) */
    int n_fronts;               /* supernodes / frontal matrices */
    int n_levels;               /* levels of the assembly tree */
    int max_front;              /* largest frontal matrix order */
    int max_pivots;             /* most pivots in one front */
    double flops;               /* dense front flops per refactor */
    double flops_exact;         /* flops on the exact (non-amalgamated) structure */
    int64_t device_bytes;       /* device memory kkt_analyze would allocate (one instance) */
    int batch;                  /* instances of the context (kkt_get_plan) */
    int tree_levels;            /* top levels run by the persistent tree kernels */
    int tree_units;             /* refactorization work units of those kernels (one instance) */
    int64_t tree_bytes;         /* multifrontal traffic of one refactorization of the tree part
                                   (one instance): original entries (value, position, source),
                                   factor panels written, contribution blocks written and read once */
    int64_t tree_nnz_k;         /* nonzeros of K assembled into the fronts of the tree part */
    int64_t tree_nnz_lu;        /* structural nonzeros of L + U in the tree part's pivot columns
                                   and rows (diagonal once) */
    int tree_pivots;            /* pivots eliminated by the tree part */
} kkt_plan_info;

/* Fill *opt with the defaults listed above. */
void kkt_default_options(kkt_options *opt);

/* Host-only: run the analysis of kkt_analyze (ordering, symbolic
 * factorization, supernodes, schedule) and report its sizes without touching
 * the GPU. Used for memory-budget admission. opt may be NULL (defaults).
 * Errors: KKT_E_ARG, KKT_E_STRUCT. */
kkt_status kkt_plan(int32_t n, const int32_t *h_rowptr, const int32_t *h_colidx,
                    const kkt_options *opt, kkt_plan_info *out);

/* Host-only: the supernodal fronts the analysis of kkt_plan builds, for
 * inspection (the dense blocks of the factorization; Sec. II notes that these
 * KKT matrices are sparse and irregular, with few dense blocks). On return
 * *count = number of fronts; h_order (front order F, pivot rows plus
 * contribution rows) and h_pivots (pivots w) receive min(*count, capacity)
 * entries each, in assembly-tree postorder; both may be NULL with capacity 0
 * to query the count. Errors: as kkt_plan. */
kkt_status kkt_plan_fronts(int32_t n, const int32_t *h_rowptr, const int32_t *h_colidx,
                           const kkt_options *opt, int32_t capacity, int32_t *h_order, int32_t *h_pivots,
                           int32_t *count);

/* Analysis stage (Sec. II, first of the three stages; Alg. 1 setup). n_primal is the size
 * of the (1,1) block (used only for reporting). The pattern arrays are read
 * and copied; h_vals is not needed by the static-pivot analysis and may be
 * NULL. Allocates every device buffer the context will use, on the current
 * device, and uploads the schedule. On success *out receives a context
 * that kkt_destroy frees. Synchronous: the uploads go through the context's
 * own non-blocking stream, which is waited for before the call returns, so
 * the first refactorization may be issued on any stream of the caller
 * (including a non-blocking one) without further synchronization.
 * Errors: KKT_E_ARG, KKT_E_STRUCT, KKT_E_NOMEM, KKT_E_CUDA. */
kkt_status kkt_analyze(int32_t n, int32_t n_primal, const int32_t *h_rowptr,
                       const int32_t *h_colidx, const double *h_vals,
                       const kkt_options *opt, kkt_ctx **out);

/* Batched context: the analysis of kkt_analyze done once and `count` numeric
 * instances that share it (one pattern, different values: e.g. scenarios of
 * one grid). Every numeric call on such a context works on all instances at
 * once -- each level of the assembly tree is one launch for all of them --
 * with instance-major arrays: values count x nnz, right-hand sides and
 * solutions count x n; kkt_refine and kkt_step_host fill count kkt_info
 * entries. Factor export and scaling queries report instance 0.
 * Errors: as kkt_analyze. */
kkt_status kkt_analyze_batch(int32_t n, int32_t n_primal, const int32_t *h_rowptr,
                             const int32_t *h_colidx, const kkt_options *opt, int32_t count,
                             kkt_ctx **out);

/* Numeric refactorization (Alg. 1) of the matrix with values
 * d_vals (device, nnz FP64 in the CSR order given to kkt_analyze):
 * power-of-two symmetric Ruiz equilibration D K D (FP64), scatter into the
 * frozen pattern, multifrontal LU without pivoting of P (D K D) P^T with
 * static pivot perturbation, in the context's precision. Asynchronous.
 * Device-detected NaN/Inf are reported by kkt_get_info (status field).
 * Errors: KKT_E_ARG, KKT_E_CUDA. */
kkt_status kkt_refactor(kkt_ctx *ctx, const double *d_vals, void *stream);

/* x = K^{-1} b with the current factors (Alg. 1, without refinement):
 * x = D P^T U^{-1} L^{-1} P D b. d_rhs and d_x are device FP64 vectors of
 * length n and may not alias. Asynchronous.
 * Errors: KKT_E_ARG, KKT_E_STATE (no refactor yet), KKT_E_CUDA. */
kkt_status kkt_solve(kkt_ctx *ctx, const double *d_rhs, double *d_x, void *stream);

/* Solve then refine with restarted FGMRES(m) on the unscaled K, right
 * preconditioned by the factors, Arnoldi and update in FP64, until the
 * backward error omega <= tol (Alg. 1 with refinement; Sec. V). The
 * backward error of every instance is evaluated on the device after the
 * solve; FGMRES runs only for instances above tol (rel_resid2 is then set,
 * else -1). Synchronizes `stream` (the restart loop reads convergence on the
 * host). info (may be NULL; one entry per instance) receives iterations and
 * the final omega.
 * Errors: KKT_E_ARG, KKT_E_STATE, KKT_E_CUDA, KKT_E_NOCONV, KKT_E_NUMERIC. */
kkt_status kkt_refine(kkt_ctx *ctx, const double *d_rhs, double *d_x, double tol,
                      kkt_info *info, void *stream);

/* z = M^{-1} r with the context's preconditioner (kkt_options.precond): the
 * exact triangular solves (as kkt_solve) or Jacobi sweeps with the factors,
 * the approximate triangular solves the paper proposes instead of the
 * level-scheduled ones (Sec. V): from y_0 = x_0 = 0, y_{s+1} = c - (L - I) y_s
 * and x_{s+1} = diag(U)^{-1} (y - (U - diag(U)) x_s) on c = P D r, then
 * z = D P^T x. d_rhs and d_z are device FP64 (count x n), may not alias.
 * Asynchronous. Errors: KKT_E_ARG, KKT_E_STATE (no refactor yet), KKT_E_CUDA. */
kkt_status kkt_precondition(kkt_ctx *ctx, const double *d_rhs, double *d_z, void *stream);

/* kkt_refactor followed by kkt_refine in one call (one interior-point
 * iteration's linear algebra, Alg. 1 loop body): with the exact preconditioner
 * the forward substitution of the first solve runs inside the refactorization
 * (each front is forward-substituted as soon as it and its children are
 * done), saving the separate forward pass. Same inputs, outputs, errors and
 * synchronization as the two calls. */
kkt_status kkt_refactor_refine(kkt_ctx *ctx, const double *d_vals, const double *d_rhs, double *d_x,
                               double tol, kkt_info *info, void *stream);

/* Asynchronous solve with a device-side accuracy check, for callers that keep
 * several solves in flight: x = K^{-1} b for every instance, then
 * h_omega[i] = backward error omega of instance i. h_omega is host memory
 * (count doubles; page-locked memory keeps the call asynchronous) and holds
 * the values once the work on `stream` has completed; an instance above the
 * caller's tolerance can then be passed to kkt_refine. No synchronization.
 * Errors: KKT_E_ARG, KKT_E_STATE, KKT_E_CUDA. */
kkt_status kkt_solve_checked(kkt_ctx *ctx, const double *d_rhs, double *d_x, double *h_omega,
                             void *stream);

/* One whole IPM step through host memory, for callers without device
 * buffers: copy h_vals and h_rhs to the device, refactor, refine to tol, copy
 * x back to h_x. Synchronous. Same errors as kkt_refine. */
kkt_status kkt_step_host(kkt_ctx *ctx, const double *h_vals, const double *h_rhs,
                         double *h_x, double tol, kkt_info *info, void *stream);

/* Refactor several different contexts (patterns and sizes may differ) at
 * once: each context works on its own internal stream, forked from `stream`
 * and joined back into it, so their level graphs run concurrently on the
 * device. ctxs must be distinct and share one precision. Asynchronous.
 * Errors: KKT_E_ARG, KKT_E_CUDA. */
kkt_status kkt_refactor_batched(kkt_ctx *const *ctxs, const double *const *d_vals,
                                int count, void *stream);

/* Refactorization of many systems of uneven sizes in one launch (Alg. 1's
 * refactor step for every member, batched across sessions or scenarios).
 * kkt_group_create takes `count` distinct contexts of one precision (their
 * patterns and sizes may differ, each may be batched) and allocates the
 * group's small device tables (the one allocating call of the group API);
 * the contexts must outlive the group. kkt_refactor_group(g, d_vals, stream)
 * then refactors member i with the values d_vals[i] (device, instance-major
 * as in kkt_refactor): equilibration and the level-launched lower levels of
 * each member on its own internal stream (forked from `stream` and joined
 * back), then the narrow tops of all members' assembly trees in ONE launch of
 * the persistent tree kernel, whose work units interleave the members by
 * height below their roots. Results are bitwise those of kkt_refactor on each
 * member. Asynchronous; kkt_solve / kkt_refine etc. then work on each member
 * as usual. The group's tree launch is counted in the first member's launch
 * counter. Errors: KKT_E_ARG (null, duplicate, mixed precision), KKT_E_NOMEM,
 * KKT_E_CUDA. */
kkt_status kkt_group_create(kkt_ctx *const *ctxs, int count, kkt_group **out);
kkt_status kkt_refactor_group(kkt_group *g, const double *const *d_vals, void *stream);
kkt_status kkt_group_destroy(kkt_group *g);

/* kkt_solve over several distinct contexts, concurrently as above.
 * Asynchronous. */
kkt_status kkt_solve_batched(kkt_ctx *const *ctxs, const double *const *d_rhs,
                             double *const *d_x, int count, void *stream);

/* Residual r = b - K x (FP64, unscaled K of the last refactor; the library
 * keeps its own copy of K, so d_vals may be released once kkt_refactor's
 * work on the stream has completed) and the
 * backward error omega of x; omega_out (host) may be NULL. Synchronous when
 * omega_out is not NULL. Errors: KKT_E_ARG, KKT_E_STATE, KKT_E_CUDA. */
kkt_status kkt_residual(kkt_ctx *ctx, const double *d_rhs, const double *d_x, double *d_r,
                        double *omega_out, void *stream);

/* Statistics of the context. Synchronizes the device to read the
 * perturbation count and NaN/Inf flag of the last refactor. */
kkt_status kkt_get_info(const kkt_ctx *ctx, kkt_info *info);

/* Residual and backward error without allocating anything (the paper has no
 * counterpart; this is a service for callers that cannot allocate device
 * memory: a host framework that owns all device memory through its own pool,
 * a serving loop held to a fixed memory budget, or a check of a solution made
 * before any kkt_ctx exists). No context is needed: K is given directly as
 * device CSR (d_rowptr n+1, d_colidx and d_vals nnz, FP64), with d_x, d_rhs
 * (n each) as inputs. Outputs: d_r = b - K x (n, device) and d_omega[0] =
 * ||r||_inf / (||K||_inf ||x||_inf + ||b||_inf) (one double, device).
 * NaN anywhere in K, x or b makes omega NaN (the maxima are taken on the bit
 * patterns, where NaN sorts above +Inf), so a NaN solution never passes a
 * tolerance test.
 * Preconditions: every pointer is memory of the current device; rowptr is
 * non-decreasing from 0 with rowptr[n] <= nnz, and every column index lies in
 * [0, n). The kernel checks both as it reads: a row that breaks them is not
 * read outside its arrays, its r_i is set to NaN, and omega is NaN.
 * The reduction scratch is a fixed 256 KiB array in device memory that the
 * library declares statically; every GPU that loads the library holds it
 * until the process exits. Limit: n <= 8,388,608 rows, else KKT_E_ARG. The
 * first call on a device looks up that array's device address (once per
 * device, with the device current); make that first call before any stream
 * capture. Every call uses the same array, so calls that overlap on the GPU
 * (on different streams, or from several threads) race and must be ordered
 * by the caller. Asynchronous on `stream`.
 * Errors: KKT_E_ARG (null pointer, n <= 0, nnz < 0, n above the limit), KKT_E_CUDA. */
kkt_status kkt_backward_error_noalloc(int32_t n, int64_t nnz, const int32_t *d_rowptr,
                                      const int32_t *d_colidx, const double *d_vals,
                                      const double *d_x, const double *d_rhs, double *d_r,
                                      double *d_omega, void *stream);

/* ---- GPU model evaluation: the KKT values of one interior-point iterate.
 *
 * The step before the linear solve in every Newton iteration: evaluating
 * the Hessian of the Lagrangian and the constraint Jacobian of the ACOPF
 * problem (Eqs. 1-4, 11) at the current iterate. The paper measures model
 * evaluation at about 30 % of the CPU run time (Sec. III, cost breakdown) and
 * projects a 2x overall speedup once it runs on the GPU (Sec. IV). Model:
 * polar voltages, line flow leaving bus i on line (i, j) with admittance
 * g + jb = 1 / (r + jx), no shunts, unit taps: P = g V_i^2 - V_i V_j (g cos t
 * + b sin t), Q = -b V_i^2 - V_i V_j (g sin t - b cos t), t = theta_i -
 * theta_j; active and reactive power balance per bus (flows leaving with a
 * minus sign, generators with +1); optionally the apparent-power limits
 * P^2 + Q^2 <= S^2 at both ends of every line; objective sum c2 Pg^2.
 * Variables: x = (|V|_1..B, theta_1..B, Pg_1..G, Qg_1..G) (n_primal = 2B + 2G);
 * constraint rows: P balance 1..B, Q balance 1..B, then (with limits) the
 * from-end and to-end limit of every line. The assembled matrix is
 * K = [[H + Sigma + dw I, J^T], [J, -dc I]] (full symmetric CSR). */

enum { KKT_MODEL_FLOW_LIMITS = 1,   /* include the line-flow limit rows */
       KKT_MODEL_HOST_ONLY = 2 };    /* build the pattern only: no device memory, no assembly */

/* Build the model of a grid and its KKT sparsity pattern (host, once per
 * grid). Lines: h_from / h_to bus indices (0-based, distinct ends), series
 * resistance h_r and reactance h_x (pu, r^2 + x^2 > 0); generators: bus
 * h_gen_bus and cost coefficient h_c2. All host arrays are read and copied.
 * flags: KKT_MODEL_* bits. Unless KKT_MODEL_HOST_ONLY, allocates the model's
 * device memory on the current device (line data, summation lists, one
 * scratch array of 40 doubles per line) and uploads the line data through a
 * private stream it waits for: synchronous, like kkt_analyze.
 * Errors: KKT_E_ARG (bad index, size or flag), KKT_E_NOMEM, KKT_E_CUDA. */
kkt_status kkt_model_create(int32_t n_bus, int32_t n_branch, int32_t n_gen, const int32_t *h_from,
                            const int32_t *h_to, const double *h_r, const double *h_x,
                            const int32_t *h_gen_bus, const double *h_c2, int flags,
                            kkt_model **out);

/* The model's KKT pattern: *n rows, *n_primal, *nnz; h_rowptr (n + 1) and
 * h_colidx (nnz) may be NULL to query the sizes. Columns sorted, unique,
 * every diagonal stored (ready for kkt_analyze). Host only. */
kkt_status kkt_model_pattern(const kkt_model *m, int32_t *n, int32_t *n_primal, int64_t *nnz,
                             int32_t *h_rowptr, int32_t *h_colidx);

/* Values of K at one iterate into d_vals (device, nnz, the pattern's order):
 * d_V, d_theta (n_bus each), d_lambda (constraint multipliers, one per
 * constraint row in the order above), d_sigma (barrier diagonal, n_primal;
 * zero on angles) are device FP64 arrays; delta_w / delta_c are the primal and
 * dual regularizations. d_dual_diag (device, one per constraint row, or NULL)
 * is added to delta_c on the (2,2) diagonal, -(delta_c + d_dual_diag[r]): the
 * eliminated slacks' term s/w of the flow-limit rows in an interior-point
 * step. Deterministic (fixed summation order, no atomics). Asynchronous on
 * `stream`; calls on one model must not overlap (they share the model's
 * scratch). Errors: KKT_E_ARG, KKT_E_STATE (host-only model), KKT_E_CUDA. */
kkt_status kkt_model_assemble(const kkt_model *m, const double *d_V, const double *d_theta,
                              const double *d_lambda, const double *d_sigma, const double *d_dual_diag,
                              double delta_w, double delta_c, double *d_vals, void *stream);

/* ---- The interior-point loop around the linear solver (Sec. II: Newton's
 * method on the barrier problem, continuation mu -> 0; one K_k per iteration).
 *
 * Problem: min sum c2 Pg^2 + rho theta_ref^2 s.t. power balance c_E(x) = 0 with loads Pd, Qd,
 * line limits |S|^2 <= Smax^2 at both ends (flow-limit models; slacks s >= 0),
 * Vmin <= |V| <= Vmax, Pmin <= Pg <= Pmax, Qmin <= Qg <= Qmax (Eqs. 1-7). The
 * term rho theta_ref^2 fixes the reference angle without changing the optimal
 * cost (all else depends on angle differences), removing the uniform angle
 * shift, a null direction of K otherwise held only by delta_w.
 * Each iteration: model evaluation on the GPU (flows, constraints, K with the
 * barrier diagonal Sigma_x = zL/(x - xL) + zU/(xU - x) and the slacks' term
 * s/w), J^T lambda read off K, the optimality error
 *   E_mu = max(||grad F + J^T lambda - zL + zU||, ||c_E||, ||c_I + s - u||,
 *              ||lambda_I - w||, ||(x - xL) zL - mu||, ||(xU - x) zU - mu||,
 *              ||s w - mu||)   (infinity norms),
 * mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu)) while E_mu <= kappa_eps mu,
 * the Newton system refactored and refined by the library (kkt_refactor_refine
 * to lin_tol), the bound and slack steps recovered, and the largest step
 * <= 1 that keeps every distance to its bound above (1 - tau) times its
 * value, tau = max(tau_min, 1 - mu), separately for the primal (x, s,
 * lambda) and dual (zL, zU, w) variables. Stops when E_0 <= tol. Start: x0
 * pushed into [xL + push (xU - xL), xU - push (xU - xL)], s0 = max(u - c_I,
 * push u), lambda = 0, zL = mu0/(x - xL), zU = mu0/(xU - x), w = mu0/s0. */
typedef struct {
    double tol;          /* stop when E_0 <= tol (default 1e-7) */
    int max_iter;        /* default 200 */
    double mu0;          /* initial barrier parameter (default 0.1) */
    double kappa_eps;    /* barrier subproblem tolerance factor (default 10) */
    double kappa_mu;     /* linear decrease factor of mu (default 0.2) */
    double theta_mu;     /* superlinear decrease exponent of mu (default 1.5) */
    double tau_min;      /* fraction to the boundary, lower bound (default 0.99) */
    double delta_w;      /* primal regularization of K (default 1e-8) */
    double delta_c;      /* dual regularization of K (default 1e-8: with 1e-10 the balance rows'
                            pivots grow the factors ~1e10 and the Newton solves stall) */
    double push;         /* interior push of the starting point (default 1e-2) */
    double lin_tol;      /* backward error of every Newton solve (default 1e-10) */
    int angle_ref;       /* bus whose angle the term angle_pin * theta_ref^2 holds at 0 (default 0) */
    double angle_pin;    /* weight of that term (default 1; 0 leaves the angle shift free) */
} kkt_ipm_options;

typedef struct {
    int iters;           /* Newton iterations taken */
    int status;          /* KKT_OK (converged), KKT_E_NOCONV (max_iter), KKT_E_NUMERIC, ... */
    double objective;    /* sum c2 Pg^2 at the last iterate */
    double err;          /* E_0 at the last iterate */
    double mu;           /* final barrier parameter */
    int lin_iters;       /* FGMRES iterations over all Newton solves */
    double lin_omega_max;/* largest backward error of a Newton solve */
    int lin_noconv;      /* Newton solves that stopped above lin_tol */
} kkt_ipm_info;

void kkt_ipm_default_options(kkt_ipm_options *opt);

/* Loads and limits of the model's ACOPF instance (host arrays, read and
 * copied): h_Pd, h_Qd, h_Vmin, h_Vmax (n_bus), h_Pmin, h_Pmax, h_Qmin, h_Qmax
 * (n_gen), h_Smax (n_branch; used with flow limits). Allocates the loop's
 * device workspace (the model's only allocation besides kkt_model_create);
 * synchronous. Errors: KKT_E_ARG (null array, empty or non-finite bound
 * interval, Vmin <= 0, Smax <= 0), KKT_E_STATE (host-only model),
 * KKT_E_NOMEM, KKT_E_CUDA. */
kkt_status kkt_model_set_limits(kkt_model *m, const double *h_Pd, const double *h_Qd, const double *h_Vmin,
                                const double *h_Vmax, const double *h_Pmin, const double *h_Pmax,
                                const double *h_Qmin, const double *h_Qmax, const double *h_Smax);

/* Run the interior-point loop on the model (after kkt_model_set_limits).
 * ctx: a single-instance context analysed for the model's own pattern
 * (kkt_model_pattern), of either precision; every Newton system goes
 * through kkt_refactor_refine on it. d_x (device, n_primal = (|V|, theta,
 * Pg, Qg)): the starting point in, the last iterate out; d_lam (device, one
 * per constraint row): the constraint multipliers out. info (may be NULL)
 * receives the counts and errors. Synchronous on `stream`.
 * Returns KKT_OK on convergence, KKT_E_NOCONV after max_iter, KKT_E_NUMERIC on
 * NaN or a zero step, KKT_E_ARG (sizes of ctx and model differ, bad option),
 * KKT_E_STATE (no limits set), or the status of a failed Newton solve. */
kkt_status kkt_ipm_solve(kkt_model *m, kkt_ctx *ctx, const kkt_ipm_options *opt, double *d_x, double *d_lam,
                         kkt_ipm_info *info, void *stream);

kkt_status kkt_model_destroy(kkt_model *m);

/* Failure-injection hook for tests (no counterpart in the paper): the next
 * refactorization's first unit of the persistent tree kernel waits on a flag
 * that nothing sets, so its bounded wait (kkt_options.spin_limit polls)
 * expires; the kernel then stops every other unit, and the refactorization
 * reports KKT_E_TIMEOUT through kkt_get_info and kkt_refine. The context stays
 * usable: the refactorization after it runs normally. Synchronous.
 * Errors: KKT_E_ARG, KKT_E_STATE (the context has no tree part), KKT_E_CUDA. */
kkt_status kkt_debug_stall(kkt_ctx *ctx);

/* Test hook for the pivot reciprocal (no counterpart in the paper): d_out[i] =
 * the value every factorization and back-substitution kernel uses for 1 /
 * d_in[i] (multiplying by it replaces the division by the pivot u_pp of Alg. 1's
 * factorization and triangular solves). d_in, d_out: device arrays of n
 * elements, FP64 for precision = KKT_FP64 and FP32 for KKT_FP32_IR; they may
 * be the same array. Stated bound: within one unit in the last place of the
 * correctly rounded 1 / d; the IEEE division itself for |d| outside
 * [2^-1000, 2^1000] (FP32: [2^-100, 2^100]), zero, infinities and NaN.
 * Asynchronous on `stream`. Errors: KKT_E_ARG (n < 0, a null pointer with n >
 * 0, unknown precision, n beyond one launch), KKT_E_CUDA. */
kkt_status kkt_debug_pivot_rcp(const void *d_in, void *d_out, int64_t n, int precision, void *stream);

/* Profiling mode: when on, every launch group is bracketed by a pair of CUDA
 * events on its stream (adds a little host overhead). */
kkt_status kkt_set_profiling(kkt_ctx *ctx, int on);

/* Synchronize, aggregate the event pairs recorded since the last call per
 * kernel, write up to max_out entries and reset. Returns the number of
 * entries written, or -1 on error. */
int kkt_kernel_stats(kkt_ctx *ctx, kkt_kernel_stat *out, int max_out);
kkt_status kkt_get_plan(const kkt_ctx *ctx, kkt_plan_info *info);

/* Elimination order chosen by the analysis (after postordering):
 * h_perm[k] = original index eliminated k-th (n entries, host). */
kkt_status kkt_get_perm(const kkt_ctx *ctx, int32_t *h_perm);

/* Equilibration factors d of the last refactor (n FP64, host). Synchronous. */
kkt_status kkt_get_scaling(const kkt_ctx *ctx, double *h_d);

/* Export the factors of the last refactor as coordinate lists keyed by
 * ORIGINAL indices, for checking: every stored entry (amalgamation zeros
 * included) of L (strictly lower, unit diagonal implied) and of U (upper,
 * diagonal included) of P (D K D) P^T, widened to FP64. h_*_row/col are
 * original row/column indices. Pass NULL arrays to query the counts only
 * (*nl, *nu). Synchronous.
 * Errors: KKT_E_ARG, KKT_E_STATE, KKT_E_CUDA. */
kkt_status kkt_export_factors(const kkt_ctx *ctx, int64_t *nl, int32_t *h_l_row, int32_t *h_l_col,
                              double *h_l_val, int64_t *nu, int32_t *h_u_row, int32_t *h_u_col,
                              double *h_u_val);

kkt_status kkt_destroy(kkt_ctx *ctx);

const char *kkt_status_string(kkt_status s);

/* ---- Saddle-point specialised solve (Sec. V) ------------------------------
 * Sec. V names a solver specialised to the saddle-point structure of these
 * KKT systems as a way forward, without giving its method. This is the hybrid
 * direct-iterative approach of the GPU ACOPF literature. With the unknowns
 * ordered (x, y_E, y_I) -- n_primal primal, then m_eq equality duals, then
 * the rest, inequality duals -- and K = [H J_E^T J_I^T; J_E -D_E 0; J_I 0 -D_I]
 * with D_E, D_I diagonal (stored, every dual row's diagonal present):
 *   H_g = H + J_I^T D_I^{-1} J_I + gamma J_E^T J_E   (factored by an inner
 *          context of this library: multifrontal LU, FP64, static pivoting),
 *   (C^{1/2} J_E H_g^{-1} J_E^T C^{1/2} + D_E) w = C^{1/2} (J_E H_g^{-1} r'' - r_E)
 *          by conjugate gradients, C = I - gamma D_E, y_E = C^{-1/2} w,
 *   x = H_g^{-1} (r'' - J_E^T C y_E), y_I = D_I^{-1} (J_I x - r_I),
 * with r'' = r_x + J_I^T D_I^{-1} r_I + gamma J_E^T r_E. gamma trades the
 * conjugate-gradient iterations against the conditioning of H_g; it must make
 * the reduced operator positive definite (H_g need not be). */
typedef struct kkt_hykkt kkt_hykkt;

typedef struct {
    int cg_iters;               /* conjugate-gradient iterations */
    int status;                 /* KKT_OK, or KKT_E_NOCONV if cg_resid > tol at max_iter */
    int n_perturbed;            /* static pivot perturbations of the factorization of H_g */
    int launches;               /* kernels this call launched, the inner factorization's and solves' included */
    double cg_resid;            /* ||b' - A w|| / ||b'|| of the reduced system at exit */
    double backward_err;        /* ||K z - b||_inf / (||K||_inf ||z||_inf + ||b||_inf) */
} kkt_hykkt_info;

/* Analysis from the host CSR pattern of K (n x n, structurally symmetric,
 * 0-based, sorted or not): the blocks, the pattern of H_g with, per entry, its
 * contributions in a fixed order, and the inner context's analysis of H_g.
 * gamma >= 0 (finite). Synchronous.
 * Errors: KKT_E_ARG, KKT_E_STRUCT (the (2,2) block is not diagonal or a dual
 * diagonal is missing), KKT_E_NOMEM, KKT_E_CUDA. */
kkt_status kkt_hykkt_analyze(int32_t n, int32_t n_primal, int32_t m_eq, const int32_t *h_rowptr,
                             const int32_t *h_colidx, double gamma, kkt_hykkt **out);

/* z = K^{-1} b by the method above for K's values d_vals (device, nnz FP64 in
 * the CSR order given to the analysis); d_rhs, d_z device FP64 vectors of
 * length n, not aliased. Stops when the reduced residual is <= tol times its
 * initial value or after max_iter iterations. Synchronizes `stream` (the host
 * reads the reduced residual after every iteration); info may be NULL.
 * Errors: KKT_E_ARG (also for d_z == d_rhs), KKT_E_NUMERIC (some d_I <= 0, gamma d_E >= 1, or NaN),
 * KKT_E_NOCONV (z written, info filled), KKT_E_CUDA. */
kkt_status kkt_hykkt_solve(kkt_hykkt *h, const double *d_vals, const double *d_rhs, double *d_z, double tol,
                           int32_t max_iter, kkt_hykkt_info *info, void *stream);

/* The inner context that factors H_g, borrowed: owned by h and valid until
 * kkt_hykkt_destroy(h). For kkt_get_plan, kkt_get_info, kkt_set_profiling and
 * kkt_kernel_stats only; the caller must not destroy, refactor or solve with it.
 * Errors: KKT_E_ARG. */
kkt_status kkt_hykkt_inner(kkt_hykkt *h, kkt_ctx **out);

void kkt_hykkt_destroy(kkt_hykkt *h);

#ifdef __cplusplus
}
#endif
#endif /* KKT_GB300_H */
