/*
 * gpfvm.h -- C ABI of the GB300-native GP-FVM hot path.
 *
 * GP-FVM conditions a Gaussian-process prior on finite-volume observations of
 * a linear PDE plus initial/boundary data (Weiland, Pfoertner, Hennig,
 * "Scaling up Probabilistic PDE Simulators with Structured Volumetric
 * Information").  This library implements, on one GPU:
 *   - the 1D factor matrices of the tensor-product Matern-5/2 prior under
 *     interval functionals (Sec. 3.1, Eq. linop-simplified; Sec. 3.2, Eq. LkL);
 *   - the Kronecker-structured Gram matvec of the volume observations
 *     (Sec. 4.1, Eq. kronecker-structure) and the point-set blocks;
 *   - the Cholesky (IC/BC) deflation of Sec. 4.2 and CG with the IterGP
 *     combined posterior (Sec. 4.1) with full reorthogonalisation (Sec. 7);
 *   - posterior mean and variance on a tensor prediction grid
 *     (Sec. 2.1, Eqs. lin-cond-mean / lin-cond-cov).
 *
 * Conventions
 *   - Axes are ordered (t, x, y); ndim is 1, 2 or 3.  Tensors over cells,
 *     point sets and the prediction grid are row-major in axis order (the
 *     last axis is contiguous).
 *   - Pointers in descriptors are HOST pointers; the library copies them in
 *     gpfvm_create and the caller keeps ownership.  Vector arguments of the
 *     compute calls are DEVICE pointers unless the name says _host.
 *   - Every call that takes `stream` enqueues its work on that cudaStream_t
 *     (NULL = legacy default stream).  Calls that return solver status
 *     synchronise the stream before returning.
 *   - Return codes: 0 = success, +1 = iteration budget exhausted before the
 *     tolerance (a result is still written), negative = error (see
 *     gpfvm_strerror).  On error nothing is written to outputs.
 *   - A problem handle is not thread-safe; distinct handles are independent.
 *
 * Environment switches
 *   - GPFVM_ICBC=dense (read by gpfvm_create): invert G_BB by a dense
 *     Cholesky instead of the structured stage (eigenbasis of the largest
 *     IC/BC set + Schur complement of the others); both give the same
 *     posterior.
 *   - GPFVM_HOST_LOOP=1 (read by gpfvm_create): CG runs are replayed pass by
 *     pass from the host instead of a device-side graph loop (same kernels
 *     and results; for per-kernel profilers).
 *   - GPFVM_LOOP_UNROLL=k (1..8, default 2; read once per process): CG
 *     iterations per pass of a device-side loop.
 *   - GPFVM_PERSIST=1 (read once per process): Gram operators run as one
 *     cooperative launch each (bit-identical results; slower on the
 *     measured workloads).
 */
#ifndef GPFVM_H
#define GPFVM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPFVM_MAX_DIM 3
#define GPFVM_MAX_TERMS 16
#define GPFVM_MAX_SETS 8
#define GPFVM_MAX_OUTPUTS 4

enum gpfvm_status {
  GPFVM_OK = 0,
  GPFVM_NOT_CONVERGED = 1,
  GPFVM_ERR_INVALID_ARG = -1,  /* descriptor or argument rejected by validation */
  GPFVM_ERR_OUT_OF_MEMORY = -2,/* device allocation failed or memory budget exceeded */
  GPFVM_ERR_NOT_SPD = -3,      /* Cholesky pivot <= 0 in the IC/BC Gram matrix */
  GPFVM_ERR_BREAKDOWN = -4,    /* CG breakdown: p^T G p <= 0 or not finite */
  GPFVM_ERR_DEVICE = -5,       /* a CUDA call failed */
  GPFVM_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
  GPFVM_ERR_STATE = -7,        /* call out of order (e.g. solve before assemble) */
  GPFVM_ERR_NOT_FOUND = -8,    /* unknown ticket */
  GPFVM_ERR_TOO_LARGE = -9     /* request exceeds the fixed capacity of gpfvm_kron_matvec_noalloc */
};

/* One tensor grid of point functionals  d^order u (x)  (Sec. 2.2: initial and
 * boundary data as linear functionals).  order[i] in {0,1} is the derivative
 * order along axis i (e.g. order = {1,0,0} observes u_t, a Neumann wall on x
 * uses {0,1,0}).  The grid has prod n_pts points; `values` lists the
 * observed values row-major over the per-axis coordinate lists (NULL = all
 * zero).  noise_var > 0 is the Gaussian noise variance of each value. */
typedef struct {
  int order[GPFVM_MAX_DIM];
  int n_pts[GPFVM_MAX_DIM];
  const double* coords[GPFVM_MAX_DIM];
  const double* values;
  double noise_var;
} gpfvm_point_set;

/* A linear IBVP discretised by a factorized box scheme (Sec. 4.1, Definition
 * of factorized structure) under a tensor-product Matern-5/2 prior
 * (Eq. tensorproduct-cov-def).
 *   edges[i]       n_cells[i]+1 strictly increasing cell edges of axis i;
 *                  every cell of the tensor grid is one volume observation
 *                  int_V D[u] = rhs  (Eq. linop-def).
 *   alpha, coef    D = sum_k coef[k] d^alpha[k]  (Eq. multi-input-fv), each
 *                  alpha[k][i] in {0,1,2}.
 *   lengthscale    per-axis Matern-5/2 lengthscales; outputscale multiplies
 *                  the product kernel once.
 *   rhs            N = prod n_cells volume integrals of the forcing f,
 *                  row-major (NULL = homogeneous PDE).
 *   jitter         noise variance added to every volume observation.
 *   sets           initial/boundary point sets (the Cholesky-deflated part).
 *   pred           per-axis coordinates of the tensor prediction grid.
 *   observe        0: finite volumes (the PDE integrated over every cell);
 *                  1: collocation (Sec. 3, the operator D[u](x)): the PDE at
 *                  the centre of every cell, rhs then holding point values of
 *                  the forcing; the same Kronecker structure with point
 *                  factors (kernel derivatives up to order 4).
 *   coef_field     per term NULL (constant coefficient) or N values, one per
 *                  cell row-major, multiplying coef[k]: a piecewise-constant
 *                  variable coefficient (App. C.4, variable bathymetry).
 *                  Every Kronecker term of the Gram matrix then becomes its
 *                  Hadamard product with the rank-one matrix of the two terms'
 *                  coefficients, applied as diagonal scalings.  Terms passing
 *                  the same pointer share one field.  Such problems run the
 *                  FP64 and FP32 SIMT operators (no tensor-core precisions).
 *   fp64_products  0: the FP64 CG iteration and the FP64 residual of the mixed
 *                  solves apply G_PP on the tensor cores by exact digit
 *                  products (FP64 matrix-product accuracy; every axis <= 128
 *                  cells and constant coefficients, else FP64 FMA); 1: always
 *                  FP64 FMA (SIMT) mode products.  Ops 0/1 of gpfvm_gram_matvec
 *                  are FP64 FMA and ops 12/13 the digit-product form either way.
 *   n_outputs      0: one equation on one output u (term_eq, term_out and
 *                  set_out are not read).  >= 1 (at most GPFVM_MAX_OUTPUTS): a
 *                  system in u = (u_0 .. u_{n_outputs-1}) with independent
 *                  priors of the same hyperparameters (Sec. 3.3, Eq.
 *                  multioutput-cov-def).  Term k belongs to equation
 *                  term_eq[k] and differentiates component term_out[k]
 *                  (Sec. 3.3: an operator sum_alpha sum_i c_{alpha,i} D^alpha
 *                  u_i); the equations are numbered 0 .. n_eq - 1 without
 *                  gaps, and every cell yields one observation per equation.
 *                  Set s observes component set_out[s].  With n_outputs = 1
 *                  and one equation this is the one-output problem.  Vectors over the PDE
 *                  observations (rhs, gram_matvec, the CG directions) hold
 *                  n_eq blocks of prod n_cells, equation-major; the prediction
 *                  grid is evaluated for every output, output-major (P =
 *                  n_outputs prod n_pred).  Such systems are solved in FP64
 *                  with FMA mode products and the dense IC/BC stage (no
 *                  mixed precisions, coefficient fields, multigrid start,
 *                  targeted actions, batches or server). */
typedef struct {
  int ndim;
  int n_cells[GPFVM_MAX_DIM];
  const double* edges[GPFVM_MAX_DIM];
  double lengthscale[GPFVM_MAX_DIM];
  double outputscale;
  int n_terms;
  int alpha[GPFVM_MAX_TERMS][GPFVM_MAX_DIM];
  double coef[GPFVM_MAX_TERMS];
  const double* rhs;
  double jitter;
  int n_sets;
  gpfvm_point_set sets[GPFVM_MAX_SETS];
  int n_pred[GPFVM_MAX_DIM];
  const double* pred[GPFVM_MAX_DIM];
  int observe;
  const double* coef_field[GPFVM_MAX_TERMS];
  int fp64_products;
  int n_outputs;
  int term_eq[GPFVM_MAX_TERMS];
  int term_out[GPFVM_MAX_TERMS];
  int set_out[GPFVM_MAX_SETS];
} gpfvm_desc;

/* Precision of the CG iteration. */
enum gpfvm_precision {
  GPFVM_FP64 = 0,        /* every product and vector in FP64 */
  GPFVM_MIXED_FP32 = 1,  /* iterative refinement: FP64 residual b - G^ x with the FP64
                            operator; inner CG on an FP32 operator (FP32 SIMT mode
                            products, FP32 vectors) with FP64 scalars and reductions */
  GPFVM_MIXED_TF32X3 = 2, /* as MIXED_FP32, with the G_PP mode products on tcgen05 tensor
                            cores in split TF32 (hi*hi + hi*lo + lo*hi, FP32 accumulate) */
  GPFVM_MIXED_BF16X3 = 3, /* as MIXED_TF32X3 with split bf16 operands (tcgen05 kind::f16:
                            hi = bf16(x), lo = bf16(x - hi), three products, FP32 accumulate) */
  GPFVM_MIXED_BF16 = 4    /* as MIXED_BF16X3 with one bf16 product (hi*hi) */
};

typedef struct {
  int max_iter;        /* iteration budget (>= 1); also sizes the stored directions */
  double rtol;         /* stop when ||b - G^ x|| / ||b|| <= rtol (recursive residual) */
  int precision;       /* enum gpfvm_precision */
  int reorth;          /* 1 = full G^-conjugate reorthogonalisation of directions (mixed: one
                          conjugate set across all refinement runs, stores for every run);
                          2 = mixed only: within each run (stores for one run, the variance
                          from the first run's actions); 0 = none */
  int want_var;        /* 1 = accumulate the IterGP variance downdate on the grid */
  int check_every;     /* unused (kept for layout): every CG run is one device-side loop */
  int inner_max_iter;  /* mixed: iteration cap of one inner CG run, i.e. the period of the FP64
                          residual replacement (<= 0: no cap beyond max_iter) */
  double inner_rtol;   /* mixed: residual reduction of one inner CG run (<= 0: 1e-2) */
  int inner_reorth_first; /* unused (kept for layout): with reorth every inner run continues one
                             G^-conjugate direction set (see gpfvm_solve) */
  int coarse;          /* FP64 with reorth: multigrid warm start (appendix "Multigrid
                          preconditioners") on coarse cells of coarse^ndim fine cells (every
                          n_cells divisible by it, at most 4096 coarse cells): the coarse FVM
                          observations are conditioned on exactly (Cholesky of W^T G^ W) and
                          become the first stored actions, before CG on the fine cells;
                          0 or 1 = off.  max_iter counts CG iterations only, and the problem's
                          direction capacity must hold both. */
} gpfvm_solve_opts;

typedef struct {
  int iterations;      /* CG iterations taken */
  int status;          /* same code as the return value */
  double rel_residual; /* recursive ||r||/||b|| at exit */
  double true_rel_residual; /* FP64 ||b - G^ x||/||b|| recomputed at exit */
  double t_assemble_ms, t_solve_ms, t_query_ms; /* device time per phase (CUDA events) */
  double latency_ms;   /* server only: host wall time from submit to result */
} gpfvm_solve_info;

typedef struct gpfvm_problem gpfvm_problem;

/* Validates and copies the descriptor, allocates device memory for the whole
 * solve (factors, IC/BC matrices, CG state with room for max_iter stored
 * directions, prediction outputs).  max_iter <= 0 selects 2000.  Errors:
 * INVALID_ARG (bad sizes, orders, non-increasing edges, lengthscale <= 0,
 * observe not 0 or 1), OUT_OF_MEMORY. */
int gpfvm_create(const gpfvm_desc* desc, int max_iter, gpfvm_problem** out);

/* Frees every device and host resource of the problem (NULL is a no-op). */
void gpfvm_destroy(gpfvm_problem* p);

/* Sizes: out[0] = N volumes, out[1] = M point observations, out[2] = P
 * prediction points, out[3] = direction capacity. */
int gpfvm_sizes(const gpfvm_problem* p, int64_t out[4]);

/* Setup (Sec. 4.1 "precompute the 1D factors", Sec. 4.2): assembles all 1D
 * factor matrices (FP64 closed forms), the dense IC/BC Gram matrix G_BB,
 * its Cholesky factor and explicit inverse factor L^-1, and the conditioned
 * right-hand side  b = y_PDE - G_PB G_BB^-1 y_B.  Errors: NOT_SPD, DEVICE. */
int gpfvm_assemble(gpfvm_problem* p, void* stream);

/* Structured Gram products on device vectors (for parity tests and the
 * matvec benchmark):
 *   op 0: out = G_PP v            (N -> N, Eq. kronecker-structure + jitter)
 *   op 1: out = G^ v = G_PP v - G_PB G_BB^-1 G_BP v   (N -> N, Sec. 4.2)
 *   op 2: out = G_BP v            (N -> M)
 *   op 3: out = G_PB v            (M -> N)
 *   op 4: out = G_PP v in the FP32 form of the mixed solver (FP64 in/out)
 *   op 5: out = G_PP v in the split-TF32 tensor-core form (FP64 in/out)
 *   op 6: out = G^ v, the inner operator of GPFVM_MIXED_FP32 (FP32, FP64 in/out)
 *   op 7: out = G^ v, the inner operator of GPFVM_MIXED_TF32X3 (FP64 in/out)
 *   op 8 / op 9: G_PP / G^ (inner operator) in split bf16 (GPFVM_MIXED_BF16X3)
 *   op 10 / op 11: G_PP / G^ (inner operator) in one bf16 product (GPFVM_MIXED_BF16)
 *   op 12 / op 13: G_PP / G^ in FP64 with the G_PP mode products computed on
 *                  the bf16 tensor cores by exact digit products (every row of
 *                  an operand split into 8 balanced 7-bit digits, the digit
 *                  products accumulated exactly in FP32 and recombined in
 *                  64-bit integers; the splitting of Ozaki et al. 2012):
 *                  GPFVM_ERR_INVALID_ARG where an axis has more than 128 cells
 *                  or a coefficient field is given
 * Ops 6, 7, 9 and 11 use the mixed solver's FP32 work vectors: not between the
 * begin and end of a solve on the same problem.  Requires gpfvm_assemble.  v and out must not overlap. */
int gpfvm_gram_matvec(gpfvm_problem* p, int op, const double* v, double* out, void* stream);

/* As gpfvm_gram_matvec (same ops, device pointers), for measurement: the
 * op's launch sequence is captured once as a CUDA graph, replayed 2 + reps
 * times, and *ms_per_application receives the device time of one application
 * (CUDA events around the reps replays on the problem's stream).  out holds
 * the result.  reps >= 1.  Errors as gpfvm_gram_matvec. */
int gpfvm_gram_matvec_bench(gpfvm_problem* p, int op, const double* v, double* out, int reps, void* stream,
                            double* ms_per_application);

/* CG / IterGP on the deflated system (Sec. 4.1, 4.2), x0 = 0.  max_iter
 * counts CG iterations (for the mixed precisions: inner iterations).  All scalars
 * stay on the device; a whole CG run is one CUDA graph launch whose WHILE node
 * repeats the captured iteration until the device state reports convergence,
 * breakdown or max_iter (bounded by max_iter + 2 passes in any case), so the
 * host reads the state once per run.  Returns OK, NOT_CONVERGED
 * (budget exhausted; the iterate and variance downdate are kept), BREAKDOWN,
 * STATE (not assembled) or DEVICE.  info may be NULL.
 * Mixed precisions: inner CG runs on the FP32 (or tensor-core) operator
 * with FP64 scalars, separated by FP64 residual replacements r = b - G^ x.
 * With reorth the runs continue ONE G^-conjugate direction set: each run
 * starts with the Galerkin projection of its residual onto all stored
 * directions and makes every new direction conjugate to them, so with an
 * exact operator the iterates are those of the FP64 recurrence and the
 * IterGP downdate sums over the directions of all runs (the same actions).
 * A run stops at inner_rtol, at inner_max_iter, or where its recurrence
 * reaches rtol; the solve ends when the FP64 residual is <= rtol (or <= 2
 * rtol right after a run that aimed at rtol: the FP32 recurrence's estimate)
 * or max_iter iterations are spent.  Without reorth the runs are independent
 * refinement steps and the downdate uses the first run's directions. */
int gpfvm_solve(gpfvm_problem* p, const gpfvm_solve_opts* opts, gpfvm_solve_info* info,
                void* stream);

/* Posterior on the prediction grid (device outputs of P doubles each):
 *   mean = k_B(X*)^T G_BB^-1 (y_B - G_BP x) + L_PDE k(X*)^T x
 *   var  = k(x,x) - ||L^-1 k_B(x)||^2 - sum_j (Lhat k(x)^T p_j)^2 / eta_j
 * var may be NULL; a variance needs want_var in the preceding solve. */
int gpfvm_query(gpfvm_problem* p, double* mean, double* var, void* stream);

/* Mode-product autotuner (an addition of this library; the paper has no
 * counterpart).  Times the solver operator of `precision` on this problem
 * (graph replays on `stream`) under each candidate plan policy -- the row
 * tile of the SIMT mode-product GEMMs (the size heuristic, or always 64, 32
 * or 16 rows) and, for the tensor-core precisions, with and without the
 * segment grouping of idle levels -- rebuilds the problem's plans with the
 * fastest and caches that choice per (precision, operator terms, axis sizes
 * rounded up to 16), so that later problems of the same size class take it
 * without timing.  Results are unchanged up to the summation order of the
 * split levels.  report (may be NULL) receives up to report_cap doubles: the
 * ms of each timed candidate, then the choice (3 (tile + 1) + grouping off).
 * Returns 0 (timed), 1 (taken from the cache) or an error (STATE before
 * gpfvm_assemble).  Allocates two N-vectors while timing. */
int gpfvm_autotune(gpfvm_problem* p, int precision, void* stream, double* report, int report_cap);

/* Targeted uncertainty reduction (appendix "Targeted uncertainty reduction"):
 * continues the IterGP state of the last solve with n_actions more actions,
 * each aimed at a weighted set of prediction points.  beta is a DEVICE array
 * of n_actions x P doubles, row a holding the weights of action a on the
 * prediction grid (row-major like the grid; in the appendix a Dir(1, ..., 1)
 * sample over the target points and zero elsewhere -- the caller draws it).
 * Action a takes t = Lhat k(X*) beta_a, the residual s = t - G^ C t of that
 * system with respect to the inverse approximation C = sum_j p_j p_j^T/eta_j
 * of every earlier action (so the actions run CG on the target system), and
 * its conjugate direction d = s - C G^ s; then C += d d^T/(d^T G^ d), the
 * iterate x = C b moves by d (d^T r)/(d^T G^ d), and the variance downdate by
 * (Lhat k(X*)^T d)^2/(d^T G^ d).  A following gpfvm_query returns the
 * refined mean and variance.  Requires a preceding FP64 gpfvm_solve with
 * reorth and want_var (STATE otherwise) and room for the new directions
 * (stored directions + n_actions <= the max_iter given to gpfvm_create, else
 * INVALID_ARG).  BREAKDOWN if an action adds no new direction (d^T G^ d <= 0). */
int gpfvm_target(gpfvm_problem* p, const double* beta, int n_actions, void* stream);

/* One call doing assemble + solve + query with HOST input/output buffers:
 * copies the point-set values (M doubles, may be NULL to keep the
 * descriptor's) host->device, solves and copies mean/var (P doubles each;
 * var may be NULL) device->host.  This is the end-to-end path of a user. */
int gpfvm_solve_host(gpfvm_problem* p, const double* values_host, const gpfvm_solve_opts* opts,
                     double* mean_host, double* var_host, gpfvm_solve_info* info, void* stream);

/* Replaces the observed values of all point sets (M doubles, DEVICE pointer,
 * ordered set by set as in the descriptor) and recomputes the conditioned
 * right-hand side.  Geometry, factors and the IC/BC Cholesky stay valid, so a
 * new initial condition on the same grid needs no re-assembly.  Requires
 * gpfvm_assemble. */
int gpfvm_set_values(gpfvm_problem* p, const double* values, void* stream);

/* Number of kernels this library has launched in the process so far (graph
 * replays count every kernel node).  Used to report launch counts. */
int64_t gpfvm_launch_count(void);

/* Copies internal device arrays to a HOST buffer for inspection:
 *   what 0: conditioned rhs b (N)      what 1: CG iterate x (N)
 *   what 2: G_BB with noise (M*M)      what 3: L^-1 (M*M, lower)
 *   what 4: 1D factor (axis, kind_a, ord_a, kind_b, ord_b) -- see gpfvm_factor
 *   what 5: variance downdate sum (P)  what 6: eta_j (iterations)
 *   what 7: device time (ms) of the last assemble, solve and query (3 values)
 *   what 8: refinement steps of the last mixed-precision solve (1 value)
 *   what 9: eigensolver sweeps of the structured IC/BC stage, (FP32, FP64)
 *           per axis (2 * ndim values; 0 written without that stage)
 *   what 10: IC/BC stage layout: (structured 1 / dense 0, rows of the set
 *           inverted through its eigen-structure, rows of the Schur block)
 *   what 11: the stored directions p_j of the last solve with reorth (k rows
 *           of N; FP32 stores of the mixed precisions widened to doubles)
 *   what 12: eta_j = p_j^T G^ p_j of those k directions (k values)
 * Returns the number of doubles written or a negative error. */
int64_t gpfvm_export(gpfvm_problem* p, int what, double* host_out, int64_t capacity, void* stream);

/* A 1D covariance factor as assembled on the device (unit output scale):
 * rows = functional family A, cols = family B on axis `axis`.  kind 0 =
 * cell family with derivative order ord (0 integral, 1 difference of values,
 * 2 difference of first derivatives: Eq. linop-simplified); kind 1 = point
 * set `set` with its order on that axis; kind 2 = prediction points.
 * Writes rows*cols doubles row-major to host_out. */
int64_t gpfvm_factor(gpfvm_problem* p, int axis, int kind_a, int arg_a, int kind_b, int arg_b,
                     double* host_out, int64_t capacity, void* stream);

/* ------------------------------------------------------------------------
 * Batched execution: many independent problems of uneven sizes advanced
 * together.  Each problem must be created and assembled.  Every problem runs
 * on its own stream, each CG run as one device-side loop (graph WHILE node),
 * so the problems overlap on the device; the host only advances the
 * refinement steps of problems whose streams are idle.  Returns the worst
 * status; infos (may be NULL) receives one entry per problem.
 * ------------------------------------------------------------------------ */
int gpfvm_solve_batch(gpfvm_problem** ps, int n, const gpfvm_solve_opts* opts,
                      gpfvm_solve_info* infos, void* stream);

/* The same batch as ONE graph launch: every problem's whole solve is a
 * device-driven loop (a WHILE node whose body computes the FP64 residual,
 * takes the refinement decision on the device, runs the inner CG as a nested
 * WHILE node and applies the correction; an FP64 problem's body is its CG
 * iteration), all problems' loops are independent branches of one graph, and
 * the host only sets them up before and reads their states after.  Results
 * equal gpfvm_solve_batch's (the same kernels and decisions).  The direction
 * stores cannot grow inside a graph, so they are allocated up front: for
 * every run (up to max_iter directions) with reorth 1, for one run
 * (inner_max_iter) with reorth 0 or 2 -- use reorth 2 when max_iter directions
 * of every problem do not fit.  *launches_out (may be NULL) receives the
 * kernels executed.  Problems must be distinct. */
int gpfvm_solve_batch_graph(gpfvm_problem** ps, int n, const gpfvm_solve_opts* opts, gpfvm_solve_info* infos,
                            void* stream, int64_t* launches_out);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching loop.  Requests are admitted into slots as
 * device memory and slots free up, their CG state stays resident, and their
 * device-side CG loops overlap with those of requests already running.
 * ------------------------------------------------------------------------ */
typedef struct gpfvm_server gpfvm_server;

typedef struct {
  int max_slots;            /* requests resident at once */
  int64_t memory_budget;    /* bytes of device memory the server may hold (0 = 90% of free) */
  gpfvm_solve_opts solve;   /* per-request solver options */
  int steps_per_tick;       /* unused (kept for layout): CG runs are device-side loops */
} gpfvm_server_opts;

int gpfvm_server_create(const gpfvm_server_opts* opts, gpfvm_server** out);
/* Queues a request (descriptor copied); returns its ticket (>= 0) in *ticket. */
int gpfvm_server_submit(gpfvm_server* s, const gpfvm_desc* desc, int64_t* ticket);
/* One scheduling pass: admits queued requests, advances every request whose
 * stream is idle (next refinement step, or retire with its result) and
 * returns without waiting for running loops (it sleeps ~50 us when nothing
 * advanced).  Returns the number of requests still queued or running. */
int gpfvm_server_step(gpfvm_server* s);
/* If the request is done, copies mean/var (host, P each; var may be NULL) and
 * its info, returns OK/NOT_CONVERGED or its error; returns 2 if still pending. */
int gpfvm_server_poll(gpfvm_server* s, int64_t ticket, double* mean_host, double* var_host,
                      gpfvm_solve_info* info);
void gpfvm_server_destroy(gpfvm_server* s);

/* ------------------------------------------------------------------------
 * Allocation-free Kronecker Gram matvec.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they
 * need the product -- frameworks whose allocator owns the whole device and
 * refuse foreign allocations, real-time loops that must not enter the
 * driver's allocator (a cudaMalloc can synchronise the device).  It computes
 *   out = scale * sum_k coef[k] (F[k][0] (x) ... (x) F[k][ndim-1]) v + diag * v
 * for a row-major tensor of dims n[0..ndim) (ndim 1..3), where F[k][i] =
 * factors[k*ndim + i] is a DEVICE pointer to an n[i] x n[i] row-major matrix
 * (for instance a 1D factor exported by gpfvm_factor), coef is a HOST array
 * of n_terms (<= 64) coefficients, and v, out are DEVICE vectors of prod n
 * doubles that must not overlap.
 * Memory: it calls no cudaMalloc/cudaFree or allocating routine.  The
 * intermediates (at most 4,194,304 doubles = 32 MiB; a three-axis product
 * needs (distinct last-axis factors + distinct first-axis factors) * prod n
 * doubles) and the argument tables live in file-scope device arrays that
 * every GPU loading the library keeps until the process exits; larger
 * requests return GPFVM_ERR_TOO_LARGE without launching anything.  The
 * argument tables travel as a by-value kernel parameter, so no host memory is
 * read after the call returns.
 * The first call on a device looks up those arrays' device addresses with
 * that device current (serialised across host threads).
 * All calls share the arrays and leave the last call's contents behind
 * (nothing in them needs to start at zero); calls that overlap on the GPU
 * (different streams, or host threads racing) race on them.  The work is
 * enqueued on `stream`; the call returns without synchronising. */
int gpfvm_kron_matvec_noalloc(int ndim, const int* n, int n_terms, const double* const* factors,
                              const double* coef, double scale, double diag, const double* v, double* out,
                              void* stream);

const char* gpfvm_strerror(int code);

/* Library build identification (architecture string and version). */
const char* gpfvm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPFVM_H */
