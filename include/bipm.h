/*
 * bipm — batched primal-dual interior-point solver for many small NLPs on one
 * GB300 (sm_103a).  C ABI.
 *
 * The problem class is the parametric NLP of Sec. III, Eq. 1 of "Scaling
 * Nonlinear Optimization: Many Problems One GPU":
 *     min_x f(x, theta)  s.t.  c(x, theta) = 0,  x_L <= x <= x_U,
 * batched as in Eq. 2: a batch holds many instances that share f, c and the
 * bounds and differ only in their parameter vector theta_i.  Each call below
 * advances or reads every instance ("slot") of one batch.
 *
 * The built-in problem family is quadrotor NMPC (Sec. VI): nq rigid-body
 * quadrotors (12 states, 4 rotor thrusts each), RK4 multiple shooting over N
 * intervals, a quadratic tracking cost, thrust bounds, and squared-distance
 * inequalities written with slacks (spheres, vertical cylinders, pairwise
 * separation).
 *
 * Layouts (one problem; double precision):
 *   theta : xbar (12 nq) | reference circles (6 nq: cx, cy, cz, radius, rate,
 *           phase; radius 0 = fixed goal) | spheres (4 n_spheres: cx, cy, cz, r) |
 *           cylinders (3 n_cylinders: cx, cy, r) | moving spheres (7 n_moving:
 *           cx, cy, cz, r, vx, vy, vz; centre at time t: c + v t)
 *   x     : for k = 0..N: x_k (12 nq), then u_k (4 nq) if k < N, then s_k (ni)
 *           if k >= 1; n = 12nq(N+1) + (4nq + ni) N
 *   y     : x_0 - xbar (12 nq), then for k = 0..N-1: dynamics rows
 *           x_{k+1} - F(x_k, u_k) (12 nq), then stage-(k+1) inequality rows
 *           (ni); m = 12nq(N+1) + ni N
 *   ni    : nq * (n_spheres + n_cylinders + n_moving) + (pair_dist > 0 ? nq(nq-1)/2 : 0),
 *           in that order (obstacle rows quadrotor-major, pairs last)
 *
 * Ownership: the batch owns all device memory it uses; caller buffers are
 * only read or written during the call.  `on_device` = 1 means the pointer is
 * a device pointer valid on the batch's stream, 0 a host pointer.
 *
 * Errors: every int-returning call returns 0 on success or a negative code
 * (BIPM_EINVAL bad argument or size, BIPM_ENOMEM allocation failure,
 * BIPM_ECUDA CUDA error, BIPM_ESTATE call not valid in this state,
 * BIPM_ETIMEOUT the call's device time budget bipm_options.time_limit_ms ran
 * out before every problem terminated); bipm_last_error() returns a
 * thread-local message for the last failure.  Per-problem outcomes (converged,
 * iteration cap, ...) are data, reported in bipm_stats.status /
 * bipm_result.status, never as a call error.
 */
#ifndef BIPM_H
#define BIPM_H

#ifdef __cplusplus
extern "C" {
#endif

#define BIPM_EINVAL (-22)
#define BIPM_ENOMEM (-12)
#define BIPM_ECUDA (-100)
#define BIPM_ESTATE (-101)
#define BIPM_ETIMEOUT (-102)

/* Per-problem status (the termination tests of Sec. IV and Table I):
 * RUNNING        not terminated (also: stopped by the time budget)
 * CONVERGED      scaled optimality error E_0 of Eq. 5 (mu = 0) <= tol
 * MAX_ITER       iteration cap reached
 * RESTO_FAILED   hard feasibility restoration (Table I row 6) failed: its own
 *                line search failed, it converged to an infeasible stationary
 *                point, or restoration was needed at a feasible point
 * EVAL_ERROR     non-finite objective, constraint or gradient value
 * TINY_STEP      a tiny step (Table I row 4) at the smallest barrier parameter
 * EMPTY          the slot holds no problem (a queue problem never started)
 * FP64_ESCALATION_FAILED  mixed precision: iterative refinement of the FP32
 *                step failed, and the FP64 re-factorisation that replaced it
 *                gave a Newton step (Eq. 7) that is not finite either */
#define BIPM_RUNNING 0
#define BIPM_CONVERGED 1
#define BIPM_MAX_ITER 2
#define BIPM_RESTO_FAILED 3
#define BIPM_EVAL_ERROR 4
#define BIPM_TINY_STEP 5
#define BIPM_EMPTY 6
#define BIPM_FP64_ESCALATION_FAILED 7

#define BIPM_FILTER_CAP 64

typedef struct bipm_batch bipm_batch;

/* Shared structure of one batch (Sec. III, Eq. 2: every instance of a batch
 * has the same f, c and bounds; the quadrotor NMPC family of Sec. VI). */
typedef struct {
  int n_quads;        /* quadrotors per problem, 1..8 */
  int horizon;        /* N, number of RK4 intervals, >= 1 */
  double dt;          /* interval length [s] */
  int n_spheres;      /* spherical obstacles (applied to every quadrotor) */
  int n_cylinders;    /* vertical cylinders (applied to every quadrotor) */
  double pair_dist;   /* minimum pairwise distance; 0 disables the pair rows */
  int n_moving;       /* moving spherical obstacles (applied to every quadrotor):
                         centre c + v t at the stage time t = k dt, known in
                         advance (the time-varying obstacles of Sec. VI) */
} bipm_problem_desc;

/* Algorithm options (Sec. IV; the constants the paper defers to IPOPT are
 * fixed inside the library).  A zero-initialised record is not valid: start
 * from the documented defaults. */
typedef struct {
  double tol;         /* scaled KKT tolerance E_0 (default 1e-6) */
  int max_iter;       /* iteration cap, restoration iterations included (500) */
  double mu_init;     /* initial barrier parameter (0.1) */
  int precision;      /* 0: FP64 throughout; 1: FP32 derivative blocks and FP32
                         factorisation with FP64 iterative refinement of the
                         Newton step (see fp32_switch); 2: FP32 derivative
                         blocks, double-float (two-FP32, ~48-bit) factorisation
                         and solves.  Residuals, acceptance tests and the
                         inertia (pivot) test are FP64 in every form. */
  int schedule;       /* 0: warp per problem for the first iterations, then a
                         block per remaining problem; 1: warp per problem only;
                         2: block per problem only */
  double fp32_switch; /* precision = 1: an iteration factorises in FP32 only while
                         the largest barrier diagonal of the condensed system
                         (input Sigma, slack condensation weight) is at most
                         this; above it the factorisation is FP64.  0 selects
                         the default (1e5); negative: always FP64. */
  double warm_mu_init;    /* mu_0 of a warm-started problem (0 = default 1e-2) */
  double warm_bound_push; /* bound push and bound fraction of a warm start
                             (0 = default 1e-3) */
  int warm_max_iter;      /* iteration budget of a warm-started run before the
                             cold fallback (0 = default 60; capped by max_iter) */
  int time_limit_ms;      /* device time budget of one solve or step call in
                             milliseconds, 0 = none.  Measured on the GPU's
                             clock from the call's first iteration; every team
                             checks it before each iteration and before starting
                             a queue problem.  When it runs out, running
                             problems stop at an iteration boundary (status
                             RUNNING; a batch's slots keep their state and the
                             next bipm_solve continues them), queue problems not
                             yet started report EMPTY, and the call returns
                             BIPM_ETIMEOUT. */
  /* Schedule of the persistent kernels (iteration-level batching, Sec. V).
   * None of them changes a result beyond the order of floating-point sums;
   * 0 selects the default. */
  int visit_cap;      /* queue with more slots than resident warps: iterations
                         a problem runs in its warp before it is parked for the
                         block teams (default 96; >= 1) */
  int warps_per_sm;   /* resident warps per SM of the warp-team kernels: 4, 8,
                         ..., 24 (default 24, the most that fit) */
  int team_threads;   /* threads of a block team: 128 or 256 (default 256) */
  /* Globalisation branches of Table I for the original problem (off = 0):
   * watchdog (row 3): after 10 consecutive shortened steps the full step is
   * taken for up to 3 iterations, judged against the iterate where it started,
   * and if none becomes acceptable the iterate returns there and backtracks
   * along its step; soft restoration (row 5): when the line search fails, a
   * primal-dual step that reduces the barrier problem's primal-dual error
   * |grad L|_1 + |c|_1 + |S z - mu|_1 by the factor 1 - 1e-4 is taken, for at
   * most 10 iterations, until a step passes the original tests; else hard
   * restoration follows. */
  int watchdog;
  int soft_resto;
  /* Barrier update (Table I row 7): 0 monotone (mu falls once the barrier
   * problem is solved, E_mu <= 10 mu); 1 adaptive: free mode sets mu every
   * iteration by LOQO's centrality rule, mu = 0.1 min(0.05 (1 - xi)/xi, 2)^3 *
   * (average complementarity), xi = min / average complementarity, within
   * [1e-11, 1e3 * the starting average], while the optimality error E_0 keeps
   * falling below 0.9999 times the largest of its last four values; without that
   * progress (or after a tiny step) the monotone rule takes over from 0.8 times
   * the average complementarity, until a solved barrier problem with progress
   * returns to free mode.  Restoration always uses the monotone rule. */
  int mu_strategy;
} bipm_options;

/* Per-slot outcome and counters: the branches of Table I each problem took
 * and the optimality measures of Eq. 5 at its final iterate. */
typedef struct {
  int status;
  int iters;            /* iterations taken (restoration included) */
  int resto_iters;
  int soc;              /* second-order-correction solves */
  int inertia_corr;     /* factorisations with delta_x > 0 */
  int ir_steps;         /* iterative-refinement correction solves */
  int fp64_escalations; /* FP32 factorisations redone in FP64 */
  int tiny_steps;
  int factorizations;   /* Riccati factorisations (inertia retries and FP64 redo included) */
  int solves;           /* triangular solve sweeps (steps, SOC, refinement) */
  int trials;           /* line-search trial-point evaluations */
  int fact32;           /* factorisations done in FP32 (the rest in FP64) */
  int solve32;          /* solve sweeps done in FP32 */
  int reserved;
  double obj;           /* f at the final iterate */
  double kkt_err;       /* scaled optimality error E_0 at the final iterate */
  double primal_inf;    /* max |c| at the final iterate */
  double mu;            /* final barrier parameter */
} bipm_stats;

/* Per-slot SM clock cycles spent in the phases of the iterations so far
 * (profile counters; the paper has no counterpart): eval, derivatives,
 * factorisation, solve, line search, other, least-squares multipliers, total.
 * out (host) holds count x 8 values.  Errors: BIPM_EINVAL for a bad slot
 * range or a NULL out. */
int bipm_get_phase_cycles(const bipm_batch* b, long long* out, int first_slot, int count);

/* Outcome of one problem solved through the queue (Sec. V, iteration-level
 * batching: results leave the slot when the problem terminates). */
typedef struct {
  int status;
  int iters;
  int factorizations; /* work counters as in bipm_stats */
  int solves;
  int trials;
  int ir_steps;
  int fp64_escalations;
  int resto_iters;
  int fact32;         /* factorisations / solves done in FP32 */
  int solve32;
  int warm;           /* 0 cold start; 1 warm start accepted; 2 warm start
                         rejected by the KKT test, problem re-solved cold */
  int warm_iters;     /* iterations of a rejected warm-started run (warm = 2) */
  double obj;
  double kkt_err;
} bipm_result;

/* Complete solver state of one slot (state injection, Sec. VI "Correctness").
 * Vector members point to caller-owned host arrays of the stated length; a
 * NULL vector member is skipped.  Restoration members are meaningful only in
 * restoration mode (mode == 1) and read back as zeros otherwise. */
typedef struct {
  double* x;        /* n   primal (in restoration: the original variables) */
  double* y;        /* m   equality multipliers (restoration: of c - p + n = 0) */
  double* zl;       /* n   lower-bound multipliers (0 where no lower bound) */
  double* zu;       /* n   upper-bound multipliers */
  double* p;        /* m   restoration elastic variables p, n and their */
  double* nn;       /* m   bound multipliers */
  double* zp;       /* m */
  double* zn;       /* m */
  double* x_ref;    /* n   point where restoration started (x_R) */
  double* filter;   /* 2*BIPM_FILTER_CAP (theta, phi) pairs, original problem */
  double* filter_r; /* 2*BIPM_FILTER_CAP pairs, restoration problem */
  int mode;         /* 0 original problem, 1 restoration */
  int status;
  int iter;
  int need_init;    /* theta_max/theta_min and least-squares y pending */
  int need_y_ls;    /* least-squares y at the next evaluation */
  int tiny;         /* last step was a tiny step (original / restoration) */
  int tiny_r;
  int n_filter;
  int n_filter_r;
  double mu, dw_last, theta_max, theta_min;
  double mu_r, dw_last_r, theta_max_r, theta_min_r, zeta, theta_ref;
  /* watchdog and soft restoration state (original problem; meaningful when the
   * options enable them): the iterate stored when the watchdog started and its
   * step, counters, and the stored iterate's reference values */
  double* wd_x;     /* n */
  double* wd_y;     /* m */
  double* wd_zl;    /* n */
  double* wd_zu;    /* n */
  double* wd_dx;    /* n   primal step at the stored iterate */
  double* wd_dy;    /* m   multiplier step */
  int wd_short;     /* consecutive shortened steps */
  int wd_active;
  int wd_trials;    /* unconditional watchdog steps taken */
  int soft_active;
  int soft_iters;   /* soft restoration steps in the current soft phase */
  int reserved_wd;
  double wd_theta, wd_phi, wd_gdx, wd_amax, wd_amin;
  /* adaptive barrier update: free mode flag, the reference values of E_0 and
   * the cap of mu */
  int mu_free;
  int n_refs;       /* 0..4 */
  double mu_refs[4];
  double mu_max;
} bipm_iterate;

/* Creates a batch of `capacity` slots for problems of structure `desc` (the
 * batch of Sec. III, Eq. 2: instances sharing f, c and bounds, differing in
 * theta).  opt NULL = defaults.  `cuda_stream` is a cudaStream_t (NULL = default
 * stream) used by every later call on the batch.  *out receives the batch
 * (NULL on error); the batch owns its device memory until bipm_destroy.
 * Errors: BIPM_EINVAL (bad desc, capacity < 0, bad options), BIPM_ENOMEM,
 * BIPM_ECUDA. */
int bipm_create_batch(const bipm_problem_desc* desc, int capacity, const bipm_options* opt,
                      void* cuda_stream, bipm_batch** out);

/* Sizes of one problem of Eq. 1: primal n (slacks included), equalities m,
 * parameters n_theta; any output pointer may be NULL.  Errors: BIPM_EINVAL for
 * a NULL batch. */
int bipm_dims(const bipm_batch* b, int* n, int* m, int* n_theta);

/* Loads `count` parameter vectors theta_i (the rows of Theta in Eq. 2;
 * count x n_theta, row-major, host or device per on_device) into slots
 * first_slot.. and resets those slots to the default starting point (states
 * at xbar, hover thrust, slacks at the inequality values), pushed inside the
 * bounds as in IPOPT's initialisation (Sec. IV defers to it); z = 1; y from
 * least squares at the first iteration; mu = mu_init.  Returns after the copy
 * and initialisation finished.  Errors: BIPM_EINVAL (slot range outside the
 * capacity, NULL theta), BIPM_ECUDA. */
int bipm_set_problems(bipm_batch* b, const double* theta, int first_slot, int count,
                      int on_device);

/* Replaces the primal starting point x (count x n, the variable order of
 * the layout above) of slots first_slot.. after bipm_set_problems; y
 * (count x m) may be NULL (least squares at the first iteration).  The point
 * is pushed inside the bounds as the default start is.  Host or device
 * pointers per on_device.  Errors: BIPM_EINVAL, BIPM_ENOMEM (staging),
 * BIPM_ECUDA. */
int bipm_set_initial_guess(bipm_batch* b, const double* x, const double* y, int first_slot,
                           int count, int on_device);

/* Runs every loaded slot to termination: the iteration of Sec. IV with every
 * branch of Table I taken per problem inside one persistent kernel
 * (heterogeneous iteration fusion, Sec. V); a warp that finishes its problem
 * takes the next unfinished one.  Per-problem outcomes go to bipm_get_stats.
 * Errors: BIPM_EINVAL (NULL batch), BIPM_ESTATE (nothing loaded), BIPM_ECUDA,
 * BIPM_ETIMEOUT (time_limit_ms ran out; call again to continue). */
int bipm_solve(bipm_batch* b);

/* Iteration-level batching (Sec. V "Iteration level batching"): solves the
 * `n_queue` problems of `theta_queue` (n_queue x n_theta, row-major) through
 * the batch's slots.  Every resident warp owns one slot; when its problem
 * terminates it writes that problem's solution (x_out row, n doubles; x_out
 * may be NULL) and result record, then starts the next problem of the queue
 * in the same slot.  Problems start in queue order from the default starting
 * point.  All pointers are device pointers (on_device = 1) or host pointers
 * (0; copies in and out are part of the call).  The slots' previous contents
 * are overwritten.  Returns when every problem has its record.  Errors:
 * BIPM_EINVAL (NULL theta_queue or results, n_queue < 0), BIPM_ESTATE (no
 * slots), BIPM_ENOMEM (host-pointer staging), BIPM_ECUDA, BIPM_ETIMEOUT
 * (records of unfinished problems say RUNNING or EMPTY). */
int bipm_solve_queue(bipm_batch* b, const double* theta_queue, int n_queue, double* x_out,
                     bipm_result* results, int on_device);

/* Iteration-level batching with a learned warm start (Sec. V; the warm-start
 * proposer of the method): as bipm_solve_queue, but problem i starts from the
 * primal point x_guess row i (n_queue x n, e.g. from bipm_warm_decode) pushed
 * inside the bounds by warm_bound_push, with mu_0 = warm_mu_init and bound
 * multipliers centred on the barrier (z = mu_0 / distance to the bound); y by
 * least squares.  Cold start is the fallback and the KKT residual the judge:
 * a warm-started run that has not terminated converged (E_0 <= tol) within
 * warm_max_iter iterations is rerun from the cold start in the same slot
 * (bipm_result.warm = 2).  The learned proposer has no counterpart in the
 * paper.  Pointers and errors as for bipm_solve_queue (x_guess on the same
 * side as theta_queue; BIPM_EINVAL if it is NULL). */
int bipm_solve_queue_warm(bipm_batch* b, const double* theta_queue, const double* x_guess, int n_queue,
                          double* x_out, bipm_result* results, int on_device);

/* Iteration-level batching over problems of different structures (Sec. V:
 * problems of uneven horizon and agent count in one persistent launch).
 * classes[0..n_classes) are the structure classes (1 <= n_classes <= 64);
 * problem i (0 <= i < n_queue) has class cls[i] (host array) and its
 * parameter row (n_theta of its class) packed after those of problems 0..i-1
 * in `theta`; its solution row (n of its class) goes to the same packed
 * position in x_out (may be NULL) and its record to results[i].  All
 * `n_slots` slots are sized for the largest class: one per resident warp,
 * the rest take stragglers, which 256-thread block teams finish after the
 * queue drains.  Precision 0 or 1 (options as for bipm_create_batch; NULL =
 * defaults).  theta, x_out and results are device pointers (on_device = 1) or
 * host pointers (0).  The call allocates its workspace, runs on cuda_stream
 * (NULL = default stream) and returns when the solve has finished.  Errors:
 * BIPM_EINVAL (bad class, count or option), BIPM_ENOMEM, BIPM_ECUDA,
 * BIPM_ETIMEOUT. */
int bipm_solve_mixed(const bipm_problem_desc* classes, int n_classes, const bipm_options* opt, int n_slots,
                     const int* cls, const double* theta, int n_queue, double* x_out, bipm_result* results,
                     int on_device, void* cuda_stream);

/* One-shot solve that allocates nothing.  The paper has no counterpart: this
 * entry point is an addition for callers that cannot allocate device memory at
 * the moment they need a solve -- real-time control loops that must stay out
 * of the CUDA allocator (cudaMalloc can block, synchronise the device or fail
 * under fragmentation), and processes whose device memory is budgeted in
 * advance and may not grow after start-up.
 *
 * Solves `count` problems of structure `desc` (theta: count x n_theta) with
 * the same queue (iteration-level batching) kernel as bipm_solve_queue, but
 * with the whole workspace in one 64 MiB file-scope __device__ array of the
 * library instead of memory owned by a batch.  Every GPU that loads the
 * library holds that array until the process exits.  theta, x_out
 * (count x n, may be NULL) and results (count records) are DEVICE pointers;
 * nothing is allocated or freed (no cudaMalloc, no cudaFree, no allocating
 * library call).  The number of problems solved concurrently is what fits in
 * the array (at least one); a problem whose workspace alone exceeds 64 MiB
 * is rejected with BIPM_EINVAL and a message naming both sizes.
 *
 * The first call on a device looks up the array's device address on that
 * device (with it current); make that first call before any stream capture.
 * The call copies its launch record from host memory and waits for the solve
 * to finish on `cuda_stream` (NULL = default stream) before it returns.  All
 * calls share the array and find the previous call's contents in it; the call
 * resets what must start afresh (the queue and time-budget counters and each
 * problem's slot), but calls that overlap on the GPU (other streams, other
 * threads) race on the array and must be serialised by the caller.  Errors as
 * for bipm_solve_queue (bipm_last_error). */
int bipm_solve_static(const bipm_problem_desc* desc, const bipm_options* opt, const double* theta,
                      int count, double* x_out, bipm_result* results, void* cuda_stream);

/* ---------------------------------------------------------------- warm start
 * Encodings of the learned warm start for the cluttered-environment family
 * (one quadrotor, n_cylinders vertical cylinders, no spheres, no pairs, a fixed
 * goal in the reference slot).  The paper has no counterpart (it names
 * imitation learning on this solver's trajectories only as future work,
 * Sec. VII); the proposer maps a problem's parameters theta (Eq. 2) to a
 * primal starting point.  All pointers are DEVICE pointers on
 * `cuda_stream` (NULL = default stream); the calls return after launching.
 *
 * bipm_warm_features: network input of each problem, count x (12 + 3 k_near)
 *   floats: (p0 - goal)/10, v0/2, eta0, omega0/2, then the k_near cylinders
 *   nearest to p0 in the horizontal plane (centre distance, ties by index):
 *   (cx - p0x)/10, (cy - p0y)/10, r; zeros past 30 m or past n_cylinders.
 * bipm_warm_encode: training targets from primal trajectories x (count x n):
 *   count x (12 (N+1) + 4 N) floats, (x_k - xbar)/S with
 *   S = (2,2,2, 2,2,2, .5,.5,.5, 2,2,2), then (u_k - u_hover)/u_hover.
 * bipm_warm_decode: primal starting points (count x n doubles) from network
 *   outputs in the target encoding: x_0 = xbar, x_k = xbar + S o_k (k >= 1),
 *   u_k = u_hover (1 + o), slacks at the cylinder inequality values g(x_k).
 * Errors: BIPM_EINVAL for another problem family or bad sizes; BIPM_ECUDA. */
int bipm_warm_features(const bipm_problem_desc* desc, const double* theta, int count, int k_near,
                       float* features, void* cuda_stream);
int bipm_warm_encode(const bipm_problem_desc* desc, const double* theta, const double* x, int count,
                     float* targets, void* cuda_stream);
int bipm_warm_decode(const bipm_problem_desc* desc, const double* theta, const float* net_out, int count,
                     double* x_guess, void* cuda_stream);

/* ------------------------------------------------------------ warm-start network
 * The proposer: a tanh multilayer perceptron
 *     a_0 = x,  a_l = tanh(a_{l-1} W_l^T + b_l) (hidden),  out = a_{L-1} W_L^T + b_L,
 * trained on solutions of this solver with loss 1/(2B) sum |out - t|^2 and
 * Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments).
 * Precision: matrix-product operands (inputs, weights, activations, errors)
 * are bfloat16, products accumulate in FP32 on the tensor cores; biases,
 * activations kept for the derivative, gradients and Adam's master weights
 * and moments are FP32.
 * Parameters are one flat FP32 vector: per layer W_l (width_l x width_{l-1},
 * row-major) then b_l.  x: rows x widths[0], t and out: rows x widths[last],
 * row-major FP32.  The network owns its device memory; `on_device` selects
 * device (1) or host (0) pointers for the caller's buffers.  The paper has no
 * counterpart (see the warm-start encodings above).  Errors: BIPM_EINVAL (bad
 * sizes, NULL pointers, rows above max_rows), BIPM_ENOMEM, BIPM_ECUDA. */
typedef struct bipm_mlp bipm_mlp;

/* widths: n_widths layer widths (input, hidden..., output), 2 <= n_widths <= 9;
 * max_rows: largest batch of a gradient or training call.  Parameters start
 * at zero (set them with bipm_mlp_set_params).  Errors as for the network calls
 * (above). */
int bipm_mlp_create(const int* widths, int n_widths, int max_rows, void* cuda_stream, bipm_mlp** out);
/* Number of flat parameters.  Errors as for the network calls (above). */
int bipm_mlp_param_count(const bipm_mlp* net, long long* count);
/* Loads the FP32 master parameters and resets Adam's moments and step count.
 * Errors as for the network calls (above). */
int bipm_mlp_set_params(bipm_mlp* net, const float* params, int on_device);
/* Copies the FP32 master parameters out.  Errors as for the network calls
 * (above). */
int bipm_mlp_get_params(const bipm_mlp* net, float* params, int on_device);
/* out = network(x) for any number of rows (processed max_rows at a time).
 * Errors as for the network calls (above). */
int bipm_mlp_forward(bipm_mlp* net, const float* x, int rows, float* out, int on_device);
/* Loss and its gradient with respect to the flat parameters (rows <= max_rows);
 * grad (n_params floats) and loss (one double) may be NULL.  Errors as for the
 * network calls (above). */
int bipm_mlp_loss_grad(bipm_mlp* net, const float* x, const float* t, int rows, float* grad, double* loss,
                       int on_device);
/* One Adam step on the batch of rows idx[0..rows) of the n_data rows of x and
 * t (DEVICE pointers; idx NULL = the first `rows` rows) with learning rate lr.
 * An index outside [0, n_data) is replaced by row 0 and reported by the next
 * call with a loss pointer (BIPM_EINVAL).  loss (host, may be NULL) receives
 * the batch loss before the step; without it the call returns after
 * launching.  Errors as for the network calls (above). */
int bipm_mlp_train_step(bipm_mlp* net, const float* x, const float* t, int n_data, const int* idx, int rows,
                        float lr, double* loss);
/* Frees the network and its device memory (NULL is a no-op; no error; the
 * paper has no counterpart). */
void bipm_mlp_destroy(bipm_mlp* net);

/* Runs exactly `n_iterations` iterations (the fused iteration body of
 * Sec. V, one step of Sec. IV per problem) on every running slot; terminated
 * slots are left as they are.  Used by the state-injection test of Sec. VI
 * (Eq. 8) with n_iterations = 1.  Errors: BIPM_EINVAL (NULL batch,
 * n_iterations < 1), BIPM_ESTATE (nothing loaded), BIPM_ECUDA, BIPM_ETIMEOUT. */
int bipm_step(bipm_batch* b, int n_iterations);

/* Copies the current original-problem iterate (x, y_c, z_L, z_U) of Eq. 4 of
 * slots first_slot.. -- the rows X_i of Eq. 2 and their multipliers; any
 * output pointer may be NULL.  Shapes count x n (x, zl, zu; zeros where a
 * variable has no such bound) and count x m (y).  Host or device pointers per
 * on_device.  Errors: BIPM_EINVAL (slot range), BIPM_ENOMEM (staging),
 * BIPM_ECUDA. */
int bipm_get_solution(const bipm_batch* b, double* x, double* y, double* zl, double* zu,
                      int first_slot, int count, int on_device);

/* Per-slot status and counters (host array of `count` records; see
 * bipm_stats).  Errors: BIPM_EINVAL (slot range, NULL out), BIPM_ECUDA. */
int bipm_get_stats(const bipm_batch* b, bipm_stats* out, int first_slot, int count);

/* Reads / writes the complete solver state of one slot (host arrays; see
 * bipm_iterate): the state-injection interface of Sec. VI "Correctness"
 * (Eq. 8).  bipm_set_iterate needs the slot's problem loaded first
 * (BIPM_ESTATE) and rejects filter lengths outside 0..64 and modes other than
 * 0 and 1 (BIPM_EINVAL). */
int bipm_get_iterate(const bipm_batch* b, int slot, bipm_iterate* out);
int bipm_set_iterate(bipm_batch* b, int slot, const bipm_iterate* in);

/* Self-check of the FP64 reciprocal square root used by the pivot-block
 * Cholesky of the Riccati recursion (Sec. IV, the factorisation of Eq. 7; the
 * paper has no counterpart of the routine itself): writes to *max_ulp (host)
 * the largest distance, in FP64 units in the last place, between it and
 * CUDA's correctly rounded 1.0 / sqrt(x) over n log-spaced x in [1e-40, 1e40],
 * computed on the current device with the default stream.  BIPM_EINVAL for
 * n < 1 or a null pointer, BIPM_ECUDA on a CUDA error. */
int bipm_check_rsqrt(int n, double* max_ulp);

/* Thread-local message of the last failed call ("" if none); the pointer
 * stays valid until the thread's next failing call.  The paper has no
 * counterpart; it cannot fail. */
const char* bipm_last_error(void);

/* Frees the batch of Sec. III, Eq. 2 and all its device memory (NULL is a
 * no-op; no error).  Waits for nothing: call it after the batch's last call
 * returned. */
void bipm_destroy(bipm_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* BIPM_H */
