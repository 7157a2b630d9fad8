// Shared device definitions of the batched interior-point solver: dual numbers,
// warp reductions, the per-slot state record and the workspace layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bipm.h"
#include "scalar.cuh"
#include "dfloat.cuh"

namespace bipm {

// --------------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_or(int v) { return __any_sync(0xffffffffu, v); }

// 1 / sqrt(x) for x > 0 in FP64 without the FP64 square root and division:
// an FP32 estimate y refined by one step of the second-order Newton iteration
// for the reciprocal square root (Householder's method of order 2).  With
// e = 1 - x y^2, 1 / sqrt(x) = y (1 - e)^(-1/2) = y (1 + e/2 + 3 e^2/8 + O(e^3)).
// The FP32 estimate is within a few FP32 ulp (|e| < 2^-20), so the truncated
// series is exact to about 2^-60 and the result lies within about one FP64
// ulp of 1 / sqrt(x).  Outside the normal FP32 range the plain expression.
__device__ __forceinline__ double rsqrt_fp64(double x) {
  if (!(x >= 1e-36 && x <= 1e36)) return 1.0 / sqrt(x);
  const double y = (double)rsqrtf((float)x);
  const double e = fma(-(x * y), y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}

// Team primitives.  A team is either one warp (T = 32; several teams share a
// block) or a whole block (T = blockDim.x; one team per block).  `c` is any
// context with members lane (thread index in the team), T and red (a shared
// buffer of at least T/32 doubles, block teams only).
template <class C>
__device__ __forceinline__ void team_sync(const C& c) {
  if (c.T == 32)
    __syncwarp();
  else
    __syncthreads();
}
template <class C, class Op>
__device__ __forceinline__ double team_reduce(const C& c, double v, Op op) {
  if (c.T == 32) return v;
  __syncthreads();
  if ((c.lane & 31) == 0) c.red[c.lane >> 5] = v;
  __syncthreads();
  double r = c.red[0];
  for (int i = 1; i < (c.T >> 5); ++i) r = op(r, c.red[i]);
  return r;
}
struct OpSum { __device__ double operator()(double a, double b) const { return a + b; } };
struct OpMax { __device__ double operator()(double a, double b) const { return fmax(a, b); } };
struct OpMin { __device__ double operator()(double a, double b) const { return fmin(a, b); } };
template <class C>
__device__ __forceinline__ double team_sum(const C& c, double v) {
  return team_reduce(c, warp_sum(v), OpSum());
}
template <class C>
__device__ __forceinline__ double team_max(const C& c, double v) {
  return team_reduce(c, warp_max(v), OpMax());
}
template <class C>
__device__ __forceinline__ double team_min(const C& c, double v) {
  return team_reduce(c, warp_min(v), OpMin());
}
template <class C>
__device__ __forceinline__ int team_or(const C& c, int v) {
  return team_reduce(c, warp_or(v) ? 1.0 : 0.0, OpMax()) != 0.0;
}
// value of thread 0 of the team, for every thread
template <class C>
__device__ __forceinline__ int team_bcast0(const C& c, int v) {
  if (c.T == 32) return __shfl_sync(0xffffffffu, v, 0);
  __syncthreads();
  if (c.lane == 0) c.red[0] = (double)v;
  __syncthreads();
  return (int)c.red[0];
}

// ---------------------------------------------------------- algorithm options
struct Options {
  double tol;
  int max_iter;
  double mu_init;
  int precision;  // 0 FP64; 1 FP32 factorisation + FP64 refinement; 2 double-float factorisation
  double fp32_switch;  // barrier scale above which precision 1 factorises in FP64
  double warm_mu;      // mu_0 of a warm start
  double warm_push;    // bound push and fraction of a warm start
  int warm_max_iter;   // iteration budget of a warm-started run
  int watchdog;        // Table I row 3 on the original problem
  int soft_resto;      // Table I row 5 on the original problem
  int mu_strategy;     // 0 monotone, 1 adaptive (Table I row 7)
};

// IPOPT constants (Wachter & Biegler 2006 defaults)
constexpr double kSmax = 100.0, kKappaEps = 10.0, kKappaMu = 0.2, kThetaMu = 1.5;
constexpr double kTauMin = 0.99, kKappaSigma = 1e10;
constexpr double kGammaTheta = 1e-5, kGammaPhi = 1e-8, kDelta = 1.0, kSTheta = 1.1;
constexpr double kSPhi = 2.3, kEtaPhi = 1e-8, kGammaAlpha = 0.05, kKappaSoc = 0.99;
constexpr int kPmax = 4;
constexpr double kKappaD = 1e-4;
constexpr double kDwInit = 1e-4, kDwMin = 1e-20, kDwMax = 1e40;
constexpr double kKwMinus = 1.0 / 3.0, kKwPlus = 8.0, kKwPlusBar = 100.0;
constexpr double kBoundPush = 1e-2, kBoundFrac = 1e-2, kYmax = 1e3;
constexpr double kRho = 1000.0, kKappaResto = 0.9;
constexpr int kFilterCap = 64;
constexpr int kLsMaxTrials = 60;
constexpr int kWdTrigger = 10, kWdTrialMax = 3;  // watchdog: shortened steps, unconditional steps
constexpr double kKappaSoft = 1e-4;              // soft restoration: required error reduction
constexpr int kSoftMax = 10;                     // soft restoration steps per soft phase
// adaptive barrier update: free-mode floor, cap factor, progress factor, references,
// and the fixed mode's start as a fraction of the average complementarity
constexpr double kMuMinFree = 1e-11, kMuMaxFact = 1e3, kRefsRedFact = 0.9999, kMuMonoInit = 0.8;
constexpr int kNumRefs = 4;
constexpr int kIrMaxSteps = 10;
constexpr double kIrTol = 1e-10;
constexpr int kGmresM = 6;        // Krylov dimension per restart
constexpr double kFp32BarrierMax = 1e5;  // above: factorise in FP64 this iteration
constexpr int kGmresRestarts = 3;
constexpr double kEpsMach = 2.220446049250313e-16;

enum Mode : int { MODE_NORMAL = 0, MODE_RESTO = 1 };
// phases of one iteration timed with the SM clock (per-slot profile counters)
enum Phase : int {
  PH_EVAL = 0,    // c, f, grad f, J^T y at the iterate
  PH_DERIV = 1,   // Jacobian and Hessian blocks
  PH_FACTOR = 2,  // factorisations incl. inertia correction
  PH_SOLVE = 3,   // solves incl. refinement (main step)
  PH_LS = 4,      // line search: trial points, SOC solves, acceptance
  PH_MISC = 5,    // barrier terms, error norms, mu update, restoration bookkeeping
  PH_LSQ = 6,     // least-squares multipliers
  PH_TOTAL = 7
};
enum VarKind : int { VK_FREE = 0, VK_BOX = 1, VK_LOWER = 2 };

// ------------------------------------------------------------ problem layout
struct Dims {
  int nq, N, nx, nu, ni, n, m;
  int n_sph, n_cyl, n_pairs, n_mov;
  int n_theta;
  double dt, pair_d;
  // offsets inside theta
  int th_x, th_ref, th_sph, th_cyl, th_mov;
};

// Dims with the per-quadrotor sizes fixed at compile time: NQ quadrotors per
// problem (12 states, 4 inputs each); NQ = 0 keeps the runtime fields.  The
// static members hide the base fields of the same name, so code written
// against `d.nx` gets a constant in the specialised kernels.
template <int NQ>
struct DimsT : Dims {
  static constexpr int nq = NQ, nx = 12 * NQ, nu = 4 * NQ;
};
template <>
struct DimsT<0> : Dims {};

// primal offset of x_k, u_k, s_k inside one problem's variable vector
template <class D>
__device__ __forceinline__ int off_x(const D& d, int k) {
  return k == 0 ? 0 : (d.nx + d.nu) + (k - 1) * (d.nx + d.nu + d.ni);
}
template <class D>
__device__ __forceinline__ int off_u(const D& d, int k) { return off_x(d, k) + d.nx; }
template <class D>
__device__ __forceinline__ int off_s(const D& d, int k) {  // k >= 1
  return off_x(d, k) + d.nx + (k < d.N ? d.nu : 0);
}
// equality rows: init block [0, nx), then per k: dynamics (nx) then inequalities (ni)
template <class D>
__device__ __forceinline__ int row_dyn(const D& d, int k) { return d.nx + k * (d.nx + d.ni); }
template <class D>
__device__ __forceinline__ int row_ineq(const D& d, int k) {  // inequalities of stage k >= 1
  return d.nx + (k - 1) * (d.nx + d.ni) + d.nx;
}

template <class D>
__device__ __forceinline__ int var_kind(const D& d, int i) {
  if (i < d.nx + d.nu) return i < d.nx ? VK_FREE : VK_BOX;
  int j = i - (d.nx + d.nu);
  int blk = d.nx + d.nu + d.ni;
  int k = 1 + j / blk;
  int loc = j - (k - 1) * blk;
  if (k >= d.N) return loc < d.nx ? VK_FREE : VK_LOWER;
  if (loc < d.nx) return VK_FREE;
  return loc < d.nx + d.nu ? VK_BOX : VK_LOWER;
}

// Offsets (in elements) of the per-slot arrays.  Every slot owns `slot_f64`
// doubles and `slot_tf` factor-type elements; arrays of one slot are contiguous
// so the warp that owns the slot reads them with unit stride.
// "W-sized" arrays have nw = n + 2m entries: the primal variables x followed
// by the restoration elastics p and n (used in restoration mode only).
// "K-sized" arrays have nw + m entries: a W-sized part then an m-sized part.
struct Layout {
  long long nw, nk;
  // FP64 arrays
  long long x, zl, zu, y, xt, c, ct, csoc, gf, jty, gphi, xr, xref, sig;
  long long dsv, ev, ipv, inv, dv;  // condensation diagonals (slacks / rows)
  long long rds, evr;               // 1 / D_s and E / D_s per slack
  long long qpos, qin, wrow;        // condensed inequality terms (factorisation / solve)
  long long igr;                    // inequality-row position gradients at the iterate (3 per row)
  long long fdg;                    // diagonal terms of an FP64 factorisation ((N+1) nx + N nu)
  long long rhs, sol, rhs2, sol2, res, corr, rct;
  long long filt, filt_r;
  long long wd_x, wd_zl, wd_zu, wd_y, wd_dir;  // watchdog: stored iterate and its K-sized step
  long long sft_g, sft_j, sft_y;               // soft restoration: gradient, J^T y, y at the trial
  long long f64_fac;  // FP64 factor arrays (mixed precision: escalation and LS)
  long long gscr;     // factorisation scratch in global memory (large problems)
  long long gmv;      // GMRES basis (kGmresM + 1 K-sized vectors, mixed precision)
  long long slot_f64;
  // derivative blocks (block type) and factor arrays (factor type), per slot
  long long A, B, H;
  long long slot_tb;
  long long Pt, K, Lr, LM, Yr, kff, ptv;  // offsets inside a factor region
  long long fac_size;
};
// Per-slot scalar state (the complete solver state besides the vectors).
struct SlotState {
  int status, mode, iter, need_init, need_y_ls, tiny, tiny_r, n_filt, n_filt_r;
  int n_soc, n_resto_iter, n_inertia_corr, n_ir_steps, n_escalations, n_tiny, problem_id;
  int n_fact, n_solve, n_trial, n_fact32, n_solve32;
  int parked;              // queue straggler left to the block teams (results pending)
  int warm_flag, warm_it;  // warm-start outcome of a parked problem (bipm_result.warm / warm_iters)
  int cls;                 // structure class of the slot's problem (mixed queues)
  int wd_short, wd_active, wd_trials;  // watchdog (Table I row 3)
  int soft_active, soft_iters;         // soft restoration (Table I row 5)
  int mu_free, n_refs;                 // adaptive barrier update: mode, references kept
  long long cyc[8];  // clock cycles per phase (see kPhase*)
  double mu, dw_last, theta_max, theta_min;
  double mu_r, dw_last_r, theta_max_r, theta_min_r, zeta, theta_ref;
  double obj, kkt, inf, last_alpha;
  double wd_theta, wd_phi, wd_gdx, wd_amax, wd_amin;  // watchdog reference values
  double mu_refs[kNumRefs], mu_max;                   // E_0 references, cap of mu (0: unset)
};

struct Params {
  Dims d;
  Layout L;
  Options opt;
  int n_slots;
  double* f64;        // n_slots * slot_f64
  void* tb;           // n_slots * slot_tb (double or float)
  void* tf;           // n_slots * fac_size (double or float)
  double* theta;      // n_slots * n_theta
  SlotState* st;      // n_slots
  int* work_counter;  // persistent scheduling counter
  int smem_per_warp;  // bytes of dynamic shared memory per warp
  // queue stragglers: a problem still running after visit_cap iterations in a
  // warp is parked in its slot (finished later by block teams) while the warp
  // continues in one of the n_spare spare slots (spare_counter hands them out)
  int* spare_counter;
  int n_spare;
  int visit_cap;
  // doubles between the parameter rows of consecutive slots (0: d.n_theta);
  // a mixed queue sizes every slot for its largest structure class
  long long theta_stride;
  // time budget of one call (0 = none): *t0 holds the device time (ns) at which
  // the call's first iteration started (0 until then; the host clears it), and
  // *timeout_flag is set by every team that stops because the budget ran out
  unsigned long long time_limit_ns;
  unsigned long long* t0;
  int* timeout_flag;
};

// device clock in nanoseconds
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// True once the call's time budget has run out (evaluated by one thread; the
// caller broadcasts it to its team).  The first thread to ask starts the clock.
__device__ __forceinline__ bool budget_spent(const Params* P) {
  if (P->time_limit_ns == 0) return false;
  const unsigned long long now = global_ns();
  unsigned long long t0 = atomicCAS(P->t0, 0ull, now);
  if (t0 == 0ull) t0 = now;
  if (now - t0 < P->time_limit_ns) return false;
  atomicExch(P->timeout_flag, 1);
  return true;
}

__host__ __device__ __forceinline__ long long theta_stride(const Params* P) {
  return P->theta_stride ? P->theta_stride : (long long)P->d.n_theta;
}

}  // namespace bipm
