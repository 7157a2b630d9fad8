// C-ABI library: batch management, the persistent iteration kernel and the
// copies in and out of the per-slot workspaces.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bipm.h"
#include "host_api.h"
#include "kernels.cuh"

using namespace bipm;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CUDA_TRY(expr)                                                               \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(BIPM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
  } while (0)

}  // namespace

namespace bipm {
// records the message bipm_last_error() returns (used by every entry point)
void set_last_error(const std::string& msg) { g_err = msg; }

void* queue_kernel_ptr(int precision, int nq) {
  if (nq == 1)
    return precision == 2 ? queue_kernel_df_q1() : precision ? queue_kernel_f32_q1() : queue_kernel_f64_q1();
  return precision == 2 ? queue_kernel_df() : precision ? queue_kernel_f32() : queue_kernel_f64();
}

bipm_options default_options() {
  bipm_options o;
  std::memset(&o, 0, sizeof(o));
  o.tol = 1e-6;
  o.max_iter = 500;
  o.mu_init = 0.1;
  return o;
}

// Validated dims of one problem structure (0, or an error code with message).
int dims_from_desc(const bipm_problem_desc* desc, Dims* out) {
  if (desc->n_quads < 1 || desc->n_quads > 8) return fail(BIPM_EINVAL, "n_quads must be 1..8");
  if (desc->horizon < 1 || desc->horizon > 1000) return fail(BIPM_EINVAL, "horizon must be 1..1000");
  if (!(desc->dt > 0.0) || !std::isfinite(desc->dt)) return fail(BIPM_EINVAL, "dt must be > 0");
  if (desc->n_spheres < 0 || desc->n_cylinders < 0 || desc->n_spheres > 256 || desc->n_cylinders > 256)
    return fail(BIPM_EINVAL, "obstacle counts must be 0..256");
  if (!(desc->pair_dist >= 0.0)) return fail(BIPM_EINVAL, "pair_dist must be >= 0");
  if (desc->n_moving < 0 || desc->n_moving > 256) return fail(BIPM_EINVAL, "n_moving must be 0..256");
  Dims d;
  std::memset(&d, 0, sizeof(d));
  d.nq = desc->n_quads;
  d.N = desc->horizon;
  d.nx = 12 * d.nq;
  d.nu = 4 * d.nq;
  d.n_sph = desc->n_spheres;
  d.n_cyl = desc->n_cylinders;
  d.n_mov = desc->n_moving;
  d.n_pairs = desc->pair_dist > 0.0 ? d.nq * (d.nq - 1) / 2 : 0;
  d.ni = d.nq * (d.n_sph + d.n_cyl + d.n_mov) + d.n_pairs;
  d.n = d.nx * (d.N + 1) + (d.nu + d.ni) * d.N;
  d.m = d.nx * (d.N + 1) + d.ni * d.N;
  d.dt = desc->dt;
  d.pair_d = desc->pair_dist;
  d.th_x = 0;
  d.th_ref = 12 * d.nq;
  d.th_sph = d.th_ref + 6 * d.nq;
  d.th_cyl = d.th_sph + 4 * d.n_sph;
  d.th_mov = d.th_cyl + 3 * d.n_cyl;
  d.n_theta = d.th_mov + 7 * d.n_mov;
  *out = d;
  return 0;
}

// Options with defaults filled in, validated; device options in *dev.
int options_from(const bipm_options* opt, bipm_options* o_out, Options* dev) {
  bipm_options o = opt ? *opt : default_options();
  if (o.fp32_switch == 0.0) o.fp32_switch = kFp32BarrierMax;
  if (o.warm_mu_init == 0.0) o.warm_mu_init = 1e-2;
  if (o.warm_bound_push == 0.0) o.warm_bound_push = 1e-3;
  if (o.warm_max_iter == 0) o.warm_max_iter = 60;
  if (o.warm_max_iter < 0) return fail(BIPM_EINVAL, "warm_max_iter must be >= 0");
  if (!(o.warm_mu_init > 0.0) || !(o.warm_bound_push > 0.0) || !(o.warm_bound_push < 0.5))
    return fail(BIPM_EINVAL, "warm_mu_init must be > 0 and warm_bound_push in (0, 0.5)");
  if (!(o.tol > 0.0) || o.max_iter < 0 || !(o.mu_init > 0.0) || o.precision < 0 || o.precision > 2 ||
      o.schedule < 0 || o.schedule > 2)
    return fail(BIPM_EINVAL, "bad options");
  if (o.time_limit_ms < 0) return fail(BIPM_EINVAL, "time_limit_ms must be >= 0");
  if (o.visit_cap == 0) o.visit_cap = kQueueVisit;
  if (o.warps_per_sm == 0) o.warps_per_sm = 24;
  if (o.team_threads == 0) o.team_threads = kBlockTeam;
  if (o.visit_cap < 1) return fail(BIPM_EINVAL, "visit_cap must be >= 1");
  if (o.warps_per_sm < kWarpsPerBlock || o.warps_per_sm > 24 || o.warps_per_sm % kWarpsPerBlock)
    return fail(BIPM_EINVAL, "warps_per_sm must be a multiple of 4 in 4..24");
  if (o.team_threads != 128 && o.team_threads != 256) return fail(BIPM_EINVAL, "team_threads must be 128 or 256");
  if (o.mu_strategy != 0 && o.mu_strategy != 1) return fail(BIPM_EINVAL, "mu_strategy must be 0 or 1");
  if ((o.watchdog != 0 && o.watchdog != 1) || (o.soft_resto != 0 && o.soft_resto != 1))
    return fail(BIPM_EINVAL, "watchdog and soft_resto must be 0 or 1");
  dev->tol = o.tol;
  dev->max_iter = o.max_iter;
  dev->mu_init = o.mu_init;
  dev->precision = o.precision;
  dev->fp32_switch = o.fp32_switch;
  dev->warm_mu = o.warm_mu_init;
  dev->warm_push = o.warm_bound_push;
  dev->warm_max_iter = std::min(o.warm_max_iter, o.max_iter);
  dev->watchdog = o.watchdog;
  dev->soft_resto = o.soft_resto;
  dev->mu_strategy = o.mu_strategy;
  *o_out = o;
  return 0;
}

}  // namespace bipm

struct bipm_batch {
  bipm_problem_desc desc;
  Dims d;
  Layout L;
  Options opt;
  int capacity;
  cudaStream_t stream;
  double* f64 = nullptr;
  void* tb = nullptr;
  void* tf = nullptr;
  double* theta = nullptr;
  SlotState* st = nullptr;
  int* counter = nullptr;
  Params* dparams = nullptr;
  double* stage = nullptr;  // staging buffer for gathers / scatters
  size_t stage_bytes = 0;
  int smem_per_warp = 0;
  int blocks = 0;
  int block_blocks = 0;
  int schedule = 0;
  int loaded = 0;
  int time_limit_ms = 0;
  int team_threads = kBlockTeam;  // threads of a block team
};

namespace bipm {

Layout make_layout(const Dims& d, int precision) {
  Layout L;
  std::memset(&L, 0, sizeof(L));
  const long long n = d.n, m = d.m, N = d.N, nx = d.nx, nu = d.nu;
  L.nw = n + 2 * m;
  L.nk = L.nw + m;
  long long o = 0;
  auto take = [&](long long len) {
    long long at = o;
    o += (len + 3) & ~3LL;  // 32-byte aligned arrays
    return at;
  };
  L.x = take(L.nw);
  L.zl = take(L.nw);
  L.zu = take(L.nw);
  L.y = take(m);
  L.xt = take(L.nw);
  L.c = take(m);
  L.ct = take(m);
  L.csoc = take(m);
  L.gf = take(L.nw);
  L.jty = take(L.nw);
  L.gphi = take(L.nw);
  L.xr = take(n);
  L.xref = take((N + 1) * nx);
  L.sig = take(L.nw);
  L.dsv = take(N * d.ni);
  L.ev = take(N * d.ni);
  L.rds = take(N * d.ni);
  L.evr = take(N * d.ni);
  L.qpos = take(N * 9LL * d.nq * d.nq);
  L.qin = take(N * 3LL * d.nq);
  L.wrow = take(N * d.ni);
  L.igr = take(N * 3LL * d.ni);
  L.fdg = take((N + 1) * nx + N * nu);
  L.ipv = take(m);
  L.inv = take(m);
  L.dv = take(m);
  L.rhs = take(L.nk);
  L.sol = take(L.nk);
  L.rhs2 = take(L.nk);
  L.sol2 = take(L.nk);
  L.res = take(L.nk);
  L.corr = take(L.nk);
  L.rct = take(m);
  L.filt = take(2 * (kFilterCap + 1));  // one spare entry: a full filter appends before dropping
  L.filt_r = take(2 * (kFilterCap + 1));
  L.wd_x = take(L.nw);
  L.wd_zl = take(L.nw);
  L.wd_zu = take(L.nw);
  L.wd_y = take(m);
  L.wd_dir = take(L.nk);
  L.sft_g = take(L.nw);
  L.sft_j = take(L.nw);
  L.sft_y = take(m);
  // factor region layout (element offsets)
  long long fo = 0;
  auto ftake = [&](long long len) {
    long long at = fo;
    fo += (len + 7) & ~7LL;
    return at;
  };
  L.Pt = ftake((N + 1) * nx * nx);
  L.K = ftake(N * nu * nx);
  L.Lr = ftake(N * nu * nu);
  L.LM = ftake((N + 1) * nx * nx);
  L.Yr = ftake((N + 1) * nx * nx);
  L.kff = ftake(N * nu);
  L.ptv = ftake((N + 1) * nx);
  L.fac_size = fo;
  L.f64_fac = precision ? take(L.fac_size) : 0;
  L.gscr = take((scratch_bytes(d.nq, d.nx, d.nu, 8) + 7) / 8);
  L.gmv = precision ? take((kGmresM + 1) * L.nk) : 0;
  L.slot_f64 = o;
  long long bo = 0;
  L.A = bo;
  bo += ((N * d.nq * 144) + 7) & ~7LL;
  L.B = bo;
  bo += ((N * d.nq * 48) + 7) & ~7LL;
  L.H = bo;
  bo += ((N * d.nq * 100) + 7) & ~7LL;
  L.slot_tb = bo;
  return L;
}

}  // namespace bipm

namespace {

__global__ void gather_kernel(const Params* __restrict__ P, int first, int count, long long off,
                              int len, double* __restrict__ out) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)count * len) return;
  int j = (int)(t / len), i = (int)(t - (t / len) * len);
  out[t] = P->f64[(long long)(first + j) * P->L.slot_f64 + off + i];
}

// ------------------------------------------------------------- host helpers
// kernel entry points of a precision form; problems of one quadrotor take the
// instantiation whose sizes are compile-time constants
void* iter_kernel_ptr(int precision, int nq) {
  if (nq == 1) return precision == 2 ? iter_kernel_df_q1() : precision ? iter_kernel_f32_q1() : iter_kernel_f64_q1();
  return precision == 2 ? iter_kernel_df() : precision ? iter_kernel_f32() : iter_kernel_f64();
}
void* init_kernel_ptr(int precision) {
  return precision == 2 ? init_kernel_df() : precision ? init_kernel_f32() : init_kernel_f64();
}
void* block_kernel_ptr(int precision, int nq) {
  if (nq == 1)
    return precision == 2 ? block_kernel_df_q1() : precision ? block_kernel_f32_q1() : block_kernel_f64_q1();
  return precision == 2 ? block_kernel_df() : precision ? block_kernel_f32() : block_kernel_f64();
}

int check_slots(const bipm_batch* b, int first, int count) {
  if (!b) return fail(BIPM_EINVAL, "null batch");
  if (first < 0 || count < 0 || first + count > b->capacity)
    return fail(BIPM_EINVAL, "slot range [" + std::to_string(first) + ", " +
                                 std::to_string(first + count) + ") outside capacity " +
                                 std::to_string(b->capacity));
  return 0;
}

int ensure_stage(bipm_batch* b, size_t bytes) {
  if (bytes <= b->stage_bytes) return 0;
  if (b->stage) cudaFree(b->stage);
  b->stage = nullptr;
  b->stage_bytes = 0;
  if (cudaMalloc(&b->stage, bytes) != cudaSuccess) return fail(BIPM_ENOMEM, "staging buffer");
  b->stage_bytes = bytes;
  return 0;
}

// Clears the time-budget clock and flag before a call's first launch.
int begin_call(int* counter, cudaStream_t stream) {
  CUDA_TRY(cudaMemsetAsync(counter + 2, 0, (kCounterInts - 2) * sizeof(int), stream));
  return 0;
}

// Waits for the call's work and reports an exhausted time budget.
int end_call(const int* counter, int time_limit_ms, cudaStream_t stream) {
  CUDA_TRY(cudaStreamSynchronize(stream));
  if (time_limit_ms > 0) {
    int flag = 0;
    CUDA_TRY(cudaMemcpy(&flag, counter + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag)
      return fail(BIPM_ETIMEOUT, "time limit of " + std::to_string(time_limit_ms) +
                                     " ms reached: unfinished problems report RUNNING (started) or EMPTY "
                                     "(not started)");
  }
  return 0;
}

int run_iterations(bipm_batch* b, int n_iter) {
  if (!b->loaded) return fail(BIPM_ESTATE, "no problems loaded");
  int rc = begin_call(b->counter, b->stream);
  if (rc) return rc;
  // warp teams: every problem (at most kBulkVisit iterations in solve mode
  // when block teams take over the remainder)
  if (b->schedule != 2) {
    int cap = (n_iter > 0 || b->schedule == 1) ? 0 : kBulkVisit;
    CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream));
    void* args[] = {&b->dparams, &n_iter, &cap};
    CUDA_TRY(cudaLaunchKernel(iter_kernel_ptr(b->opt.precision, b->d.nq), dim3(b->blocks),
                              dim3(32 * kWarpsPerBlock), args,
                              (size_t)b->smem_per_warp * kWarpsPerBlock, b->stream));
  }
  if (b->schedule == 2 || (n_iter <= 0 && b->schedule == 0)) {
    // block teams: the long-running remainder, to termination
    CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream));
    void* args2[] = {&b->dparams, &n_iter};
    CUDA_TRY(cudaLaunchKernel(block_kernel_ptr(b->opt.precision, b->d.nq), dim3(b->block_blocks),
                              dim3(b->team_threads), args2, (size_t)b->smem_per_warp + 128,
                              b->stream));
  }
  return end_call(b->counter, b->time_limit_ms, b->stream);
}

// ulp distance of the factorisation's reciprocal square root from CUDA's
// 1.0 / sqrt(x) over n log-spaced x in [1e-40, 1e40] (both sides of its FP32
// range tests); positive doubles order as their bit patterns
__global__ void rsqrt_check_kernel(int n, unsigned long long* worst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double t = n > 1 ? (double)i / (double)(n - 1) : 0.0;
    const double x = exp10(-40.0 + 80.0 * t);
    const long long a = __double_as_longlong(rsqrt_fp64(x));
    const long long r = __double_as_longlong(1.0 / sqrt(x));
    atomicMax(worst, (unsigned long long)(a > r ? a - r : r - a));
  }
}

}  // namespace

// ===================================================================== C ABI
extern "C" {

const char* bipm_last_error(void) { return g_err.c_str(); }

int bipm_create_batch(const bipm_problem_desc* desc, int capacity, const bipm_options* opt,
                      void* cuda_stream, bipm_batch** out) {
  if (!desc || !out) return fail(BIPM_EINVAL, "null argument");
  *out = nullptr;
  Dims dd;
  int rc = dims_from_desc(desc, &dd);
  if (rc) return rc;
  if (capacity < 0) return fail(BIPM_EINVAL, "capacity must be >= 0");
  bipm_options o;
  Options dopt;
  rc = options_from(opt, &o, &dopt);
  if (rc) return rc;

  bipm_batch* b = new bipm_batch();
  b->desc = *desc;
  Dims& d = b->d;
  d = dd;
  b->opt = dopt;
  b->schedule = o.schedule;
  b->capacity = capacity;
  b->stream = (cudaStream_t)cuda_stream;
  b->L = make_layout(d, o.precision);
  // shared-memory scratch per warp: the factorisation precision's scratch when
  // it fits in 24 KB, otherwise none (the slot's global scratch is used)
  {
    size_t need = scratch_bytes(d.nq, d.nx, d.nu, o.precision == 1 ? 4 : 8);
    size_t need64 = scratch_bytes(d.nq, d.nx, d.nu, 8);
    size_t cap_b = 24 * 1024;
    b->smem_per_warp = (int)(need64 <= cap_b ? need64 : (need <= cap_b ? need : 128));
  }

  auto cleanup = [&](int code, const std::string& msg) {
    bipm_destroy(b);
    return fail(code, msg);
  };
  size_t cap = (size_t)std::max(capacity, 1);
  // element sizes: derivative blocks FP32 for precision 1 and 2; factors FP32
  // for precision 1, double or double-float (8 bytes) otherwise
  size_t tsz = o.precision ? sizeof(float) : sizeof(double);
  size_t fsz = o.precision == 1 ? sizeof(float) : sizeof(double);
  if (cudaMalloc(&b->f64, cap * b->L.slot_f64 * sizeof(double)) != cudaSuccess)
    return cleanup(BIPM_ENOMEM, "workspace (FP64 vectors)");
  if (cudaMalloc(&b->tb, cap * b->L.slot_tb * tsz) != cudaSuccess)
    return cleanup(BIPM_ENOMEM, "workspace (derivative blocks)");
  if (cudaMalloc(&b->tf, cap * b->L.fac_size * fsz) != cudaSuccess)
    return cleanup(BIPM_ENOMEM, "workspace (factors)");
  if (cudaMalloc(&b->theta, cap * d.n_theta * sizeof(double) + 8) != cudaSuccess)
    return cleanup(BIPM_ENOMEM, "parameters");
  if (cudaMalloc(&b->st, cap * sizeof(SlotState)) != cudaSuccess) return cleanup(BIPM_ENOMEM, "states");
  if (cudaMalloc(&b->counter, kCounterInts * sizeof(int)) != cudaSuccess) return cleanup(BIPM_ENOMEM, "counter");
  if (cudaMemset(b->counter, 0, kCounterInts * sizeof(int)) != cudaSuccess) return cleanup(BIPM_ECUDA, "memset");
  if (cudaMalloc(&b->dparams, sizeof(Params)) != cudaSuccess) return cleanup(BIPM_ENOMEM, "params");
  if (cudaMemset(b->f64, 0, cap * b->L.slot_f64 * sizeof(double)) != cudaSuccess)
    return cleanup(BIPM_ECUDA, "memset");
  {
    std::vector<SlotState> empty(cap);
    std::memset(empty.data(), 0, cap * sizeof(SlotState));
    for (auto& s : empty) s.status = BIPM_EMPTY;
    if (cudaMemcpy(b->st, empty.data(), cap * sizeof(SlotState), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(BIPM_ECUDA, "state init");
  }
  Params P;
  std::memset(&P, 0, sizeof(P));
  P.d = d;
  P.L = b->L;
  P.opt = b->opt;
  P.n_slots = capacity;
  P.f64 = b->f64;
  P.tb = b->tb;
  P.tf = b->tf;
  P.theta = b->theta;
  P.st = b->st;
  P.work_counter = b->counter;
  P.smem_per_warp = b->smem_per_warp;
  set_budget(P, b->counter, o.time_limit_ms);
  b->time_limit_ms = o.time_limit_ms;
  if (cudaMemcpy(b->dparams, &P, sizeof(P), cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(BIPM_ECUDA, "params copy");

  // persistent grid: as many resident blocks as fit, capped by the work
  void* kfn = iter_kernel_ptr(o.precision, d.nq);
  size_t smem = (size_t)b->smem_per_warp * kWarpsPerBlock;
  if (smem > 48 * 1024) {
    if (cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(queue_kernel_ptr(o.precision, d.nq), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return cleanup(BIPM_ECUDA, "shared memory attribute");
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * kWarpsPerBlock, smem) !=
          cudaSuccess ||
      per_sm < 1)
    return cleanup(BIPM_ECUDA, "kernel does not fit on an SM (shared memory " + std::to_string(smem) + " B)");
  int need = (int)((cap + kWarpsPerBlock - 1) / kWarpsPerBlock);
  // resident blocks per SM: what fits, capped by the requested warps per SM
  per_sm = std::min(per_sm, o.warps_per_sm / kWarpsPerBlock);
  b->blocks = std::max(1, std::min(need, sms * per_sm));
  b->team_threads = o.team_threads;
  {
    void* bfn = block_kernel_ptr(o.precision, d.nq);
    size_t bsm = (size_t)b->smem_per_warp + 128;
    if (bsm > 48 * 1024 &&
        cudaFuncSetAttribute(bfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm) != cudaSuccess)
      return cleanup(BIPM_ECUDA, "shared memory attribute (block kernel)");
    int per_sm_b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, bfn, b->team_threads, bsm) != cudaSuccess ||
        per_sm_b < 1)
      return cleanup(BIPM_ECUDA, "block kernel does not fit on an SM");
    b->block_blocks = std::max(1, std::min((int)cap, sms * per_sm_b));
  }
  // queue schedule: one slot per resident warp, the remaining slots are spares
  // for parking stragglers (finished by block teams after the queue drains)
  {
    const int warps = std::min(capacity, b->blocks * kWarpsPerBlock);
    P.spare_counter = b->counter + 1;
    P.n_spare = std::max(0, capacity - warps);
    P.visit_cap = P.n_spare > 0 ? o.visit_cap : 0;
    if (cudaMemcpy(b->dparams, &P, sizeof(P), cudaMemcpyHostToDevice) != cudaSuccess)
      return cleanup(BIPM_ECUDA, "params copy");
  }
  *out = b;
  g_err.clear();
  return 0;
}

int bipm_dims(const bipm_batch* b, int* n, int* m, int* n_theta) {
  if (!b) return fail(BIPM_EINVAL, "null batch");
  if (n) *n = b->d.n;
  if (m) *m = b->d.m;
  if (n_theta) *n_theta = b->d.n_theta;
  return 0;
}

int bipm_set_problems(bipm_batch* b, const double* theta, int first_slot, int count, int on_device) {
  int rc = check_slots(b, first_slot, count);
  if (rc) return rc;
  if (count == 0) return 0;
  if (!theta) return fail(BIPM_EINVAL, "null theta");
  size_t bytes = (size_t)count * b->d.n_theta * sizeof(double);
  if (bytes)
    CUDA_TRY(cudaMemcpyAsync(b->theta + (size_t)first_slot * b->d.n_theta, theta, bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  const double* none = nullptr;
  void* args[] = {&b->dparams, &first_slot, &count, &none, &none};
  int threads = 128;
  int blocks = (count * 32 + threads - 1) / threads;
  CUDA_TRY(cudaLaunchKernel(init_kernel_ptr(b->opt.precision), dim3(blocks), dim3(threads), args, 0,
                            b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  b->loaded = 1;
  return 0;
}

int bipm_set_initial_guess(bipm_batch* b, const double* x, const double* y, int first_slot, int count,
                           int on_device) {
  int rc = check_slots(b, first_slot, count);
  if (rc) return rc;
  if (count == 0) return 0;
  if (!x) return fail(BIPM_EINVAL, "null x");
  size_t xb = (size_t)count * b->d.n * sizeof(double);
  size_t yb = y ? (size_t)count * b->d.m * sizeof(double) : 0;
  if ((rc = ensure_stage(b, xb + yb))) return rc;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(b->stage, x, xb, kind, b->stream));
  double* ys = nullptr;
  if (y) {
    ys = b->stage + (size_t)count * b->d.n;
    CUDA_TRY(cudaMemcpyAsync(ys, y, yb, kind, b->stream));
  }
  double* xs = b->stage;
  void* args[] = {&b->dparams, &first_slot, &count, &xs, &ys};
  int threads = 128;
  int blocks = (count * 32 + threads - 1) / threads;
  CUDA_TRY(cudaLaunchKernel(init_kernel_ptr(b->opt.precision), dim3(blocks), dim3(threads), args, 0,
                            b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return 0;
}

int bipm_solve(bipm_batch* b) {
  if (!b) return fail(BIPM_EINVAL, "null batch");
  if (b->capacity == 0) return 0;
  return run_iterations(b, 0);
}

// every slot empty before a queue solve (spare slots must not look running)
__global__ void reset_states(const Params* __restrict__ P) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P->n_slots; i += gridDim.x * blockDim.x) {
    P->st[i].status = BIPM_EMPTY;
    P->st[i].parked = 0;
  }
}

// results of the parked stragglers the block teams finished (one warp per slot)
__global__ void queue_writeout(const Params* __restrict__ P, double* __restrict__ x_out,
                               bipm_result* __restrict__ res_out) {
  const int lane = threadIdx.x & 31;
  const int slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slot >= P->n_slots) return;
  const SlotState S = P->st[slot];
  if (!S.parked) return;
  const int n = P->d.n;
  const double* w = P->f64 + (long long)slot * P->L.slot_f64 + P->L.x;
  if (x_out)
    for (int i = lane; i < n; i += 32) x_out[(long long)S.problem_id * n + i] = w[i];
  if (lane == 0) {
    res_out[S.problem_id] = make_result(S, S.warm_flag, S.warm_it);
    P->st[slot].parked = 0;
  }
}

static int solve_queue_impl(bipm_batch* b, const double* theta_queue, const double* x_guess, int n_queue,
                            double* x_out, bipm_result* results, int on_device) {
  if (!b) return fail(BIPM_EINVAL, "null batch");
  if (n_queue < 0) return fail(BIPM_EINVAL, "n_queue must be >= 0");
  if (n_queue == 0) return 0;
  if (!theta_queue || !results) return fail(BIPM_EINVAL, "null theta_queue or results");
  if (b->capacity == 0) return fail(BIPM_ESTATE, "batch has no slots");
  const Dims& d = b->d;
  size_t tb = (size_t)n_queue * d.n_theta * sizeof(double);
  size_t xb = x_out ? (size_t)n_queue * d.n * sizeof(double) : 0;
  size_t gb = x_guess ? (size_t)n_queue * d.n * sizeof(double) : 0;
  size_t rb = (size_t)n_queue * sizeof(bipm_result);
  const double* th_dev = theta_queue;
  const double* g_dev = x_guess;
  double* x_dev = x_out;
  bipm_result* r_dev = results;
  int rc;
  if (!on_device) {
    if ((rc = ensure_stage(b, tb + xb + gb + rb + 256))) return rc;
    char* base = (char*)b->stage;
    th_dev = (const double*)base;
    x_dev = x_out ? (double*)(base + tb) : nullptr;
    g_dev = x_guess ? (const double*)(base + tb + xb) : nullptr;
    r_dev = (bipm_result*)(base + ((tb + xb + gb + 15) & ~(size_t)15));
    CUDA_TRY(cudaMemcpyAsync((void*)th_dev, theta_queue, tb, cudaMemcpyHostToDevice, b->stream));
    if (x_guess) CUDA_TRY(cudaMemcpyAsync((void*)g_dev, x_guess, gb, cudaMemcpyHostToDevice, b->stream));
  }
  // one slot per resident warp; the other slots take parked stragglers
  int warps = std::min(b->capacity, b->blocks * kWarpsPerBlock);
  int blocks = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const bool spares = b->capacity > warps;
  CUDA_TRY(cudaMemsetAsync(b->counter, 0, kCounterInts * sizeof(int), b->stream));
  if (spares) {
    reset_states<<<std::max(1, std::min(1024, (b->capacity + 255) / 256)), 256, 0, b->stream>>>(b->dparams);
    CUDA_TRY(cudaGetLastError());
  }
  void* args[] = {&b->dparams, &th_dev, &n_queue, &warps, &x_dev, &r_dev, &g_dev};
  CUDA_TRY(cudaLaunchKernel(queue_kernel_ptr(b->opt.precision, b->d.nq), dim3(blocks), dim3(32 * kWarpsPerBlock),
                            args, (size_t)b->smem_per_warp * kWarpsPerBlock, b->stream));
  if (spares) {
    // block teams finish the parked stragglers, then their results go out
    int n_iter = 0;
    CUDA_TRY(cudaMemsetAsync(b->counter, 0, sizeof(int), b->stream));
    void* args2[] = {&b->dparams, &n_iter};
    CUDA_TRY(cudaLaunchKernel(block_kernel_ptr(b->opt.precision, b->d.nq), dim3(b->block_blocks), dim3(b->team_threads),
                              args2, (size_t)b->smem_per_warp + 128, b->stream));
    queue_writeout<<<(b->capacity * 32 + 255) / 256, 256, 0, b->stream>>>(b->dparams, x_dev, r_dev);
    CUDA_TRY(cudaGetLastError());
  }
  if (!on_device) {
    if (x_out) CUDA_TRY(cudaMemcpyAsync(x_out, x_dev, xb, cudaMemcpyDeviceToHost, b->stream));
    CUDA_TRY(cudaMemcpyAsync(results, r_dev, rb, cudaMemcpyDeviceToHost, b->stream));
  }
  b->loaded = 1;
  return end_call(b->counter, b->time_limit_ms, b->stream);
}

int bipm_solve_queue(bipm_batch* b, const double* theta_queue, int n_queue, double* x_out,
                     bipm_result* results, int on_device) {
  return solve_queue_impl(b, theta_queue, nullptr, n_queue, x_out, results, on_device);
}

int bipm_solve_queue_warm(bipm_batch* b, const double* theta_queue, const double* x_guess, int n_queue,
                          double* x_out, bipm_result* results, int on_device) {
  if (n_queue > 0 && !x_guess) return fail(BIPM_EINVAL, "null x_guess");
  return solve_queue_impl(b, theta_queue, x_guess, n_queue, x_out, results, on_device);
}

// results of the parked stragglers of a mixed queue (one warp per slot)
__global__ void mixed_writeout(const Params* __restrict__ Pc, const long long* __restrict__ x_off,
                               double* __restrict__ x_out, bipm_result* __restrict__ res_out) {
  const int lane = threadIdx.x & 31;
  const int slot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (slot >= Pc->n_slots) return;
  const SlotState S = Pc->st[slot];
  if (!S.parked) return;
  const Params* P = Pc + S.cls;
  const double* w = P->f64 + (long long)slot * P->L.slot_f64 + P->L.x;
  if (x_out)
    for (int i = lane; i < P->d.n; i += 32) x_out[x_off[S.problem_id] + i] = w[i];
  if (lane == 0) {
    res_out[S.problem_id] = make_result(S, 0, 0);
    Pc->st[slot].parked = 0;
  }
}

namespace {
// device allocations of one call, freed on every return path
struct DevAllocs {
  std::vector<void*> ptrs;
  void* take(size_t bytes) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return p;
  }
  ~DevAllocs() {
    for (void* p : ptrs) cudaFree(p);
  }
};
}  // namespace

int bipm_solve_mixed(const bipm_problem_desc* classes, int n_classes, const bipm_options* opt, int n_slots,
                     const int* cls, const double* theta, int n_queue, double* x_out, bipm_result* results,
                     int on_device, void* cuda_stream) {
  if (!classes || n_classes < 1 || n_classes > kMaxClasses)
    return fail(BIPM_EINVAL, "n_classes must be 1.." + std::to_string(kMaxClasses));
  if (n_slots < 1) return fail(BIPM_EINVAL, "n_slots must be >= 1");
  if (n_queue < 0) return fail(BIPM_EINVAL, "n_queue must be >= 0");
  if (n_queue == 0) return 0;
  if (!cls || !theta || !results) return fail(BIPM_EINVAL, "null cls, theta or results");
  bipm_options o;
  Options dopt;
  int rc = options_from(opt, &o, &dopt);
  if (rc) return rc;
  if (o.precision == 2) return fail(BIPM_EINVAL, "mixed queues support precision 0 and 1");
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // per-class structure and layout; slots are sized for the largest class
  std::vector<Dims> dims(n_classes);
  std::vector<Layout> lays(n_classes);
  std::vector<int> smem_c(n_classes);
  long long mf64 = 0, mtb = 0, mfac = 0, mth = 0;
  int smem_stride = 0;
  for (int k = 0; k < n_classes; ++k) {
    if ((rc = dims_from_desc(classes + k, &dims[k]))) return rc;
    lays[k] = make_layout(dims[k], o.precision);
    mf64 = std::max(mf64, lays[k].slot_f64);
    mtb = std::max(mtb, lays[k].slot_tb);
    mfac = std::max(mfac, lays[k].fac_size);
    mth = std::max(mth, (long long)dims[k].n_theta);
    const Dims& d = dims[k];
    size_t need = scratch_bytes(d.nq, d.nx, d.nu, o.precision == 1 ? 4 : 8);
    size_t need64 = scratch_bytes(d.nq, d.nx, d.nu, 8);
    const size_t cap_b = 24 * 1024;
    smem_c[k] = (int)(need64 <= cap_b ? need64 : (need <= cap_b ? need : 128));
    smem_stride = std::max(smem_stride, smem_c[k]);
  }
  // queue offsets (packed rows)
  std::vector<long long> th_off(n_queue), x_off(n_queue);
  long long th_tot = 0, x_tot = 0;
  for (int i = 0; i < n_queue; ++i) {
    if (cls[i] < 0 || cls[i] >= n_classes)
      return fail(BIPM_EINVAL, "cls[" + std::to_string(i) + "] = " + std::to_string(cls[i]) + " is not a class");
    th_off[i] = th_tot;
    x_off[i] = x_tot;
    th_tot += dims[cls[i]].n_theta;
    x_tot += dims[cls[i]].n;
  }
  void* qfn = o.precision ? queue_mixed_f32() : queue_mixed_f64();
  void* bfn = o.precision ? block_mixed_f32() : block_mixed_f64();
  const size_t qsm = (size_t)smem_stride * kWarpsPerBlock, bsm = (size_t)smem_stride + 128;
  if (qsm > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(qfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
  if (bsm > 48 * 1024) CUDA_TRY(cudaFuncSetAttribute(bfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
  int dev = 0, sms = 0, per_sm = 0, per_sm_b = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qfn, 32 * kWarpsPerBlock, qsm));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, bfn, o.team_threads, bsm));
  if (per_sm < 1 || per_sm_b < 1) return fail(BIPM_ECUDA, "mixed queue kernels do not fit on an SM");
  per_sm = std::min(per_sm, o.warps_per_sm / kWarpsPerBlock);
  const int warps = std::min(n_slots, sms * per_sm * kWarpsPerBlock);
  const int n_spare = n_slots - warps;

  const size_t tsz = o.precision ? sizeof(float) : sizeof(double);
  const size_t fsz = o.precision == 1 ? sizeof(float) : sizeof(double);
  DevAllocs mem;
  double* f64 = (double*)mem.take((size_t)n_slots * mf64 * sizeof(double));
  void* tb = mem.take((size_t)n_slots * mtb * tsz);
  void* tf = mem.take((size_t)n_slots * mfac * fsz);
  double* th_slots = (double*)mem.take((size_t)n_slots * mth * sizeof(double));
  SlotState* st = (SlotState*)mem.take((size_t)n_slots * sizeof(SlotState));
  int* counter = (int*)mem.take(kCounterInts * sizeof(int));
  Params* dP = (Params*)mem.take((size_t)n_classes * sizeof(Params));
  int* cls_d = (int*)mem.take((size_t)n_queue * sizeof(int));
  long long* off_d = (long long*)mem.take((size_t)2 * n_queue * sizeof(long long));
  if (!f64 || !tb || !tf || !th_slots || !st || !counter || !dP || !cls_d || !off_d)
    return fail(BIPM_ENOMEM, "mixed queue workspace");
  const double* th_dev = theta;
  double* x_dev = x_out;
  bipm_result* r_dev = results;
  if (!on_device) {
    th_dev = (const double*)mem.take((size_t)th_tot * sizeof(double));
    x_dev = x_out ? (double*)mem.take((size_t)x_tot * sizeof(double)) : nullptr;
    r_dev = (bipm_result*)mem.take((size_t)n_queue * sizeof(bipm_result));
    if (!th_dev || (x_out && !x_dev) || !r_dev) return fail(BIPM_ENOMEM, "mixed queue staging");
    CUDA_TRY(cudaMemcpyAsync((void*)th_dev, theta, th_tot * sizeof(double), cudaMemcpyHostToDevice, stream));
  }
  std::vector<Params> Ps(n_classes);
  for (int k = 0; k < n_classes; ++k) {
    Params& P = Ps[k];
    std::memset(&P, 0, sizeof(P));
    P.d = dims[k];
    P.L = lays[k];
    P.L.slot_f64 = mf64;  // shared slot strides
    P.L.slot_tb = mtb;
    P.L.fac_size = mfac;
    P.opt = dopt;
    P.n_slots = n_slots;
    P.f64 = f64;
    P.tb = tb;
    P.tf = tf;
    P.theta = th_slots;
    P.st = st;
    P.work_counter = counter;
    P.smem_per_warp = smem_c[k];
    P.spare_counter = counter + 1;
    P.n_spare = n_spare;
    P.visit_cap = n_spare > 0 ? o.visit_cap : 0;
    P.theta_stride = mth;
    set_budget(P, counter, o.time_limit_ms);
  }
  CUDA_TRY(cudaMemsetAsync(f64, 0, (size_t)n_slots * mf64 * sizeof(double), stream));
  CUDA_TRY(cudaMemcpyAsync(dP, Ps.data(), n_classes * sizeof(Params), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(cls_d, cls, n_queue * sizeof(int), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(off_d, th_off.data(), n_queue * sizeof(long long), cudaMemcpyHostToDevice, stream));
  CUDA_TRY(cudaMemcpyAsync(off_d + n_queue, x_off.data(), n_queue * sizeof(long long), cudaMemcpyHostToDevice,
                           stream));
  CUDA_TRY(cudaMemsetAsync(counter, 0, kCounterInts * sizeof(int), stream));
  reset_states<<<std::max(1, std::min(1024, (n_slots + 255) / 256)), 256, 0, stream>>>(dP);
  CUDA_TRY(cudaGetLastError());
  const long long* thoff_d = off_d;
  const long long* xoff_d = off_d + n_queue;
  int nq_arg = n_queue, warps_arg = warps, stride_arg = smem_stride;
  void* args[] = {&dP, &cls_d, &thoff_d, &xoff_d, &th_dev, &nq_arg, &warps_arg, &stride_arg, &x_dev, &r_dev};
  CUDA_TRY(cudaLaunchKernel(qfn, dim3((warps + kWarpsPerBlock - 1) / kWarpsPerBlock), dim3(32 * kWarpsPerBlock),
                            args, qsm, stream));
  if (n_spare > 0) {
    CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), stream));
    void* args2[] = {&dP};
    CUDA_TRY(cudaLaunchKernel(bfn, dim3(std::max(1, std::min(n_slots, sms * per_sm_b))), dim3(o.team_threads), args2,
                              bsm, stream));
    mixed_writeout<<<(int)(((long long)n_slots * 32 + 255) / 256), 256, 0, stream>>>(dP, xoff_d, x_dev, r_dev);
    CUDA_TRY(cudaGetLastError());
  }
  if (!on_device) {
    if (x_out) CUDA_TRY(cudaMemcpyAsync(x_out, x_dev, x_tot * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(results, r_dev, n_queue * sizeof(bipm_result), cudaMemcpyDeviceToHost, stream));
  }
  return end_call(counter, o.time_limit_ms, stream);
}

int bipm_check_rsqrt(int n, double* max_ulp) {
  if (n <= 0 || !max_ulp) return fail(BIPM_EINVAL, "n must be >= 1 and max_ulp non-null");
  unsigned long long* w = nullptr;
  CUDA_TRY(cudaMalloc(&w, sizeof(*w)));
  unsigned long long h = 0;
  cudaError_t e = cudaMemset(w, 0, sizeof(*w));
  if (e == cudaSuccess) {
    rsqrt_check_kernel<<<152, 256>>>(n, w);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, w, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(w);
  if (e != cudaSuccess) return fail(BIPM_ECUDA, cudaGetErrorString(e));
  *max_ulp = (double)h;
  return 0;
}

int bipm_step(bipm_batch* b, int n_iterations) {
  if (!b) return fail(BIPM_EINVAL, "null batch");
  if (n_iterations < 1) return fail(BIPM_EINVAL, "n_iterations must be >= 1");
  if (b->capacity == 0) return 0;
  return run_iterations(b, n_iterations);
}

int bipm_get_solution(const bipm_batch* bc, double* x, double* y, double* zl, double* zu,
                      int first_slot, int count, int on_device) {
  bipm_batch* b = const_cast<bipm_batch*>(bc);
  int rc = check_slots(b, first_slot, count);
  if (rc) return rc;
  if (count == 0) return 0;
  struct Item { double* dst; long long off; int len; } items[4] = {
      {x, b->L.x, b->d.n}, {y, b->L.y, b->d.m}, {zl, b->L.zl, b->d.n}, {zu, b->L.zu, b->d.n}};
  for (auto& it : items) {
    if (!it.dst) continue;
    size_t bytes = (size_t)count * it.len * sizeof(double);
    if ((rc = ensure_stage(b, bytes))) return rc;
    long long total = (long long)count * it.len;
    int threads = 256;
    int blocks = (int)((total + threads - 1) / threads);
    gather_kernel<<<blocks, threads, 0, b->stream>>>(b->dparams, first_slot, count, it.off, it.len,
                                                     b->stage);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(it.dst, b->stage, bytes,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  return 0;
}

int bipm_get_stats(const bipm_batch* b, bipm_stats* out, int first_slot, int count) {
  int rc = check_slots(b, first_slot, count);
  if (rc) return rc;
  if (count == 0) return 0;
  if (!out) return fail(BIPM_EINVAL, "null output");
  std::vector<SlotState> h(count);
  CUDA_TRY(cudaMemcpyAsync(h.data(), b->st + first_slot, count * sizeof(SlotState),
                           cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < count; ++i) {
    const SlotState& s = h[i];
    bipm_stats& o = out[i];
    o.status = s.status;
    o.iters = s.iter;
    o.resto_iters = s.n_resto_iter;
    o.soc = s.n_soc;
    o.inertia_corr = s.n_inertia_corr;
    o.ir_steps = s.n_ir_steps;
    o.fp64_escalations = s.n_escalations;
    o.tiny_steps = s.n_tiny;
    o.factorizations = s.n_fact;
    o.solves = s.n_solve;
    o.trials = s.n_trial;
    o.fact32 = s.n_fact32;
    o.solve32 = s.n_solve32;
    o.reserved = 0;
    o.obj = s.obj;
    o.kkt_err = s.kkt;
    o.primal_inf = s.inf;
    o.mu = s.mu;
  }
  return 0;
}

int bipm_get_phase_cycles(const bipm_batch* b, long long* out, int first_slot, int count) {
  int rc = check_slots(b, first_slot, count);
  if (rc) return rc;
  if (count == 0) return 0;
  if (!out) return fail(BIPM_EINVAL, "null output");
  std::vector<SlotState> h(count);
  CUDA_TRY(cudaMemcpyAsync(h.data(), b->st + first_slot, count * sizeof(SlotState),
                           cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < count; ++i)
    for (int p = 0; p < 8; ++p) out[(size_t)i * 8 + p] = h[i].cyc[p];
  return 0;
}

int bipm_get_iterate(const bipm_batch* b, int slot, bipm_iterate* out) {
  int rc = check_slots(b, slot, 1);
  if (rc) return rc;
  if (!out) return fail(BIPM_EINVAL, "null output");
  const Dims& d = b->d;
  const Layout& L = b->L;
  const double* base = b->f64 + (size_t)slot * L.slot_f64;
  std::vector<double> buf(L.slot_f64);
  CUDA_TRY(cudaMemcpyAsync(buf.data(), base, L.slot_f64 * sizeof(double), cudaMemcpyDeviceToHost,
                           b->stream));
  SlotState s;
  CUDA_TRY(cudaMemcpyAsync(&s, b->st + slot, sizeof(s), cudaMemcpyDeviceToHost, b->stream));
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  auto put = [&](double* dst, long long off, int len) {
    if (dst) std::memcpy(dst, buf.data() + off, len * sizeof(double));
  };
  put(out->x, L.x, d.n);
  put(out->y, L.y, d.m);
  put(out->zl, L.zl, d.n);
  put(out->zu, L.zu, d.n);
  put(out->p, L.x + d.n, d.m);
  put(out->nn, L.x + d.n + d.m, d.m);
  put(out->zp, L.zl + d.n, d.m);
  put(out->zn, L.zl + d.n + d.m, d.m);
  put(out->x_ref, L.xr, d.n);
  put(out->filter, L.filt, 2 * kFilterCap);
  put(out->filter_r, L.filt_r, 2 * kFilterCap);
  out->mode = s.mode;
  out->status = s.status;
  out->iter = s.iter;
  out->need_init = s.need_init;
  out->need_y_ls = s.need_y_ls;
  out->tiny = s.tiny;
  out->tiny_r = s.tiny_r;
  out->n_filter = s.n_filt;
  out->n_filter_r = s.n_filt_r;
  out->mu = s.mu;
  out->dw_last = s.dw_last;
  out->theta_max = s.theta_max;
  out->theta_min = s.theta_min;
  out->mu_r = s.mu_r;
  out->dw_last_r = s.dw_last_r;
  out->theta_max_r = s.theta_max_r;
  out->theta_min_r = s.theta_min_r;
  out->zeta = s.zeta;
  out->theta_ref = s.theta_ref;
  put(out->wd_x, L.wd_x, d.n);
  put(out->wd_y, L.wd_y, d.m);
  put(out->wd_zl, L.wd_zl, d.n);
  put(out->wd_zu, L.wd_zu, d.n);
  put(out->wd_dx, L.wd_dir, d.n);
  put(out->wd_dy, L.wd_dir + L.nw, d.m);
  out->wd_short = s.wd_short;
  out->wd_active = s.wd_active;
  out->wd_trials = s.wd_trials;
  out->soft_active = s.soft_active;
  out->soft_iters = s.soft_iters;
  out->reserved_wd = 0;
  out->wd_theta = s.wd_theta;
  out->wd_phi = s.wd_phi;
  out->wd_gdx = s.wd_gdx;
  out->wd_amax = s.wd_amax;
  out->wd_amin = s.wd_amin;
  out->mu_free = s.mu_free;
  out->n_refs = s.n_refs;
  for (int i = 0; i < 4; ++i) out->mu_refs[i] = s.mu_refs[i];
  out->mu_max = s.mu_max;
  return 0;
}

int bipm_set_iterate(bipm_batch* b, int slot, const bipm_iterate* in) {
  int rc = check_slots(b, slot, 1);
  if (rc) return rc;
  if (!in) return fail(BIPM_EINVAL, "null input");
  if (!b->loaded) return fail(BIPM_ESTATE, "load the problem (bipm_set_problems) first");
  if (in->n_filter < 0 || in->n_filter > kFilterCap || in->n_filter_r < 0 || in->n_filter_r > kFilterCap)
    return fail(BIPM_EINVAL, "filter length outside 0..64");
  if (in->mode != 0 && in->mode != 1) return fail(BIPM_EINVAL, "mode must be 0 or 1");
  const Dims& d = b->d;
  const Layout& L = b->L;
  double* base = b->f64 + (size_t)slot * L.slot_f64;
  std::vector<double> buf(L.slot_f64);
  CUDA_TRY(cudaMemcpy(buf.data(), base, L.slot_f64 * sizeof(double), cudaMemcpyDeviceToHost));
  auto get = [&](const double* src, long long off, int len) {
    if (src)
      std::memcpy(buf.data() + off, src, len * sizeof(double));
    else
      std::memset(buf.data() + off, 0, len * sizeof(double));
  };
  get(in->x, L.x, d.n);
  get(in->y, L.y, d.m);
  get(in->zl, L.zl, d.n);
  get(in->zu, L.zu, d.n);
  get(in->p, L.x + d.n, d.m);
  get(in->nn, L.x + d.n + d.m, d.m);
  get(in->zp, L.zl + d.n, d.m);
  get(in->zn, L.zl + d.n + d.m, d.m);
  std::memset(buf.data() + L.zu + d.n, 0, 2 * d.m * sizeof(double));
  get(in->x_ref, L.xr, d.n);
  get(in->filter, L.filt, 2 * kFilterCap);
  get(in->filter_r, L.filt_r, 2 * kFilterCap);
  get(in->wd_x, L.wd_x, d.n);
  get(in->wd_y, L.wd_y, d.m);
  get(in->wd_zl, L.wd_zl, d.n);
  get(in->wd_zu, L.wd_zu, d.n);
  get(in->wd_dx, L.wd_dir, d.n);
  get(in->wd_dy, L.wd_dir + L.nw, d.m);
  CUDA_TRY(cudaMemcpy(base, buf.data(), L.slot_f64 * sizeof(double), cudaMemcpyHostToDevice));
  SlotState s;
  CUDA_TRY(cudaMemcpy(&s, b->st + slot, sizeof(s), cudaMemcpyDeviceToHost));
  s.mode = in->mode;
  s.status = in->status;
  s.iter = in->iter;
  s.need_init = in->need_init;
  s.need_y_ls = in->need_y_ls;
  s.tiny = in->tiny;
  s.tiny_r = in->tiny_r;
  s.n_filt = in->n_filter;
  s.n_filt_r = in->n_filter_r;
  s.mu = in->mu;
  s.dw_last = in->dw_last;
  s.theta_max = in->theta_max;
  s.theta_min = in->theta_min;
  s.mu_r = in->mu_r;
  s.dw_last_r = in->dw_last_r;
  s.theta_max_r = in->theta_max_r;
  s.theta_min_r = in->theta_min_r;
  s.zeta = in->zeta;
  s.theta_ref = in->theta_ref;
  s.wd_short = in->wd_short;
  s.wd_active = in->wd_active;
  s.wd_trials = in->wd_trials;
  s.soft_active = in->soft_active;
  s.soft_iters = in->soft_iters;
  s.wd_theta = in->wd_theta;
  s.wd_phi = in->wd_phi;
  s.wd_gdx = in->wd_gdx;
  s.wd_amax = in->wd_amax;
  s.wd_amin = in->wd_amin;
  if (in->n_refs < 0 || in->n_refs > kNumRefs) return fail(BIPM_EINVAL, "n_refs outside 0..4");
  s.mu_free = in->mu_free;
  s.n_refs = in->n_refs;
  for (int i = 0; i < kNumRefs; ++i) s.mu_refs[i] = in->mu_refs[i];
  s.mu_max = in->mu_max;
  CUDA_TRY(cudaMemcpy(b->st + slot, &s, sizeof(s), cudaMemcpyHostToDevice));
  return 0;
}

void bipm_destroy(bipm_batch* b) {
  if (!b) return;
  cudaFree(b->f64);
  cudaFree(b->tb);
  cudaFree(b->tf);
  cudaFree(b->theta);
  cudaFree(b->st);
  cudaFree(b->counter);
  cudaFree(b->dparams);
  cudaFree(b->stage);
  delete b;
}

}  // extern "C"
