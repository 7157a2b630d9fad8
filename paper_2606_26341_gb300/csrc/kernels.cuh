// Kernel templates of the batched solver: the persistent iteration kernel
// (warp per problem, problems taken from an atomic work counter) and the
// slot initialisation kernel.  Instantiated once per precision in
// kernels_f64.cu and kernels_f32.cu.
#pragma once

#include "ipm_iter.cuh"

namespace bipm {

constexpr int kWarpsPerBlock = 4;
constexpr int kBlockTeam = 256;    // threads of a block team
constexpr int kBulkVisit = 64;     // iterations per problem in the warp kernel
constexpr int kQueueVisit = 96;    // iterations before a queue problem is parked for block teams
constexpr int kMaxClasses = 64;    // structure classes of one mixed queue

template <class TB, class TF, int NQ, int TM>
__device__ void make_ctx(Ctx<TB, TF, NQ, TM>& c, const Params* P, int slot, int lane, int T, double* red,
                         char* smem) {
  c.P = P;
  static_cast<Dims&>(c.d) = P->d;
  c.L = P->L;
  c.lane = lane;
  if constexpr (TM == 0)
    c.T = T;
  else
    (void)T;
  c.red = red;
  c.slot = slot;
  c.f = P->f64 + (long long)slot * P->L.slot_f64;
  c.blk = (TB*)P->tb + (long long)slot * P->L.slot_tb;
  TF* fb = (TF*)P->tf + (long long)slot * P->L.fac_size;
  c.fac = make_fac<TF>(fb, P->L);
  if constexpr (std::is_same<TF, double>::value)
    c.fac64 = make_fac<double>((double*)fb, P->L);
  else
    c.fac64 = make_fac<double>(c.f + P->L.f64_fac, P->L);
  c.th = P->theta + (long long)slot * theta_stride(P);
  c.smem = smem;
  c.smem_bytes = P->smem_per_warp;
  c.gscratch = (char*)(c.f + P->L.gscr);
  c.resto = 0;
  c.nw = P->d.n;
  c.mu = 0.0;
  c.zeta = 0.0;
  c.dw = 0.0;
  c.use64 = 0;
  c.n_ir = 0;
  c.n_esc = 0;
  c.esc_failed = 0;
  c.n_fact = 0;
  c.n_solve = 0;
  c.n_trial = 0;
  c.n_fact32 = 0;
  c.n_solve32 = 0;
}

// final objective, scaled KKT error and infeasibility of the original problem
template <class TB, class TF, int NQ, int TM>
__device__ void slot_metrics(Ctx<TB, TF, NQ, TM>& c, SlotState& S) {
  c.resto = 0;
  c.nw = c.d.n;
  double* w = c.f + c.L.x;
  double* y = c.f + c.L.y;
  double* cv = c.f + c.L.c;
  double f = eval_values(c, w, cv);
  eval_grad(c, w, c.f + c.L.gf);
  eval_jty(c, w, y, c.f + c.L.jty);
  ErrParts e = err_parts(c);
  S.obj = f;
  S.kkt = opt_error(c, e, 0.0);
  S.inf = e.prim;
}

// true (in every thread of the team) once the call's time budget has run out
template <class TB, class TF, int NQ, int TM>
__device__ __forceinline__ bool team_budget_spent(Ctx<TB, TF, NQ, TM>& c) {
  if (c.P->time_limit_ns == 0) return false;
  int v = 0;
  if (c.lane == 0) v = budget_spent(c.P) ? 1 : 0;
  return team_bcast0(c, v) != 0;
}

// Iterates one slot: exactly n_iter iterations (n_iter > 0), or until it
// terminates, or (visit_cap > 0) for at most visit_cap iterations in this visit.
// Before every iteration the call's time budget is checked; returns true if the
// slot stopped because it ran out (the problem is left running, resumable).
template <class TB, class TF, int NQ, int TM>
__device__ bool run_slot(Ctx<TB, TF, NQ, TM>& c, SlotState& S, int n_iter, int visit_cap) {
  int done = 0;
  bool spent = false;
  if (n_iter > 0) {
    for (; done < n_iter && S.status == BIPM_RUNNING; ++done) {
      if ((spent = team_budget_spent(c))) break;
      iterate(c, S);
    }
  } else {
    while (S.status == BIPM_RUNNING && (visit_cap <= 0 || done < visit_cap)) {
      if ((spent = team_budget_spent(c))) break;
      iterate(c, S);
      ++done;
    }
  }
  if (n_iter > 0 || S.status != BIPM_RUNNING) slot_metrics(c, S);
  return spent;
}

// Persistent kernel, one warp per problem: each warp takes the next slot from
// the work counter and iterates it (iteration-level batching: a warp that
// finishes a problem immediately starts another one).
template <class TB, class TF, int NQ>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 6)
    ipm_kernel(const Params* __restrict__ P, int n_iter, int visit_cap) {
  extern __shared__ __align__(16) char smem_all[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  char* smem = smem_all + (size_t)warp * P->smem_per_warp;
  while (true) {
    int slot = 0;
    if (lane == 0) slot = atomicAdd(P->work_counter, 1);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= P->n_slots) break;
    SlotState S = P->st[slot];
    if (S.status != BIPM_RUNNING) continue;
    Ctx<TB, TF, NQ, 32> c;
    make_ctx(c, P, slot, lane, 32, nullptr, smem);
    run_slot(c, S, n_iter, visit_cap);
    __syncwarp();
    if (lane == 0) P->st[slot] = S;
    __syncwarp();
  }
}

// Persistent kernel, one block per problem: the same iteration with the
// block's threads spread over all four SM sub-partitions, for the few
// long-running problems left after the warp kernel (their per-iteration
// latency, not the batch throughput, bounds the solve).
template <class TB, class TF, int NQ>
__global__ void __launch_bounds__(kBlockTeam)
    ipm_block_kernel(const Params* __restrict__ P, int n_iter) {
  extern __shared__ __align__(16) char smem_all[];
  double* red = (double*)smem_all;
  char* smem = smem_all + 128;
  __shared__ int s_slot;
  while (true) {
    if (threadIdx.x == 0) s_slot = atomicAdd(P->work_counter, 1);
    __syncthreads();
    const int slot = s_slot;
    __syncthreads();
    if (slot >= P->n_slots) break;
    SlotState S = P->st[slot];
    if (S.status != BIPM_RUNNING) continue;
    Ctx<TB, TF, NQ, 0> c;
    make_ctx(c, P, slot, (int)threadIdx.x, (int)blockDim.x, red, smem);
    run_slot(c, S, n_iter, 0);
    __syncthreads();
    if (threadIdx.x == 0) P->st[slot] = S;
    __syncthreads();
  }
}

// starting point pushed inside the bounds (IPOPT initialisation): k1 is the
// absolute push, k2 the fraction of the box width
__device__ __forceinline__ double push_into_bounds(int kind, double v, double k1, double k2) {
  if (kind == VK_BOX) {
    double width = kUmax - 0.0;
    double pl = fmin(k1 * fmax(1.0, 0.0), k2 * width);
    double pu = fmin(k1 * fmax(1.0, kUmax), k2 * width);
    return fmin(fmax(v, 0.0 + pl), kUmax - pu);
  }
  if (kind == VK_LOWER) return fmax(v, 0.0 + k1 * fmax(1.0, 0.0));
  return v;
}

// Resets one slot to the starting point of the problem whose theta the slot
// holds (warp-level; lanes stride 32).  guess / yguess: optional primal /
// multiplier rows.  warm: a learned warm start (bound push and fraction
// opt.warm_push, mu_0 = opt.warm_mu, bound multipliers centred on the barrier,
// z = mu_0 / distance to the bound) instead of the cold start (push 1e-2,
// z = 1).  Returns the fresh state record (identical in all lanes).
__device__ __forceinline__ SlotState init_slot(const Params* P, int slot, int lane,
                                               const double* guess, const double* yguess,
                                               int warm = 0) {
  const Dims& d = P->d;
  const Layout& L = P->L;
  double* f = P->f64 + (long long)slot * L.slot_f64;
  const double* th = P->theta + (long long)slot * theta_stride(P);
  double* w = f + L.x;
  double* zl = f + L.zl;
  double* zu = f + L.zu;
  double* y = f + L.y;
  for (int i = lane; i < d.n; i += 32) {
    VarInfo vi = var_info(d, i);
    double v;
    if (guess) {
      v = guess[i];
    } else if (vi.loc < d.nx) {
      v = th[d.th_x + vi.loc];
    } else if (vi.kind == VK_BOX) {
      v = kHover;
    } else {
      int r = vi.loc - d.nx - (vi.k < d.N ? d.nu : 0);
      IneqRow row = ineq_row(d, th, th + d.th_x, r, vi.k);
      v = row.gval;
    }
    if (warm) {
      const double mu0 = P->opt.warm_mu, k = P->opt.warm_push;
      v = push_into_bounds(vi.kind, v, k, k);
      w[i] = v;
      zl[i] = has_lower(vi.kind) ? mu0 / (v - 0.0) : 0.0;
      zu[i] = has_upper(vi.kind) ? mu0 / (kUmax - v) : 0.0;
    } else {
      w[i] = push_into_bounds(vi.kind, v, kBoundPush, kBoundFrac);
      zl[i] = has_lower(vi.kind) ? 1.0 : 0.0;
      zu[i] = has_upper(vi.kind) ? 1.0 : 0.0;
    }
    f[L.xr + i] = 0.0;
  }
  for (int i = lane; i < 2 * d.m; i += 32) {
    w[d.n + i] = 0.0;
    zl[d.n + i] = 0.0;
    zu[d.n + i] = 0.0;
  }
  for (int i = lane; i < d.m; i += 32) y[i] = yguess ? yguess[i] : 0.0;
  for (int i = lane; i < (d.N + 1) * d.nx; i += 32) {
    int kk = i / d.nx, c = i - kk * d.nx;
    f[L.xref + i] = ref_value(th, d, kk, c / 12, c - 12 * (c / 12));
  }
  __syncwarp();
  SlotState S;
  memset(&S, 0, sizeof(S));
  S.status = BIPM_RUNNING;
  S.mode = MODE_NORMAL;
  S.need_init = 1;
  S.need_y_ls = yguess ? 0 : 1;
  S.mu = warm ? P->opt.warm_mu : P->opt.mu_init;
  S.mu_free = 1;  // the adaptive barrier update starts in free mode
  S.problem_id = slot;
  return S;
}

template <class TB, class TF, int NQ>
__global__ void init_kernel(const Params* __restrict__ P, int first, int count,
                            const double* __restrict__ guess, const double* __restrict__ yguess) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= count) return;
  const int slot = first + gw;
  SlotState S = init_slot(P, slot, lane, guess ? guess + (long long)gw * P->d.n : nullptr,
                          yguess ? yguess + (long long)gw * P->d.m : nullptr);
  if (lane == 0) P->st[slot] = S;
}

// Iteration-level batching over a queue (Sec. V): each warp owns one slot;
// when its problem terminates it writes the problem's results and refills the
// slot with the next problem of the queue, so no slot idles while the queue
// holds work.  With x_guess (n_queue x n primal rows) every problem starts
// from its warm starting point; a warm-started run that has not ended
// converged (the scaled KKT test E_0 <= tol) within opt.warm_max_iter
// iterations is rerun from the cold start in the same slot.
// result record of a terminated problem
__device__ __forceinline__ bipm_result make_result(const SlotState& S, int warm, int warm_iters) {
  bipm_result r;
  r.status = S.status;
  r.iters = S.iter;
  r.factorizations = S.n_fact;
  r.solves = S.n_solve;
  r.trials = S.n_trial;
  r.ir_steps = S.n_ir_steps;
  r.fp64_escalations = S.n_escalations;
  r.resto_iters = S.n_resto_iter;
  r.fact32 = S.n_fact32;
  r.solve32 = S.n_solve32;
  r.warm = warm;
  r.warm_iters = warm_iters;
  r.obj = S.obj;
  r.kkt_err = S.kkt;
  return r;
}

// record of a queue problem that was never started (the time budget ran out)
__device__ __forceinline__ bipm_result empty_result() {
  bipm_result r;
  memset(&r, 0, sizeof(r));
  r.status = BIPM_EMPTY;
  return r;
}

// warp-uniform time-budget test of a queue warp before it starts a problem
__device__ __forceinline__ bool queue_budget_spent(const Params* P, int lane) {
  if (P->time_limit_ns == 0) return false;
  int v = 0;
  if (lane == 0) v = budget_spent(P) ? 1 : 0;
  return __shfl_sync(0xffffffffu, v, 0) != 0;
}

template <class TB, class TF, int NQ>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 6)
    queue_kernel(const Params* __restrict__ P, const double* __restrict__ theta_q, int n_queue,
                 int n_warps, double* __restrict__ x_out, bipm_result* __restrict__ res_out,
                 const double* __restrict__ x_guess) {
  extern __shared__ __align__(16) char smem_all[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int slot = blockIdx.x * kWarpsPerBlock + warp;  // this warp's slot
  if (slot >= n_warps) return;
  char* smem = smem_all + (size_t)warp * P->smem_per_warp;
  const Dims& d = P->d;
  while (true) {
    int id = 0;
    if (lane == 0) id = atomicAdd(P->work_counter, 1);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= n_queue) break;
    if (queue_budget_spent(P, lane)) {  // out of time: the problem is not started
      if (lane == 0) res_out[id] = empty_result();
      continue;
    }
    double* th = P->theta + (long long)slot * theta_stride(P);
    for (int i = lane; i < d.n_theta; i += 32) th[i] = theta_q[(long long)id * d.n_theta + i];
    __syncwarp();
    const double* gq = x_guess ? x_guess + (long long)id * d.n : nullptr;
    SlotState S = init_slot(P, slot, lane, gq, nullptr, gq != nullptr);
    S.problem_id = id;
    Ctx<TB, TF, NQ, 32> c;
    make_ctx(c, P, slot, lane, 32, nullptr, smem);
    int warm = gq ? 1 : 0, warm_iters = 0;
    bool done = false, spent = false;
    if (gq) {
      spent = run_slot(c, S, 0, P->opt.warm_max_iter);
      if (S.status == BIPM_CONVERGED) {
        done = true;
      } else if (!spent) {
        warm = 2;
        warm_iters = S.iter;
        S = init_slot(P, slot, lane, nullptr, nullptr, 0);
        S.problem_id = id;
        make_ctx(c, P, slot, lane, 32, nullptr, smem);
      }
    }
    if (!done && !spent) {
      spent = run_slot(c, S, 0, P->visit_cap);
      if (S.status == BIPM_RUNNING && !spent) {
        // straggler: park it for the block teams when a spare slot is free
        int ns = 0;
        if (lane == 0) ns = atomicAdd(P->spare_counter, 1);
        ns = __shfl_sync(0xffffffffu, ns, 0);
        if (ns < P->n_spare) {
          if (lane == 0) {
            S.parked = 1;
            S.warm_flag = warm;
            S.warm_it = warm_iters;
            P->st[slot] = S;
          }
          __syncwarp();
          slot = n_warps + ns;
          continue;
        }
        run_slot(c, S, 0, 0);
      }
    }
    // a problem stopped by the time budget is written out with status RUNNING
    const double* w = c.f + P->L.x;
    if (x_out)
      for (int i = lane; i < d.n; i += 32) x_out[(long long)id * d.n + i] = w[i];
    if (lane == 0) {
      res_out[id] = make_result(S, warm, warm_iters);
      S.parked = 0;
      P->st[slot] = S;
    }
    __syncwarp();
  }
}

// Iteration-level batching over problems of different structures (uneven
// horizons and quadrotor counts) in one launch.  Pc[c] describes structure
// class c (its dims and slot layout; every class shares the workspace, whose
// slots are sized for the largest class).  Problem id has class cls[id], its
// parameters at theta_q + th_off[id] and its solution row at x_out + x_off[id].
// smem_stride: shared-memory bytes per warp of the launch.  Stragglers are
// parked as in queue_kernel and finished by block_mixed_kernel.
template <class TB, class TF, int NQ>
__global__ void __launch_bounds__(32 * kWarpsPerBlock, 6)
    queue_mixed_kernel(const Params* __restrict__ Pc, const int* __restrict__ cls,
                       const long long* __restrict__ th_off, const long long* __restrict__ x_off,
                       const double* __restrict__ theta_q, int n_queue, int n_warps, int smem_stride,
                       double* __restrict__ x_out, bipm_result* __restrict__ res_out) {
  extern __shared__ __align__(16) char smem_all[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  int slot = blockIdx.x * kWarpsPerBlock + warp;
  if (slot >= n_warps) return;
  char* smem = smem_all + (size_t)warp * smem_stride;
  const Params* P0 = Pc;
  while (true) {
    int id = 0;
    if (lane == 0) id = atomicAdd(P0->work_counter, 1);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= n_queue) break;
    if (queue_budget_spent(P0, lane)) {
      if (lane == 0) res_out[id] = empty_result();
      continue;
    }
    const int k = cls[id];
    const Params* P = Pc + k;
    const Dims& d = P->d;
    double* th = P->theta + (long long)slot * theta_stride(P);
    for (int i = lane; i < d.n_theta; i += 32) th[i] = theta_q[th_off[id] + i];
    __syncwarp();
    SlotState S = init_slot(P, slot, lane, nullptr, nullptr, 0);
    S.problem_id = id;
    S.cls = k;
    Ctx<TB, TF, NQ, 32> c;
    make_ctx(c, P, slot, lane, 32, nullptr, smem);
    const bool spent = run_slot(c, S, 0, P->visit_cap);
    if (S.status == BIPM_RUNNING && !spent) {
      int ns = 0;
      if (lane == 0) ns = atomicAdd(P0->spare_counter, 1);
      ns = __shfl_sync(0xffffffffu, ns, 0);
      if (ns < P0->n_spare) {
        if (lane == 0) {
          S.parked = 1;
          S.warm_flag = 0;
          S.warm_it = 0;
          P->st[slot] = S;
        }
        __syncwarp();
        slot = n_warps + ns;
        continue;
      }
      run_slot(c, S, 0, 0);
    }
    const double* w = c.f + P->L.x;
    if (x_out)
      for (int i = lane; i < d.n; i += 32) x_out[x_off[id] + i] = w[i];
    if (lane == 0) {
      res_out[id] = make_result(S, 0, 0);
      S.parked = 0;
      P->st[slot] = S;
    }
    __syncwarp();
  }
}

// Block teams finish the parked problems of a mixed queue (each slot's class
// is recorded in its state).
template <class TB, class TF, int NQ>
__global__ void __launch_bounds__(kBlockTeam)
    block_mixed_kernel(const Params* __restrict__ Pc) {
  extern __shared__ __align__(16) char smem_all[];
  double* red = (double*)smem_all;
  char* smem = smem_all + 128;
  __shared__ int s_slot;
  const Params* P0 = Pc;
  while (true) {
    if (threadIdx.x == 0) s_slot = atomicAdd(P0->work_counter, 1);
    __syncthreads();
    const int slot = s_slot;
    __syncthreads();
    if (slot >= P0->n_slots) break;
    SlotState S = P0->st[slot];
    if (S.status != BIPM_RUNNING) continue;
    const Params* P = Pc + S.cls;
    Ctx<TB, TF, NQ, 0> c;
    make_ctx(c, P, slot, (int)threadIdx.x, (int)blockDim.x, red, smem);
    run_slot(c, S, 0, 0);
    __syncthreads();
    if (threadIdx.x == 0) P0->st[slot] = S;
    __syncthreads();
  }
}

// offsets of the per-slot arrays for problems of dims d (host)
Layout make_layout(const Dims& d, int precision);

// host-side accessors of the kernel entry points of one precision; the _q1
// variants are specialised for one quadrotor per problem
void* iter_kernel_f64();
void* init_kernel_f64();
void* queue_kernel_f64();
void* block_kernel_f64();
void* iter_kernel_f32();
void* init_kernel_f32();
void* queue_kernel_f32();
void* block_kernel_f32();
void* iter_kernel_df();
void* init_kernel_df();
void* block_kernel_df();
void* queue_kernel_df();
void* iter_kernel_f64_q1();
void* queue_kernel_f64_q1();
void* block_kernel_f64_q1();
void* iter_kernel_f32_q1();
void* queue_kernel_f32_q1();
void* block_kernel_f32_q1();
void* iter_kernel_df_q1();
void* queue_kernel_df_q1();
void* block_kernel_df_q1();
void* queue_mixed_f64();
void* queue_mixed_f32();
void* block_mixed_f64();
void* block_mixed_f32();

}  // namespace bipm
