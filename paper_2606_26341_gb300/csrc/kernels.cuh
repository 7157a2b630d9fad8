// Kernel templates of the batched solver: the persistent iteration kernel
// (warp per problem, problems taken from an atomic work counter) and the
// slot initialisation kernel.  Instantiated once per precision in
// kernels_f64.cu and kernels_f32.cu.
#pragma once

#include "ipm_iter.cuh"

namespace bipm {

constexpr int kWarpsPerBlock = 4;

template <class TB, class TF>
__device__ void make_ctx(Ctx<TB, TF>& c, const Params* P, int slot, int lane, char* smem) {
  c.P = P;
  c.d = P->d;
  c.L = P->L;
  c.lane = lane;
  c.slot = slot;
  c.f = P->f64 + (long long)slot * P->L.slot_f64;
  c.blk = (TB*)P->tb + (long long)slot * P->L.slot_tb;
  TF* fb = (TF*)P->tf + (long long)slot * P->L.fac_size;
  c.fac = make_fac<TF>(fb, P->L);
  if constexpr (sizeof(TF) == 8)
    c.fac64 = make_fac<double>((double*)fb, P->L);
  else
    c.fac64 = make_fac<double>(c.f + P->L.f64_fac, P->L);
  c.th = P->theta + (long long)slot * P->d.n_theta;
  c.smem = smem;
  c.resto = 0;
  c.nw = P->d.n;
  c.mu = 0.0;
  c.zeta = 0.0;
  c.dw = 0.0;
  c.use64 = 0;
  c.n_ir = 0;
  c.n_esc = 0;
  c.n_fact = 0;
  c.n_solve = 0;
  c.n_trial = 0;
}

// final objective, scaled KKT error and infeasibility of the original problem
template <class TB, class TF>
__device__ void slot_metrics(Ctx<TB, TF>& c, SlotState& S) {
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

template <class TB, class TF>
__global__ void __launch_bounds__(32 * kWarpsPerBlock)
    ipm_kernel(const Params* __restrict__ P, int n_iter) {
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
    Ctx<TB, TF> c;
    make_ctx(c, P, slot, lane, smem);
    if (n_iter <= 0) {
      while (S.status == BIPM_RUNNING) iterate(c, S);
    } else {
      for (int it = 0; it < n_iter && S.status == BIPM_RUNNING; ++it) iterate(c, S);
    }
    slot_metrics(c, S);
    __syncwarp();
    if (lane == 0) P->st[slot] = S;
    __syncwarp();
  }
}

// default starting point, pushed inside the bounds (IPOPT initialisation)
__device__ __forceinline__ double push_into_bounds(int kind, double v) {
  if (kind == VK_BOX) {
    double width = kUmax - 0.0;
    double pl = fmin(kBoundPush * fmax(1.0, 0.0), kBoundFrac * width);
    double pu = fmin(kBoundPush * fmax(1.0, kUmax), kBoundFrac * width);
    return fmin(fmax(v, 0.0 + pl), kUmax - pu);
  }
  if (kind == VK_LOWER) return fmax(v, 0.0 + kBoundPush * fmax(1.0, 0.0));
  return v;
}

template <class TB, class TF>
__global__ void init_kernel(const Params* __restrict__ P, int first, int count,
                            const double* __restrict__ guess, const double* __restrict__ yguess) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= count) return;
  const int slot = first + gw;
  const Dims& d = P->d;
  const Layout& L = P->L;
  double* f = P->f64 + (long long)slot * L.slot_f64;
  const double* th = P->theta + (long long)slot * d.n_theta;
  double* w = f + L.x;
  double* zl = f + L.zl;
  double* zu = f + L.zu;
  double* y = f + L.y;
  for (int i = lane; i < d.n; i += 32) {
    VarInfo vi = var_info(d, i);
    double v;
    if (guess) {
      v = guess[(long long)gw * d.n + i];
    } else if (vi.loc < d.nx) {
      v = th[d.th_x + vi.loc];
    } else if (vi.kind == VK_BOX) {
      v = kHover;
    } else {
      int r = vi.loc - d.nx - (vi.k < d.N ? d.nu : 0);
      IneqRow row = ineq_row(d, th, th + d.th_x, r);
      v = row.gval;
    }
    w[i] = push_into_bounds(vi.kind, v);
    zl[i] = has_lower(vi.kind) ? 1.0 : 0.0;
    zu[i] = has_upper(vi.kind) ? 1.0 : 0.0;
    f[L.xr + i] = 0.0;
  }
  for (int i = lane; i < 2 * d.m; i += 32) {
    w[d.n + i] = 0.0;
    zl[d.n + i] = 0.0;
    zu[d.n + i] = 0.0;
  }
  for (int i = lane; i < d.m; i += 32) y[i] = yguess ? yguess[(long long)gw * d.m + i] : 0.0;
  if (lane == 0) {
    SlotState S;
    memset(&S, 0, sizeof(S));
    S.status = BIPM_RUNNING;
    S.mode = MODE_NORMAL;
    S.need_init = 1;
    S.need_y_ls = yguess ? 0 : 1;
    S.mu = P->opt.mu_init;
    S.problem_id = slot;
    P->st[slot] = S;
  }
}


// host-side accessors of the kernel entry points of one precision
void* iter_kernel_f64();
void* init_kernel_f64();
void* iter_kernel_f32();
void* init_kernel_f32();

}  // namespace bipm
