// One fused interior-point iteration for one problem, executed by one warp.
//
// Every problem of a batch runs this same code; the per-problem state record
// (mode, barrier parameter, filter, status) decides which of the branches of
// Table I a problem takes.  Branch decisions are warp-uniform, so problems only
// diverge across warps, never inside one: the heterogeneous iteration fusion of
// Sec. V realised as per-problem control flow in one kernel, without
// per-branch launches.
//
// Linear algebra: the augmented system Eq. 7 of one NMPC problem is block
// banded.  Slacks and inequality multipliers are eliminated stage by stage,
// the initial-state row fixes Delta x_0, and the remaining optimal-control KKT
// system is factorised by a backward Riccati recursion.  The inertia required
// after Eq. 7 (n positive, m negative eigenvalues) holds exactly when every
// stage pivot block R^_k is positive definite (in restoration also the state
// pivots I + D^1/2 P D^1/2), so the Cholesky factorisations of these blocks
// are the inertia test.
#pragma once

#include "common.cuh"
#include "quad_model.cuh"
#include "tri_index.cuh"

namespace bipm {

// Loops that stride over a team's lanes are never unrolled ("unroll 1" here
// and on every such loop below): many warps of one SM run different parts of
// this code at once, and the smaller instruction footprint measured faster
// than the unrolled copies.
#define LANE_LOOP(i, n) _Pragma("unroll 1") for (int i = lane; i < (n); i += c.T)

template <class T>
struct Fac {  // factor arrays of one slot in precision T
  T *Pt, *K, *Lr, *LM, *Yr, *kff, *ptv;
};

template <class T>
__device__ __forceinline__ Fac<T> make_fac(T* base, const Layout& L) {
  Fac<T> f;
  f.Pt = base + L.Pt;
  f.K = base + L.K;
  f.Lr = base + L.Lr;
  f.LM = base + L.LM;
  f.Yr = base + L.Yr;
  f.kff = base + L.kff;
  f.ptv = base + L.ptv;
  return f;
}

enum FactorFlags : int { FF_IDENT = 1, FF_RESTO = 2 };

// Team size of a kernel: TM = 32 fixes a one-warp team at compile time (the
// block-team branches of the team primitives fold away); TM = 0 keeps it a
// run-time field (block teams, T = blockDim.x).
template <int TM>
struct TeamSize {
  static constexpr int T = TM;
};
template <>
struct TeamSize<0> {
  int T;
};

template <class TB, class TF, int NQ, int TM>
struct Ctx : TeamSize<TM> {
  const Params* P;
  DimsT<NQ> d;         // problem sizes (nq, nx, nu compile-time when NQ > 0)
  Layout L;
  int lane;            // thread index within the team
  double* red;         // shared reduction buffer (block teams)
  int slot;
  double* f;           // this slot's FP64 arrays
  TB* blk;             // derivative blocks
  Fac<TF> fac;         // factor arrays in the factorisation precision
  Fac<double> fac64;   // FP64 factor arrays (= fac when TF is double)
  const double* th;    // theta of this slot
  char* smem;          // per-warp shared scratch
  char* gscratch;      // per-slot global scratch (used when shared memory is too small)
  int smem_bytes;      // bytes of `smem`
  // phase data of the current iteration
  int resto;
  int nw;              // primal length of the current phase (n or n + 2m)
  double mu;           // barrier parameter of the current phase
  double zeta;         // restoration: sqrt(mu) at its start
  double dw;           // regularisation used in the last factorisation
  int use64;           // 1: the last factorisation is the FP64 one
  int n_ir, n_esc;
  int esc_failed;      // the FP64 solve after a failed refinement missed its accuracy test
  int n_fact, n_solve, n_trial;  // work counters of the current iteration
  int n_fact32, n_solve32;        // ... of which in FP32
};

__device__ __forceinline__ double sq(double a) { return a * a; }

// 12-term dot product a[r*sa] * b[r*sb] with three independent partial sums
// (shorter dependency chains for the latency-bound stage products)
template <class TX>
__device__ __forceinline__ TX dot12(const TX* a, int sa, const TX* b, int sb) {
  TX a0 = a[0] * b[0], a1 = a[sa] * b[sb], a2 = a[2 * sa] * b[2 * sb];
#pragma unroll
  for (int r = 3; r < 12; r += 3) {
    a0 += a[r * sa] * b[r * sb];
    a1 += a[(r + 1) * sa] * b[(r + 1) * sb];
    a2 += a[(r + 2) * sa] * b[(r + 2) * sb];
  }
  return (a0 + a1) + a2;
}

// strided walk over the entries of an R x C row-major index space without a
// division per entry: (i, j) of entry e = lane, lane + T, ...
#define MAT_LOOP_BEGIN(i, j, R, C)                   \
  {                                                  \
    const int C_ = (C), RC_ = (R) * (C);             \
    int i = lane / C_, j = lane - (lane / C_) * C_;  \
    _Pragma("unroll 1") for (int e = lane; e < RC_; e += c.T) {
#define MAT_LOOP_END(i, j)     \
  j += c.T;                    \
  while (j >= C_) {            \
    j -= C_;                   \
    ++i;                       \
  }                            \
  }                            \
  }

// ------------------------------------------------------------ index helpers
struct VarInfo {
  int kind;   // VK_FREE, VK_BOX, VK_LOWER
  int k;      // stage
  int loc;    // position in the stage block
};

template <class D>
__device__ __forceinline__ VarInfo var_info(const D& d, int i) {
  VarInfo v;
  if (i < d.nx + d.nu) {
    v.k = 0;
    v.loc = i;
    v.kind = i < d.nx ? VK_FREE : VK_BOX;
    return v;
  }
  int j = i - (d.nx + d.nu);
  int blk = d.nx + d.nu + d.ni;
  v.k = 1 + j / blk;
  v.loc = j - (v.k - 1) * blk;
  if (v.k >= d.N)
    v.kind = v.loc < d.nx ? VK_FREE : VK_LOWER;
  else
    v.kind = v.loc < d.nx ? VK_FREE : (v.loc < d.nx + d.nu ? VK_BOX : VK_LOWER);
  return v;
}

// kind of entry i of a W-sized vector (x, then p, then n)
template <class D>
__device__ __forceinline__ int wkind(const D& d, int i) {
  return i < d.n ? var_kind(d, i) : VK_LOWER;
}
__device__ __forceinline__ bool has_lower(int kind) { return kind != VK_FREE; }
__device__ __forceinline__ bool has_upper(int kind) { return kind == VK_BOX; }

// Bounded entries among the first `len` entries of a W-sized vector (len = n,
// or n + 2m in restoration), numbered densely: b < N nu are the inputs (box
// bounds), then the N ni slacks, then the elastics p, n (lower bounds).  FP64
// instructions cost the same whatever the number of active lanes, so loops
// over bounds run over this numbering with every lane busy instead of
// skipping the free entries of a W-sized loop.
template <class D>
__device__ __forceinline__ int n_bounded(const D& d, int len) {
  return d.N * d.nu + d.N * d.ni + (len - d.n);
}
template <class D>
__device__ __forceinline__ int bnd_index(const D& d, int b, int& kind) {
  const int nu_all = d.N * d.nu;
  if (b < nu_all) {
    const int k = b / d.nu;
    kind = VK_BOX;
    return off_u(d, k) + (b - k * d.nu);
  }
  b -= nu_all;
  const int ni_all = d.N * d.ni;
  kind = VK_LOWER;
  if (b < ni_all) {
    const int k = b / d.ni;
    return off_s(d, k + 1) + (b - k * d.ni);
  }
  return d.n + (b - ni_all);
}

// ------------------------------------------------------ reference trajectory
// reference state component j of quad q at stage k: circle position and
// velocity, zero attitude and body rates (evaluated once per problem)
template <class D>
__device__ __forceinline__ double ref_value(const double* th, const D& d, int k, int q, int j) {
  if (j >= 6) return 0.0;
  const double* r = th + d.th_ref + 6 * q;
  double t = k * d.dt;
  double a = r[4] * t + r[5];
  double sa, ca;
  sincos(a, &sa, &ca);
  switch (j) {
    case 0: return r[0] + r[3] * ca;
    case 1: return r[1] + r[3] * sa;
    case 2: return r[2];
    case 3: return -r[3] * r[4] * sa;
    case 4: return r[3] * r[4] * ca;
    default: return 0.0;
  }
}

template <class D>
__device__ __forceinline__ double cost_weight(const D& d, int k, int j) {
  return q_weight(j) * (k == d.N ? kQNscale : 1.0);
}

// --------------------------------------------------------- inequality rows
// Value and gradient (w.r.t. the quad positions) of inequality j of a stage.
struct IneqRow {
  int q0, q1;      // quads involved (q1 < 0: one quad)
  int ncomp;       // position components involved per quad (3, or 2 for cylinders)
  double gval;     // g(x)
  double grad[6];  // d g / d p_q0 (3) then d g / d p_q1 (3)
  double hdiag;    // Hessian of g: hdiag * (I on involved components); pairs: +-hdiag
};

// Centre of moving sphere o at stage k (time k dt): c + v k dt.
template <class D>
__device__ __forceinline__ void moving_centre(const D& d, const double* th, int o, int k, double* cen) {
  const double* s = th + d.th_mov + 7 * o;
  const double t = k * d.dt;
  cen[0] = s[0] + s[4] * t;
  cen[1] = s[1] + s[5] * t;
  cen[2] = s[2] + s[6] * t;
}

template <class D>
__device__ __forceinline__ IneqRow ineq_row(const D& d, const double* th, const double* xk,
                                            int j, int k) {
  IneqRow r;
  r.q1 = -1;
  r.hdiag = 2.0;
  int nsq = d.nq * d.n_sph;
  int ncq = d.nq * d.n_cyl;
  int nmq = d.nq * d.n_mov;
  if (j >= nsq + ncq && j < nsq + ncq + nmq) {
    const int jj = j - nsq - ncq;
    const int q = jj / d.n_mov, o = jj - q * d.n_mov;
    double cen[3];
    moving_centre(d, th, o, k, cen);
    const double* p = xk + 12 * q;
    const double rad = th[d.th_mov + 7 * o + 3];
    double dx = p[0] - cen[0], dy = p[1] - cen[1], dz = p[2] - cen[2];
    r.q0 = q;
    r.ncomp = 3;
    r.gval = dx * dx + dy * dy + dz * dz - rad * rad;
    r.grad[0] = 2 * dx; r.grad[1] = 2 * dy; r.grad[2] = 2 * dz;
    return r;
  }
  if (j >= nsq + ncq) j -= nmq;  // pair rows follow the moving spheres
  if (j < nsq) {
    int q = j / d.n_sph, o = j - (j / d.n_sph) * d.n_sph;
    const double* s = th + d.th_sph + 4 * o;
    const double* p = xk + 12 * q;
    double dx = p[0] - s[0], dy = p[1] - s[1], dz = p[2] - s[2];
    r.q0 = q;
    r.ncomp = 3;
    r.gval = dx * dx + dy * dy + dz * dz - s[3] * s[3];
    r.grad[0] = 2 * dx; r.grad[1] = 2 * dy; r.grad[2] = 2 * dz;
  } else if (j < nsq + ncq) {
    int jj = j - nsq;
    int q = jj / d.n_cyl, o = jj - (jj / d.n_cyl) * d.n_cyl;
    const double* s = th + d.th_cyl + 3 * o;
    const double* p = xk + 12 * q;
    double dx = p[0] - s[0], dy = p[1] - s[1];
    r.q0 = q;
    r.ncomp = 2;
    r.gval = dx * dx + dy * dy - s[2] * s[2];
    r.grad[0] = 2 * dx; r.grad[1] = 2 * dy; r.grad[2] = 0.0;
  } else {
    int rem = j - nsq - ncq;
    int a = 0;
    while (rem >= d.nq - 1 - a) { rem -= d.nq - 1 - a; ++a; }
    int b = a + 1 + rem;
    const double* pa = xk + 12 * a;
    const double* pb = xk + 12 * b;
    double dx = pa[0] - pb[0], dy = pa[1] - pb[1], dz = pa[2] - pb[2];
    r.q0 = a;
    r.q1 = b;
    r.ncomp = 3;
    r.gval = dx * dx + dy * dy + dz * dz - d.pair_d * d.pair_d;
    r.grad[0] = 2 * dx; r.grad[1] = 2 * dy; r.grad[2] = 2 * dz;
    r.grad[3] = -2 * dx; r.grad[4] = -2 * dy; r.grad[5] = -2 * dz;
  }
  return r;
}

// Gradient of inequality j with respect to the positions (value not formed):
// d g / d p_q0 = g[0..ncomp), and for a pair row d g / d p_q1 = -g.
struct IneqGrad {
  int q0, q1, ncomp;
  double g[3];
};
template <class D>
__device__ __forceinline__ IneqGrad ineq_grad(const D& d, const double* th, const double* xk, int j, int k) {
  IneqGrad r;
  r.q1 = -1;
  const int nsq = d.nq * d.n_sph, ncq = d.nq * d.n_cyl, nmq = d.nq * d.n_mov;
  if (j >= nsq + ncq && j < nsq + ncq + nmq) {
    const int jj = j - nsq - ncq;
    const int q = jj / d.n_mov, o = jj - q * d.n_mov;
    double cen[3];
    moving_centre(d, th, o, k, cen);
    const double* p = xk + 12 * q;
    r.q0 = q;
    r.ncomp = 3;
    r.g[0] = 2 * (p[0] - cen[0]); r.g[1] = 2 * (p[1] - cen[1]); r.g[2] = 2 * (p[2] - cen[2]);
    return r;
  }
  if (j >= nsq + ncq) j -= nmq;
  if (j < nsq) {
    const int q = j / d.n_sph, o = j - q * d.n_sph;
    const double* s = th + d.th_sph + 4 * o;
    const double* p = xk + 12 * q;
    r.q0 = q;
    r.ncomp = 3;
    r.g[0] = 2 * (p[0] - s[0]); r.g[1] = 2 * (p[1] - s[1]); r.g[2] = 2 * (p[2] - s[2]);
  } else if (j < nsq + ncq) {
    const int jj = j - nsq;
    const int q = jj / d.n_cyl, o = jj - q * d.n_cyl;
    const double* s = th + d.th_cyl + 3 * o;
    const double* p = xk + 12 * q;
    r.q0 = q;
    r.ncomp = 2;
    r.g[0] = 2 * (p[0] - s[0]); r.g[1] = 2 * (p[1] - s[1]); r.g[2] = 0.0;
  } else {
    int rem = j - nsq - ncq;
    int a = 0;
    while (rem >= d.nq - 1 - a) { rem -= d.nq - 1 - a; ++a; }
    const int b = a + 1 + rem;
    const double* pa = xk + 12 * a;
    const double* pb = xk + 12 * b;
    r.q0 = a;
    r.q1 = b;
    r.ncomp = 3;
    r.g[0] = 2 * (pa[0] - pb[0]); r.g[1] = 2 * (pa[1] - pb[1]); r.g[2] = 2 * (pa[2] - pb[2]);
  }
  return r;
}
// The same gradient read from the table fill_ineq_grad wrote for the iterate
// (row t = (k - 1) ni + j of stage k >= 1).
template <class D>
__device__ __forceinline__ IneqGrad ineq_grad_tab(const D& d, const double* igr, int t, int j) {
  IneqGrad r;
  r.q1 = -1;
  const int nsq = d.nq * d.n_sph, ncq = d.nq * d.n_cyl, nmq = d.nq * d.n_mov;
  if (j >= nsq + ncq && j < nsq + ncq + nmq) {
    r.q0 = (j - nsq - ncq) / d.n_mov;
    r.ncomp = 3;
    const double* g = igr + 3LL * t;
    r.g[0] = g[0];
    r.g[1] = g[1];
    r.g[2] = g[2];
    return r;
  }
  if (j >= nsq + ncq) j -= nmq;
  if (j < nsq) {
    r.q0 = j / d.n_sph;
    r.ncomp = 3;
  } else if (j < nsq + ncq) {
    r.q0 = (j - nsq) / d.n_cyl;
    r.ncomp = 2;
  } else {
    int rem = j - nsq - ncq;
    int a = 0;
    while (rem >= d.nq - 1 - a) { rem -= d.nq - 1 - a; ++a; }
    r.q0 = a;
    r.q1 = a + 1 + rem;
    r.ncomp = 3;
  }
  const double* g = igr + 3LL * t;
  r.g[0] = g[0];
  r.g[1] = g[1];
  r.g[2] = g[2];
  return r;
}

// component comp (< 3) of quad q of that gradient
__device__ __forceinline__ double grad_pos(const IneqGrad& r, int q, int comp) {
  if (comp >= r.ncomp) return 0.0;
  if (q == r.q0) return r.g[comp];
  if (q == r.q1) return -r.g[comp];
  return 0.0;
}
// Hessian of inequality row r (squared distances: 2 I, pairs +-2 I) at
// position components (qa, ca), (qb, cb)
__device__ __forceinline__ double hess_pos(const IneqGrad& r, int qa, int ca, int qb, int cb) {
  if (ca != cb || ca >= r.ncomp) return 0.0;
  const double sa = qa == r.q0 ? 1.0 : (qa == r.q1 ? -1.0 : 0.0);
  const double sb = qb == r.q0 ? 1.0 : (qb == r.q1 ? -1.0 : 0.0);
  return 2.0 * sa * sb;
}

// ---------------------------------------------------------------- evaluation
// Constraint values c(x) (original problem) into cout and the objective f(x).
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double eval_values(Ctx<TB, TF, NQ, TM>& c, const double* x, double* cout,
                              bool dynamics = true) {
  const auto& d = c.d;
  const int lane = c.lane;
  LANE_LOOP(i, d.nx) cout[i] = x[i] - c.th[d.th_x + i];
  #pragma unroll 1
  for (int t = lane; t < (dynamics ? d.N * d.nq : 0); t += c.T) {
    int k = t / d.nq, q = t - (t / d.nq) * d.nq;
    double xx[12], uu[4], F[12];
    const double* xk = x + off_x(d, k) + 12 * q;
    const double* uk = x + off_u(d, k) + 4 * q;
#pragma unroll
    for (int i = 0; i < 12; ++i) xx[i] = xk[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) uu[i] = uk[i];
    rk4_value<double>(xx, uu, d.dt, F);
    const double* xn = x + off_x(d, k + 1) + 12 * q;
    double* cr = cout + row_dyn(d, k) + 12 * q;
#pragma unroll
    for (int i = 0; i < 12; ++i) cr[i] = xn[i] - F[i];
  }
  #pragma unroll 1
  for (int t = lane; t < d.N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, j = t - (t / d.ni) * d.ni;
    IneqRow r = ineq_row(d, c.th, x + off_x(d, k), j, k);
    cout[row_ineq(d, k) + j] = r.gval - x[off_s(d, k) + j];
  }
  double fs = 0.0;
  #pragma unroll 1
  for (int t = lane; t < (d.N + 1) * d.nx; t += c.T) {
    int k = t / d.nx, i = t - (t / d.nx) * d.nx;
    int q = i / 12, j = i - 12 * (i / 12);
    double e = x[off_x(d, k) + i] - c.f[c.L.xref + k * d.nx + i];
    (void)q;
    fs += cost_weight(d, k, j) * e * e;
  }
  #pragma unroll 1
  for (int t = lane; t < d.N * d.nu; t += c.T) {
    int k = t / d.nu, i = t - (t / d.nu) * d.nu;
    double e = x[off_u(d, k) + i] - kHover;
    fs += kRweight * e * e;
  }
  team_sync(c);
  return team_sum(c, fs);
}

// Gradient of the objective of the current phase into g (W-sized).
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void eval_grad(Ctx<TB, TF, NQ, TM>& c, const double* x, double* g) {
  const auto& d = c.d;
  const int lane = c.lane;
  const double* xr = c.f + c.L.xr;
  LANE_LOOP(i, c.nw) {
    double v;
    if (i >= d.n) {
      v = kRho;
    } else if (c.resto) {
      double dr = fmin(1.0, 1.0 / fmax(fabs(xr[i]), 1e-300));
      v = c.zeta * dr * dr * (x[i] - xr[i]);
    } else {
      VarInfo vi = var_info(d, i);
      if (vi.loc < d.nx) {
        int q = vi.loc / 12, j = vi.loc - 12 * (vi.loc / 12);
        v = 2.0 * cost_weight(d, vi.k, j) * (x[i] - c.f[c.L.xref + vi.k * d.nx + vi.loc]);
        (void)q;
      } else if (vi.kind == VK_BOX) {
        v = 2.0 * kRweight * (x[i] - kHover);
      } else {
        v = 0.0;
      }
    }
    g[i] = v;
  }
  team_sync(c);
}

// Objective of the restoration problem: rho sum(p + n) + zeta/2 |D_R (x - x_R)|^2.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double resto_objective(Ctx<TB, TF, NQ, TM>& c, const double* w) {
  const auto& d = c.d;
  const int lane = c.lane;
  const double* xr = c.f + c.L.xr;
  double acc = 0.0;
  LANE_LOOP(i, c.nw) {
    if (i >= d.n) {
      acc += kRho * w[i];
    } else {
      double dr = fmin(1.0, 1.0 / fmax(fabs(xr[i]), 1e-300));
      acc += 0.5 * c.zeta * sq(dr * (w[i] - xr[i]));
    }
  }
  return team_sum(c, acc);
}

// Jacobian / Hessian blocks of the dynamics by forward-over-reverse dual
// numbers: lane task (k, q, j) seeds direction j of (eta, omega, u) of quad q
// at stage k.  The columns of A for p and v are constant (F is affine in p, v)
// and the Hessian of lam^T F vanishes in those rows, so only ten directions
// carry derivatives.  lam = -y_dyn (the Lagrangian term is +y^T (x_{k+1} - F)).
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void eval_blocks(Ctx<TB, TF, NQ, TM>& c, const double* x, const double* y, bool hess) {
  const auto& d = c.d;
  const int lane = c.lane;
  typedef Dual<TB> DT;
  const int ntask = d.N * d.nq * 10;
  #pragma unroll 1
  for (int t = lane; t < ntask; t += c.T) {
    int j = t - (t / 10) * 10;
    int kq = t / 10;
    int k = kq / d.nq, q = kq - (kq / d.nq) * d.nq;
    const double* xk = x + off_x(d, k) + 12 * q;
    const double* uk = x + off_u(d, k) + 4 * q;
    DT xx[12], uu[4], F[12], gx[12], gu[4];
    TB lam[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      xx[i] = DT{(TB)xk[i], (TB)0};
      lam[i] = hess ? (TB)(-y[row_dyn(d, k) + 12 * q + i]) : (TB)0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) uu[i] = DT{(TB)uk[i], (TB)0};
    if (j < 6)
      xx[6 + j].d = (TB)1;
    else
      uu[j - 6].d = (TB)1;
    rk4_fwd_rev<DT>(xx, uu, (TB)d.dt, lam, F, gx, gu);
    TB* A = c.blk + c.L.A + ((long long)k * d.nq + q) * 144;
    TB* B = c.blk + c.L.B + ((long long)k * d.nq + q) * 48;
    TB* H = c.blk + c.L.H + ((long long)k * d.nq + q) * 100;
    if (j < 6) {
#pragma unroll
      for (int r = 0; r < 12; ++r) A[(6 + j) * 12 + r] = F[r].d;
    } else {
#pragma unroll
      for (int r = 0; r < 12; ++r) B[(j - 6) * 12 + r] = F[r].d;
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) H[j * 10 + r] = gx[6 + r].d;
#pragma unroll
    for (int r = 0; r < 4; ++r) H[j * 10 + 6 + r] = gu[r].d;
    if (j == 0) {
      for (int col = 0; col < 6; ++col)
        for (int r = 0; r < 12; ++r) {
          TB v = (TB)0;
          if (col < 3) v = (r == col) ? (TB)1 : (TB)0;
          else v = (r == col - 3) ? (TB)d.dt : ((r == col) ? (TB)1 : (TB)0);
          A[col * 12 + r] = v;
        }
    }
  }
  team_sync(c);
}

// J^T y of the original constraints (x-part, n entries) in FP64, plus the
// elastic parts (-y, +y) in restoration.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void eval_jty(Ctx<TB, TF, NQ, TM>& c, const double* x, const double* y, double* jty,
                         double* cout = nullptr) {
  const auto& d = c.d;
  const int lane = c.lane;
  #pragma unroll 1
  for (int t = lane; t < d.N * d.nq; t += c.T) {
    int k = t / d.nq, q = t - (t / d.nq) * d.nq;
    double xx[12], uu[4], F[12], gx[12], gu[4], lam[12];
    const double* xk = x + off_x(d, k) + 12 * q;
    const double* uk = x + off_u(d, k) + 4 * q;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      xx[i] = xk[i];
      lam[i] = -y[row_dyn(d, k) + 12 * q + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) uu[i] = uk[i];
    rk4_fwd_rev<double>(xx, uu, d.dt, lam, F, gx, gu);
    if (cout) {
      const double* xn = x + off_x(d, k + 1) + 12 * q;
      double* cr = cout + row_dyn(d, k) + 12 * q;
#pragma unroll
      for (int i = 0; i < 12; ++i) cr[i] = xn[i] - F[i];
    }
    const double* yprev = y + (k == 0 ? 0 : row_dyn(d, k - 1)) + 12 * q;
    double* jx = jty + off_x(d, k) + 12 * q;
#pragma unroll
    for (int i = 0; i < 12; ++i) jx[i] = gx[i] + yprev[i];
    double* ju = jty + off_u(d, k) + 4 * q;
#pragma unroll
    for (int i = 0; i < 4; ++i) ju[i] = gu[i];
  }
  LANE_LOOP(i, d.nx) jty[off_x(d, d.N) + i] = y[row_dyn(d, d.N - 1) + i];
  team_sync(c);
  // inequality rows: + G_k^T y_ineq on the positions, - y_ineq on the slacks
  #pragma unroll 1
  for (int t = lane; t < d.N * 3 * d.nq; t += c.T) {
    int k = 1 + t / (3 * d.nq);
    int pc = t - (t / (3 * d.nq)) * (3 * d.nq);
    int q = pc / 3, comp = pc - 3 * (pc / 3);
    int i = 12 * q + comp;
    const double* xk = x + off_x(d, k);
    const double* yi = y + row_ineq(d, k);
    double acc = 0.0;
    for (int r = 0; r < d.ni; ++r) acc += grad_pos(ineq_grad(d, c.th, xk, r, k), q, comp) * yi[r];
    jty[off_x(d, k) + i] += acc;
  }
  #pragma unroll 1
  for (int t = lane; t < d.N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, r = t - (t / d.ni) * d.ni;
    jty[off_s(d, k) + r] = -y[row_ineq(d, k) + r];
  }
  if (c.resto) {
    LANE_LOOP(i, d.m) {
      jty[d.n + i] = -y[i];
      jty[d.n + d.m + i] = y[i];
    }
  }
  team_sync(c);
}

// ------------------------------------------------- barrier quantities (FP64)
// Sigma_i = z_L/s_L + z_U/s_U of W-entry i, from the array fill_sigma wrote
// for the current iterate.
template <class TB, class TF, int NQ, int TM>
__device__ __forceinline__ double sigma_of(Ctx<TB, TF, NQ, TM>& c, int i) {
  return c.f[c.L.sig + i];
}

template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void fill_sigma(Ctx<TB, TF, NQ, TM>& c) {
  const double* x = c.f + c.L.x;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  double* sg = c.f + c.L.sig;
  #pragma unroll 1
  for (int i = c.lane; i < c.nw; i += c.T) sg[i] = 0.0;
  team_sync(c);
  const int nb = n_bounded(c.d, c.nw);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(c.d, b, kind);
    double v = zl[i] / x[i];
    if (kind == VK_BOX) v += zu[i] / (kUmax - x[i]);
    sg[i] = v;
  }
  team_sync(c);
}

// Diagonal Hessian of the objective on W-entry i (cost weights, or zeta D_R^2
// in restoration, or 1 for the least-squares multiplier system).
template <class TB, class TF, int NQ, int TM>
__device__ __forceinline__ double obj_hdiag(Ctx<TB, TF, NQ, TM>& c, int i, int flags) {
  if (flags & FF_IDENT) return 1.0;
  const auto& d = c.d;
  if (i >= d.n) return 0.0;
  if (c.resto) {
    const double* xr = c.f + c.L.xr;
    double dr = fmin(1.0, 1.0 / fmax(fabs(xr[i]), 1e-300));
    return c.zeta * dr * dr;
  }
  VarInfo vi = var_info(d, i);
  if (vi.loc < d.nx) return 2.0 * cost_weight(d, vi.k, vi.loc - 12 * (vi.loc / 12));
  if (vi.kind == VK_BOX) return 2.0 * kRweight;
  return 0.0;
}

// Position gradients of every inequality row at the point x (the iterate),
// one pass over all rows; factorisation, solves and the KKT mat-vec read them.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void fill_ineq_grad(Ctx<TB, TF, NQ, TM>& c, const double* x) {
  const auto& d = c.d;
  double* igr = c.f + c.L.igr;
  #pragma unroll 1
  for (int t = c.lane; t < d.N * d.ni; t += c.T) {
    const int k = 1 + t / d.ni, j = t - (k - 1) * d.ni;
    const IneqGrad g = ineq_grad(d, c.th, x + off_x(d, k), j, k);
    igr[3 * t] = g.g[0];
    igr[3 * t + 1] = g.g[1];
    igr[3 * t + 2] = g.g[2];
  }
  team_sync(c);
}

// Condensation diagonals for regularisation dw:
//   slack (k, r):  D_s = H_ss + Sigma_s + dw,  E = D_s / (1 + D_s D_g)
//   row i (restoration): 1/(Sigma_p + dw), 1/(Sigma_n + dw), D = their sum
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void compute_diag(Ctx<TB, TF, NQ, TM>& c, double dw, int flags) {
  const auto& d = c.d;
  const int lane = c.lane;
  double* dsv = c.f + c.L.dsv;
  double* ev = c.f + c.L.ev;
  double* ipv = c.f + c.L.ipv;
  double* inv = c.f + c.L.inv;
  double* dv = c.f + c.L.dv;
  double* rds = c.f + c.L.rds;
  double* evr = c.f + c.L.evr;
  const double* w = c.f + c.L.x;
  const double* zl = c.f + c.L.zl;
  LANE_LOOP(i, d.m) {
    if (c.resto) {
      double ip = 1.0 / (zl[d.n + i] / w[d.n + i] + dw);
      double in = 1.0 / (zl[d.n + d.m + i] / w[d.n + d.m + i] + dw);
      ipv[i] = ip;
      inv[i] = in;
      dv[i] = ip + in;
    } else {
      ipv[i] = 0.0;
      inv[i] = 0.0;
      dv[i] = 0.0;
    }
  }
  team_sync(c);
  #pragma unroll 1
  for (int t = lane; t < d.N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, r = t - (t / d.ni) * d.ni;
    int vi = off_s(d, k) + r;
    double ds = (flags & FF_IDENT) ? 1.0 : obj_hdiag(c, vi, flags) + sigma_of(c, vi) + dw;
    double dg = dv[row_ineq(d, k) + r];
    dsv[t] = ds;
    rds[t] = 1.0 / ds;
    if (c.resto) {
      const double wr = 1.0 / (1.0 + ds * dg);
      evr[t] = wr;
      ev[t] = ds * wr;
    } else {
      evr[t] = 1.0;  // E = D_s when the row has no elastic term
      ev[t] = ds;
    }
  }
  team_sync(c);
}



// Position blocks of the condensed inequality rows for every stage at once,
// with the condensation weights of the last compute_diag:
//   qpos_k(a, b) = sum_r E_r g_r(a) g_r(b) + y_r H_r(a, b),
// a, b over the 3 nq position components of stage k (no Hessian term in the
// least-squares multiplier system).
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void ineq_blocks(Ctx<TB, TF, NQ, TM>& c, int flags) {
  const auto& d = c.d;
  const int lane = c.lane;
  const double* ev = c.f + c.L.ev;
  const int np = 3 * d.nq, npp = np * np;
  const double* igr = c.f + c.L.igr;
  const double* y = c.f + c.L.y;
  double* qpos = c.f + c.L.qpos;
  #pragma unroll 1
  for (int e = lane; e < d.N * npp; e += c.T) {
    const int k = 1 + e / npp, ab = e - (k - 1) * npp;
    const int a = ab / np, b = ab - a * np;
    const int qa = a / 3, ca = a - 3 * qa, qb = b / 3, cb = b - 3 * qb;
    const double* yk = y + row_ineq(d, k);
    double v = 0.0;
    for (int r = 0; r < d.ni; ++r) {
      const IneqGrad g = ineq_grad_tab(d, igr, (k - 1) * d.ni + r, r);
      v += ev[(k - 1) * d.ni + r] * grad_pos(g, qa, ca) * grad_pos(g, qb, cb);
      if (!(flags & FF_IDENT)) v += yk[r] * hess_pos(g, qa, ca, qb, cb);
    }
    qpos[e] = v;
  }
  team_sync(c);
}

// -------------------------------------------------------- factorisation
// Builds the condensed stage matrices and runs the Riccati recursion in
// precision TX.  Returns 0 if some pivot block is not positive definite
// (wrong inertia), 1 on success, 2 on success with a pivot inside the FP32
// guard band (the caller refactors in FP64).
template <class TX>
struct Scratch {
  TX *Pb, *PA, *PB, *Rh, *Sh, *Kb, *Ab, *Bb, *v0, *v1, *v2, *v3;
  double* R64;
};

template <class TX, class D>
__device__ __forceinline__ Scratch<TX> scratch(char* smem, const D& d) {
  Scratch<TX> s;
  TX* p = (TX*)smem;
  int nx = d.nx, nu = d.nu;
  s.Pb = p; p += nx * nx;
  s.PA = p; p += nx * nx;
  s.PB = p; p += nx * nu;
  s.Rh = p; p += nu * nu;
  s.Sh = p; p += nu * nx;
  s.Kb = p; p += nu * nx;
  s.Ab = p; p += 144 * d.nq;
  s.Bb = p; p += 48 * d.nq;
  s.v0 = p; p += nx;
  s.v1 = p; p += nx;
  s.v2 = p; p += nx;
  s.v3 = p; p += nx;
  size_t off = ((size_t)((char*)p - smem) + 15) & ~(size_t)15;
  s.R64 = (double*)(smem + off);
  return s;
}

// bytes of factorisation scratch for problems of dims d with elements of
// `elem` bytes (the FP64 Cholesky block is always double)
__host__ __device__ inline size_t scratch_bytes(int nq, int nx, int nu, int elem) {
  size_t e = (size_t)2 * nx * nx + 3 * (size_t)nx * nu + (size_t)nu * nu + 192 * (size_t)nq +
             4 * (size_t)nx;
  size_t b = ((e * elem + 15) & ~(size_t)15) + (size_t)nu * nu * 8;
  return (b + 127) & ~(size_t)127;
}

// shared memory when the scratch of precision TX fits, else the slot's
// global scratch region
template <class TX, class TB, class TF, int NQ, int TM>
__device__ __forceinline__ char* scratch_base(const Ctx<TB, TF, NQ, TM>& c) {
  return scratch_bytes(c.d.nq, c.d.nx, c.d.nu, (int)sizeof(TX)) <= (size_t)c.smem_bytes ? c.smem
                                                                                        : c.gscratch;
}

// v + entry (i, j) of Q~_k, the state block of the stage Hessian including the
// inequality terms (xdg: its diagonal, precomputed in TX, or null); the terms
// are added to v one at a time.
template <class TB, class TF, int NQ, int TM, class TX>
__device__ __forceinline__ TX state_term(Ctx<TB, TF, NQ, TM>& c, int k, int i, int j, double dw, int flags,
                                         const TX* xdg, TX v) {
  const auto& d = c.d;
  const bool ident = flags & FF_IDENT;
  if (i == j) {
    if (xdg)
      v += xdg[k * d.nx + i];
    else
      v += (TX)(obj_hdiag(c, off_x(d, k) + i, flags) + (ident ? 0.0 : dw));
  }
  const int qi = i / 12, qj = j / 12;
  const int ci = i - 12 * qi, cj = j - 12 * qj;
  if (!ident && k < d.N && qi == qj && ci >= 6 && cj >= 6) {
    const TB* H = c.blk + c.L.H + ((long long)k * d.nq + qi) * 100;
    v += (TX)H[(cj - 6) * 10 + (ci - 6)];
  }
  if (k >= 1 && ci < 3 && cj < 3 && d.ni > 0) {
    const int np = 3 * d.nq;
    v += (TX)c.f[c.L.qpos + (long long)(k - 1) * np * np + (3 * qi + ci) * np + 3 * qj + cj];
  }
  return v;
}

// Q~_k written to the full nx x nx block Q.
template <class TB, class TF, int NQ, int TM, class TX>
__device__ __noinline__ void add_state_block(Ctx<TB, TF, NQ, TM>& c, int k, TX* Q, double dw, int flags,
                                             const TX* xdg = nullptr) {
  const int lane = c.lane;
  const int nx = c.d.nx;
  MAT_LOOP_BEGIN(i, j, nx, nx)
    Q[e] = state_term<TB, TF, NQ, TM, TX>(c, k, i, j, dw, flags, xdg, (TX)0);
  MAT_LOOP_END(i, j)
}

// Cholesky of the n x n symmetric matrix in `a` (row-major, double) in place
// by the team: the lower triangle holds L below the diagonal and 1 / L_jj on
// it.  Returns false if a pivot is not positive and finite (every thread reads
// the same pivot, so the return is uniform).
template <class C>
__device__ inline bool warp_cholesky_rdiag(const C& c, double* a, int n) {
  const int lane = c.lane;
  for (int j = 0; j < n; ++j) {
    team_sync(c);
    // a_jj already holds the Schur complement pivot
    const double piv = a[j * n + j];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    const double il = rsqrt_fp64(piv);
    team_sync(c);
    if (lane == 0) a[j * n + j] = il;
    #pragma unroll 1
    for (int i = j + 1 + lane; i < n; i += c.T) a[i * n + j] *= il;
    team_sync(c);
    const int rem = n - j - 1;
    #pragma unroll 1
    for (int e = lane; e < rem * rem; e += c.T) {
      const int i = j + 1 + e / rem, t = j + 1 + (e - (e / rem) * rem);
      if (t <= i) a[i * n + t] -= a[i * n + j] * a[t * n + j];
    }
  }
  team_sync(c);
  return true;
}

// Cholesky of the nxn matrix in `a` (row-major, precision TX) in place by
// the team; lower triangle holds L.  Returns false if a pivot is not positive
// and finite (every thread reads the same pivot, so the return is uniform).
template <class C, class TX>
__device__ inline bool team_cholesky(const C& c, TX* a, int n) {
  const int lane = c.lane;
  for (int j = 0; j < n; ++j) {
    team_sync(c);
    const TX piv = a[j * n + j];
    if (!(piv > (TX)0) || !isfinite(piv)) return false;
    const TX l = sqrt(piv);
    const TX il = (TX)1 / l;
    team_sync(c);
    if (lane == 0) a[j * n + j] = l;
    #pragma unroll 1
    for (int i = j + 1 + lane; i < n; i += c.T) a[i * n + j] *= il;
    team_sync(c);
    const int rem = n - j - 1;
    #pragma unroll 1
    for (int e = lane; e < rem * rem; e += c.T) {
      const int i = j + 1 + e / rem, t = j + 1 + (e - (e / rem) * rem);
      if (t <= i) a[i * n + t] -= a[i * n + j] * a[t * n + j];
    }
  }
  team_sync(c);
  return true;
}

// FP64 inertia test of the pivot blocks R^_k, k in [k0, N), that an FP32
// factorisation assembled (stored as TX at R + k nu^2): one stage per thread,
// LDL^T in FP64 in the scratch a64 (N nu^2 doubles).  Returns 0 if a pivot is
// not positive, else 1, and the smallest ratio pivot / original diagonal.
template <class C, class TX>
__device__ inline int stage_pivot_check(const C& c, const TX* R, double* a64, int k0, int N, int nu,
                                        double& ratio) {
  int bad = 0;
  double rmin = 1.0;
  const int nn = nu * nu;
  #pragma unroll 1
  for (int k = k0 + c.lane; k < N; k += c.T) {
    double* a = a64 + (long long)k * nn;
    const TX* r = R + (long long)k * nn;
    for (int e = 0; e < nn; ++e) a[e] = (double)r[e];
    for (int j = 0; j < nu && !bad; ++j) {
      // pivot d_j = a_jj - sum_t l_jt^2 d_t (d_t on the diagonal, l_jt below it)
      double dj = a[j * nu + j];
      for (int t = 0; t < j; ++t) dj -= a[j * nu + t] * a[j * nu + t] * a[t * nu + t];
      if (!(dj > 0.0) || !isfinite(dj)) {
        bad = 1;
        break;
      }
      rmin = fmin(rmin, dj / (double)r[j * nu + j]);
      const double inv = 1.0 / dj;
      for (int i = j + 1; i < nu; ++i) {
        double v = a[i * nu + j];
        for (int t = 0; t < j; ++t) v -= a[i * nu + t] * a[j * nu + t] * a[t * nu + t];
        a[i * nu + j] = v * inv;
      }
      a[j * nu + j] = dj;
    }
  }
  bad = team_or(c, bad);
  ratio = team_min(c, rmin);
  return bad ? 0 : 1;
}

// Restoration: P~ = P - Y^T Y with Y = L_M^{-1} D^1/2 P, M = I + D^1/2 P D^1/2 = L_M L_M^T.
template <class TB, class TF, int NQ, int TM, class TX>
__device__ __noinline__ bool resto_transform(Ctx<TB, TF, NQ, TM>& c, TX* Pb, const double* D, TX* LM, TX* Y) {
  const auto& d = c.d;
  const int lane = c.lane;
  const int nx = d.nx;
  // M in LM (as TX) ; factor in double would need nx^2 doubles: factor in TX
  LANE_LOOP(e, nx * nx) {
    int i = e / nx, j = e - (e / nx) * nx;
    double v = sqrt(D[i]) * (double)Pb[e] * sqrt(D[j]) + (i == j ? 1.0 : 0.0);
    LM[e] = (TX)v;
  }
  team_sync(c);
  for (int j = 0; j < nx; ++j) {
    team_sync(c);
    double piv = (double)LM[j * nx + j];
    if (!(piv > 0.0) || !isfinite(piv)) return false;
    double l = sqrt(piv);
    team_sync(c);
    if (lane == 0) LM[j * nx + j] = (TX)l;
    #pragma unroll 1
    for (int i = j + 1 + lane; i < nx; i += c.T) LM[i * nx + j] = (TX)((double)LM[i * nx + j] / l);
    team_sync(c);
    int rem = nx - j - 1;
    #pragma unroll 1
    for (int e = lane; e < rem * rem; e += c.T) {
      int i = j + 1 + e / rem, t = j + 1 + (e - (e / rem) * rem);
      if (t <= i) LM[i * nx + t] = (TX)((double)LM[i * nx + t] - (double)LM[i * nx + j] * (double)LM[t * nx + j]);
    }
  }
  team_sync(c);
  // Y = L^{-1} (D^1/2 P): forward substitution, one column per lane
  #pragma unroll 1
  for (int col = lane; col < nx; col += c.T) {
    for (int i = 0; i < nx; ++i) {
      double acc = sqrt(D[i]) * (double)Pb[i * nx + col];
      for (int t = 0; t < i; ++t) acc -= (double)LM[i * nx + t] * (double)Y[t * nx + col];
      Y[i * nx + col] = (TX)(acc / (double)LM[i * nx + i]);
    }
  }
  team_sync(c);
  LANE_LOOP(e, nx * nx) {
    int i = e / nx, j = e - (e / nx) * nx;
    double acc = 0.0;
    for (int t = 0; t < nx; ++t) acc += (double)Y[t * nx + i] * (double)Y[t * nx + j];
    Pb[e] = (TX)((double)Pb[e] - acc);
  }
  team_sync(c);
  return true;
}

template <class TB, class TF, int NQ, int TM, class TX>
__device__ __noinline__ int factor(Ctx<TB, TF, NQ, TM>& c, Fac<TX> F, double dw, int flags, const double* y) {
  const auto& d = c.d;
  const int lane = c.lane;
  const int nx = d.nx, nu = d.nu, nq = d.nq, N = d.N;
  const bool ident = flags & FF_IDENT;
  const bool resto = flags & FF_RESTO;
  Scratch<TX> s = scratch<TX>(scratch_base<TX>(c), d);
  const double* dv = c.f + c.L.dv;
  c.n_fact++;
  if (sizeof(TX) == 4) c.n_fact32++;
  compute_diag(c, dw, flags);
  if (d.ni > 0) ineq_blocks(c, flags);
  double min_ratio = 1.0;
  // FP32 factorisation (never in restoration): the stage loop runs without
  // FP64 instructions.  The diagonal terms are formed once in FP64 and stored
  // in TX, the pivot blocks R^_k are kept for one FP64 inertia test of all
  // stages after the recursion; both live in the restoration-only arrays
  // LM (R^_k) and Yr (diagonals), which an FP32 factorisation never uses.
  constexpr bool f32 = sizeof(TX) == 4;
  constexpr bool pre_diag = f32 || std::is_same<TX, double>::value;
  const TX* xdg = nullptr;
  const TX* udg = nullptr;
  int k_fail32 = -1;
  if constexpr (pre_diag) {
    // FP32: the restoration-only array Yr; FP64: a workspace array of its own
    TX* dg;
    if constexpr (f32)
      dg = F.Yr;
    else
      dg = c.f + c.L.fdg;
    LANE_LOOP(e, (N + 1) * nx) {
      const int k = e / nx, i = e - k * nx;
      dg[e] = (TX)(obj_hdiag(c, off_x(d, k) + i, flags) + (ident ? 0.0 : dw));
    }
    LANE_LOOP(e, N * nu) {
      const int k = e / nu, a = e - k * nu;
      const int ui = off_u(d, k) + a;
      dg[(N + 1) * nx + e] = (TX)(obj_hdiag(c, ui, flags) + (ident ? 0.0 : sigma_of(c, ui) + dw));
    }
    team_sync(c);
    xdg = dg;
    udg = dg + (N + 1) * nx;
  }

  // terminal block P_N = Q~_N
  add_state_block<TB, TF, NQ, TM, TX>(c, N, s.Pb, dw, flags, xdg);
  team_sync(c);
  if (resto) {
    if (!resto_transform<TB, TF, NQ, TM, TX>(c, s.Pb, dv + row_dyn(d, N - 1), F.LM + (long long)N * nx * nx,
                                     F.Yr + (long long)N * nx * nx))
      return 0;
  }
  LANE_LOOP(e, nx * nx) F.Pt[(long long)N * nx * nx + e] = s.Pb[e];
  team_sync(c);

  for (int k = N - 1; k >= 0; --k) {
    // stage Jacobian blocks
    const TB* Ag = c.blk + c.L.A + (long long)k * nq * 144;
    const TB* Bg = c.blk + c.L.B + (long long)k * nq * 48;
    LANE_LOOP(e, 144 * nq) s.Ab[e] = (TX)Ag[e];
    LANE_LOOP(e, 48 * nq) s.Bb[e] = (TX)Bg[e];
    team_sync(c);
    // PA = P~ A, PB = P~ B (block-diagonal A, B; column-major blocks).  The
    // first six columns of each A block are constant (p and v enter F
    // affinely): column c < 3 is e_c, column c in 3..5 is e_c + dt e_(c-3),
    // with dt read from the stored block.  They cost a copy or one FMA; the
    // twelve-term products of the other six columns and those of PB share one
    // pass (an FP64 instruction costs the same whatever the active lanes).
    const int n6 = 6 * nq;
    const int nPA = nx * n6, nPB = nx * nu;
    #pragma unroll 1
    for (int e = lane; e < nPA; e += c.T) {
      const int i = e / n6, r6 = e - i * n6, q = r6 / 6, cc = r6 - 6 * q;
      const TX* prow = s.Pb + i * nx + 12 * q;
      s.PA[i * nx + 12 * q + cc] = cc < 3 ? prow[cc] : prow[cc - 3] * s.Ab[q * 144 + cc * 12 + cc - 3] + prow[cc];
    }
    #pragma unroll 1
    for (int e = lane; e < nPA + nPB; e += c.T) {
      const TX* col;
      TX* dst;
      int i, q;
      if (e < nPA) {
        i = e / n6;
        const int r6 = e - i * n6;
        q = r6 / 6;
        const int cc = 6 + r6 - 6 * q;
        col = s.Ab + q * 144 + cc * 12;
        dst = s.PA + i * nx + 12 * q + cc;
      } else {
        const int e2 = e - nPA;
        i = e2 / nu;
        const int cu = e2 - i * nu;
        q = cu >> 2;
        col = s.Bb + q * 48 + (cu & 3) * 12;
        dst = s.PB + e2;
      }
      *dst = dot12(s.Pb + i * nx + 12 * q, 1, col, 1);
    }
    team_sync(c);
    // R^ = R~ + B^T P~ B and S^ = S + B^T (P~ A), in one pass.  S^ and Q^ below
    // are both products with the same PA (entry (i, j) of Q^ from column j of
    // PA): in P_k = Q^ - S^T R^-1 S^ the rounding errors of PA then enter both
    // terms alike and partly cancel, which keeps ill-conditioned stages as
    // accurate as the plain recursion.  (Forming the constant columns of S^
    // from PB, or mirroring Q^ from its upper triangle, is cheaper but breaks
    // this pairing.)
    const int nR = nu * nu;
    #pragma unroll 1
    for (int e = lane; e < nR + nu * nx; e += c.T) {
      int a, colx, sb;
      const TX* v;
      if (e < nR) {
        a = e / nu;
        colx = e - a * nu;
        v = s.PB + (12 * (a >> 2)) * nu + colx;
        sb = nu;
      } else {
        const int e2 = e - nR;
        a = e2 / nx;
        colx = e2 - a * nx;
        v = s.PA + (12 * (a >> 2)) * nx + colx;
        sb = nx;
      }
      const int qa = a >> 2, ca = a & 3;
      TX acc = dot12(s.Bb + qa * 48 + ca * 12, 1, v, sb);
      const TB* H = c.blk + c.L.H + ((long long)k * nq + qa) * 100;
      if (e < nR) {
        const int b = colx;
        if (a == b) {
          if constexpr (pre_diag) {
            acc += udg[k * nu + a];
          } else {
            const int ui = off_u(d, k) + a;
            acc += (TX)(obj_hdiag(c, ui, flags) + (ident ? 0.0 : sigma_of(c, ui) + dw));
          }
        }
        if (!ident && qa == (b >> 2)) acc += (TX)H[(6 + (b & 3)) * 10 + (6 + ca)];
        if constexpr (f32) {
          s.Rh[e] = acc;
          F.LM[(long long)k * nu * nu + e] = acc;
        } else if constexpr (std::is_same<TX, double>::value) {
          s.Rh[e] = acc;
        } else {
          s.R64[e] = (double)acc;
        }
      } else {
        const int qc = colx / 12, cc = colx - 12 * qc;
        if (!ident && qc == qa && cc >= 6) acc += (TX)H[(cc - 6) * 10 + (6 + ca)];
        s.Sh[a * nx + colx] = acc;
      }
    }
    // Q^ = A^T P~ A + Q~_k on the lower triangle only (overwrites Pb; the
    // update of P_k below reads no other entry).  Rows at the constant columns
    // of A are a copy or one FMA of PA, the others twelve-term products.
    #pragma unroll 1
    for (int e = lane; e < tri_rows_count(d, 6); e += c.T) {
      int i, j;
      tri_rows_entry(d, e, 6, i, j);
      const int qi = i / 12;
      const TX q = dot12(s.Ab + qi * 144 + (i - 12 * qi) * 12, 1, s.PA + (12 * qi) * nx + j, nx);
      s.Pb[i * nx + j] = state_term<TB, TF, NQ, TM, TX>(c, k, i, j, dw, flags, xdg, q);
    }
    #pragma unroll 1
    for (int e = lane; e < tri_rows_count(d, 0); e += c.T) {
      int i, j;
      tri_rows_entry(d, e, 0, i, j);
      const int qi = i / 12, ci = i - 12 * qi;
      TX q = s.PA[i * nx + j];
      if (ci >= 3) q += s.PA[(i - 3) * nx + j] * s.Ab[qi * 144 + ci * 12 + ci - 3];
      s.Pb[i * nx + j] = state_term<TB, TF, NQ, TM, TX>(c, k, i, j, dw, flags, xdg, q);
    }
    if constexpr (f32) {
      // FP32 Cholesky of R^ for the gains; the FP64 inertia test follows the
      // recursion.  A pivot FP32 cannot factor ends the recursion here.
      if (!team_cholesky(c, s.Rh, nu)) {
        k_fail32 = k;
        break;
      }
      LANE_LOOP(e, nu * nu) if (e % (nu + 1) == 0) s.Rh[e] = (TX)1 / s.Rh[e];
      team_sync(c);
    } else if constexpr (std::is_same<TX, double>::value) {
      // Cholesky of R^ in FP64 (the inertia test), in place; the diagonal is
      // left as the reciprocals of L_ii, the form every use of it takes
      team_sync(c);
      if (!warp_cholesky_rdiag(c, s.Rh, nu)) return 0;
    } else {
      // Cholesky of R^ in FP64 (the inertia test), then the factor in the
      // factorisation precision with the reciprocal diagonal
      team_sync(c);
      if (!warp_cholesky_rdiag(c, s.R64, nu)) return 0;
      LANE_LOOP(e, nu * nu) s.Rh[e] = (TX)s.R64[e];
      team_sync(c);
    }
    // K = -R^{-1} S^: one column per lane
    #pragma unroll 1
    for (int col = lane; col < nx; col += c.T) {
      TX z[32];
      for (int i = 0; i < nu; ++i) {
        TX acc = s.Sh[i * nx + col];
        for (int t = 0; t < i; ++t) acc -= s.Rh[i * nu + t] * z[t];
        z[i] = acc * s.Rh[i * nu + i];
      }
      for (int i = nu - 1; i >= 0; --i) {
        TX acc = z[i];
        for (int t = i + 1; t < nu; ++t) acc -= s.Rh[t * nu + i] * z[t];
        z[i] = acc * s.Rh[i * nu + i];
      }
      for (int i = 0; i < nu; ++i) s.Kb[i * nx + col] = -z[i];
    }
    team_sync(c);
    // P_k = Q^ + S^T K on the lower triangle, mirrored (exactly symmetric);
    // in place: each thread reads lower entries and writes their mirror images
    {
      const int ntri = nx * (nx + 1) / 2;
      #pragma unroll 1
      for (int e = lane; e < ntri; e += c.T) {
        int i, j;
        tri_index(e, i, j);
        TX a0 = 0, a1 = 0;
        int a = 0;
        for (; a + 1 < nu; a += 2) {
          a0 += s.Sh[a * nx + i] * s.Kb[a * nx + j];
          a1 += s.Sh[(a + 1) * nx + i] * s.Kb[(a + 1) * nx + j];
        }
        if (a < nu) a0 += s.Sh[a * nx + i] * s.Kb[a * nx + j];
        const TX v = s.Pb[i * nx + j] + (a0 + a1);
        s.Pb[i * nx + j] = v;
        s.Pb[j * nx + i] = v;
      }
    }
    TX* Kg = F.K + (long long)k * nu * nx;
    LANE_LOOP(e, nu * nx) Kg[e] = s.Kb[e];
    TX* Lg = F.Lr + (long long)k * nu * nu;
    LANE_LOOP(e, nu * nu) Lg[e] = s.Rh[e];
    team_sync(c);
    if (resto) {
      const double* D = dv + (k == 0 ? 0 : row_dyn(d, k - 1));
      if (!resto_transform<TB, TF, NQ, TM, TX>(c, s.Pb, D, F.LM + (long long)k * nx * nx,
                                       F.Yr + (long long)k * nx * nx))
        return 0;
    }
    LANE_LOOP(e, nx * nx) F.Pt[(long long)k * nx * nx + e] = s.Pb[e];
    team_sync(c);
  }
  if constexpr (f32) {
    // FP64 inertia test of every stage the recursion reached
    team_sync(c);
    const int k0 = k_fail32 >= 0 ? k_fail32 : 0;
    if (!stage_pivot_check(c, F.LM, c.fac64.Lr, k0, N, nu, min_ratio)) return 0;
    if (k_fail32 >= 0 || min_ratio < 1e-5) return 2;
  }
  return 1;
}

// ------------------------------------------------------------------ solve
// Solves K delta = -r for the current factorisation (precision TX), where K
// is the augmented matrix of Eq. 7 (restoration: with the elastic variables)
// and r is K-sized: [r_x (n) | r_p (m) | r_n (m) | r_c (m)] (r_p, r_n only in
// restoration; the layout always reserves them).  out has the same layout.
template <class TB, class TF, int NQ, int TM, class TX>
__device__ __noinline__ void solve(Ctx<TB, TF, NQ, TM>& c, Fac<TX> F, const double* r, double* out, int flags,
                      const double* y) {
  const auto& d = c.d;
  const int lane = c.lane;
  const int nx = d.nx, nu = d.nu, N = d.N, n = d.n, m = d.m;
  const bool resto = flags & FF_RESTO;
  Scratch<TX> s = scratch<TX>(scratch_base<TX>(c), d);
  c.n_solve++;
  if (sizeof(TX) == 4) c.n_solve32++;
  const double* ev = c.f + c.L.ev;
  const double* evr = c.f + c.L.evr;
  const double* rds = c.f + c.L.rds;
  const double* ipv = c.f + c.L.ipv;
  const double* inv = c.f + c.L.inv;
  const double* dv = c.f + c.L.dv;
  const double* x = c.f + c.L.x;
  const long long nwk = c.L.nw;  // offset of r_c inside K-sized vectors
  const double* rx = r;
  const double* rp = r + n;
  const double* rn = r + n + m;
  const double* rc = r + nwk;
  double* ox = out;
  double* op = out + n;
  double* on = out + n + m;
  double* oy = out + nwk;
  // condensed constraint residual r~_c (restoration folds r_p, r_n in)
  double* rct = c.f + c.L.rct;  // condensed constraint residual (m)
  LANE_LOOP(i, m) rct[i] = resto ? rc[i] + rp[i] * ipv[i] - rn[i] * inv[i] : rc[i];
  team_sync(c);
  // inequality rows folded into q~ at the position components, every stage at
  // once: qin_k(a) = sum_r g_r(a) w_r, w_r = E_r (r_s / D_s + r~_g)
  const int np = 3 * d.nq;
  double* wrow = c.f + c.L.wrow;
  double* qin = c.f + c.L.qin;
  const double* igr = c.f + c.L.igr;
  if (d.ni > 0) {
    #pragma unroll 1
    for (int t = lane; t < N * d.ni; t += c.T) {
      const int k = 1 + t / d.ni, rr = t - (k - 1) * d.ni;
      wrow[t] = evr[t] * rx[off_s(d, k) + rr] + ev[t] * rct[row_ineq(d, k) + rr];
    }
    team_sync(c);
    #pragma unroll 1
    for (int e = lane; e < N * np; e += c.T) {
      const int k = 1 + e / np, a = e - (k - 1) * np;
      const int q = a / 3, comp = a - 3 * q;
      double v = 0.0;
      for (int rr = 0; rr < d.ni; ++rr)
        v += grad_pos(ineq_grad_tab(d, igr, (k - 1) * d.ni + rr, rr), q, comp) * wrow[(k - 1) * d.ni + rr];
      qin[e] = v;
    }
    team_sync(c);
  }
  TX* pv = s.v0;  // p_k / p~_k
  TX* tv = s.v1;
  TX* gv = s.v2;  // nu entries (nu <= nx)
  TX* wv = s.v3;
  // q~_k into pv: r_x(x_k) + sum_r g_r E_r (r_s / D_s + r~_g)
  auto qtilde = [&](int k) {
    LANE_LOOP(i, nx) {
      double v = rx[off_x(d, k) + i];
      const int q = i / 12, ci = i - 12 * q;
      if (k >= 1 && ci < 3 && d.ni > 0) v += qin[(k - 1) * np + 3 * q + ci];
      pv[i] = (TX)v;
    }
    team_sync(c);
  };
  // p~ = p - Y^T L^{-1} D^1/2 p (restoration), in place on pv
  auto ptransform = [&](int k, const double* D) {
    const TX* LM = F.LM + (long long)k * nx * nx;
    const TX* Y = F.Yr + (long long)k * nx * nx;
    if (lane == 0) {
      for (int i = 0; i < nx; ++i) {
        double acc = sqrt(D[i]) * (double)pv[i];
        for (int t = 0; t < i; ++t) acc -= (double)LM[i * nx + t] * (double)wv[t];
        wv[i] = (TX)(acc / (double)LM[i * nx + i]);
      }
    }
    team_sync(c);
    LANE_LOOP(i, nx) {
      double acc = 0.0;
      for (int t = 0; t < nx; ++t) acc += (double)Y[t * nx + i] * (double)wv[t];
      tv[i] = (TX)((double)pv[i] - acc);
    }
    team_sync(c);
    LANE_LOOP(i, nx) pv[i] = tv[i];
    team_sync(c);
  };

  // ---- backward sweep
  qtilde(N);
  if (resto) ptransform(N, dv + row_dyn(d, N - 1));
  LANE_LOOP(i, nx) F.ptv[(long long)N * nx + i] = pv[i];
  team_sync(c);
  // stage Jacobian blocks in the factorisation precision (converted once per
  // stage when the blocks are stored in another precision)
  auto stage_blocks = [&](int k, const TX*& Ab, const TX*& Bb) {
    const TB* Ag = c.blk + c.L.A + (long long)k * d.nq * 144;
    const TB* Bg = c.blk + c.L.B + (long long)k * d.nq * 48;
    if constexpr (std::is_same<TB, TX>::value) {
      Ab = Ag;
      Bb = Bg;
    } else {
      LANE_LOOP(e, 144 * d.nq) s.Ab[e] = (TX)Ag[e];
      LANE_LOOP(e, 48 * d.nq) s.Bb[e] = (TX)Bg[e];
      Ab = s.Ab;
      Bb = s.Bb;
    }
  };
  for (int k = N - 1; k >= 0; --k) {
    const TX* Pt = F.Pt + (long long)(k + 1) * nx * nx;
    const TX* Ab;
    const TX* Bb;
    stage_blocks(k, Ab, Bb);
    // d~_k = -r~_c(dyn_k) into wv (free until p_k is formed)
    LANE_LOOP(j, nx) wv[j] = (TX)(-rct[row_dyn(d, k) + j]);
    team_sync(c);
    // t = P~_{k+1} d~_k + p~_{k+1}
    LANE_LOOP(i, nx) {
      TX acc = pv[i];
      for (int j = 0; j < nx; ++j) acc += Pt[i * nx + j] * wv[j];
      tv[i] = acc;
    }
    team_sync(c);
    // A^T t (the first part of p_k, lanes e < nx) and g^ = r_u + B^T t (lanes
    // nx.. nx + nu) in one pass: both are twelve-term products of t, so the
    // two kinds of lane share one instruction stream.  g^ is kept in kff; the
    // feed-forward terms k_k = -R^-1 g^ of all stages are formed after the
    // sweep, one stage per lane.
    const TX* Kg = F.K + (long long)k * nu * nx;
    TX* gk = F.kff + (long long)k * nu;
    LANE_LOOP(e, nx + nu) {
      const TX* col;
      const TX* tq;
      TX acc;
      if (e < nx) {
        const int q = e / 12;
        col = Ab + q * 144 + (e - 12 * q) * 12;
        tq = tv + 12 * q;
        acc = 0;
      } else {
        const int a = e - nx, q = a >> 2;
        col = Bb + q * 48 + (a & 3) * 12;
        tq = tv + 12 * q;
        acc = (TX)rx[off_u(d, k) + a];
      }
      for (int rr = 0; rr < 12; ++rr) acc += col[rr] * tq[rr];
      if (e < nx) {
        wv[e] = acc;
      } else {
        gv[e - nx] = acc;
        gk[e - nx] = acc;
      }
    }
    team_sync(c);
    // p_k = q~_k + A^T t + K^T g^
    LANE_LOOP(i, nx) {
      TX acc = wv[i];
      for (int aa = 0; aa < nu; ++aa) acc += Kg[aa * nx + i] * gv[aa];
      wv[i] = acc;
    }
    team_sync(c);
    qtilde(k);
    LANE_LOOP(i, nx) pv[i] = pv[i] + wv[i];
    team_sync(c);
    if (resto) ptransform(k, dv + (k == 0 ? 0 : row_dyn(d, k - 1)));
    LANE_LOOP(i, nx) F.ptv[(long long)k * nx + i] = pv[i];
    team_sync(c);
  }

  // feed-forward terms k_k = -R^_k^-1 g^_k of every stage, one stage per lane,
  // in place in kff (the stored factor holds 1 / L_ii on its diagonal)
  #pragma unroll 1
  for (int k = lane; k < N; k += c.T) {
    const TX* Lr = F.Lr + (long long)k * nu * nu;
    TX* kf = F.kff + (long long)k * nu;
    TX z[32];
    for (int i = 0; i < nu; ++i) {
      TX acc = kf[i];
      for (int t = 0; t < i; ++t) acc -= Lr[i * nu + t] * z[t];
      z[i] = acc * Lr[i * nu + i];
    }
    for (int i = nu - 1; i >= 0; --i) {
      TX acc = z[i];
      for (int t = i + 1; t < nu; ++t) acc -= Lr[t * nu + i] * z[t];
      z[i] = acc * Lr[i * nu + i];
    }
    for (int i = 0; i < nu; ++i) kf[i] = -z[i];
  }
  team_sync(c);

  // ---- forward sweep; pv = Delta x_k, tv = xi / lambda scratch
  {
    const TX* Pt0 = F.Pt;
    const TX* pt0 = F.ptv;
    // xi_0 = -r~_c(init); lambda_0 = P~_0 xi_0 + p~_0; dx_0 = xi_0 - D lambda_0
    LANE_LOOP(i, nx) wv[i] = (TX)(-rct[i]);
    team_sync(c);
    LANE_LOOP(i, nx) {
      TX acc = pt0[i];
      for (int j = 0; j < nx; ++j) acc += Pt0[i * nx + j] * wv[j];
      tv[i] = acc;
    }
    team_sync(c);
    LANE_LOOP(i, nx) {
      double lam = (double)tv[i];
      double dx0 = (double)wv[i] - (resto ? dv[i] * lam : 0.0);
      pv[i] = (TX)dx0;
      ox[i] = dx0;
      oy[i] = -lam;
    }
    team_sync(c);
  }
  for (int k = 0; k < N; ++k) {
    const TX* Ab;
    const TX* Bb;
    stage_blocks(k, Ab, Bb);
    const TX* Kg = F.K + (long long)k * nu * nx;
    const TX* kf = F.kff + (long long)k * nu;
    // d~_k + A dx_k (the first part of xi, lanes e < nx) and du_k = k_k + K dx_k
    // (lanes nx .. nx + nu) in one pass over one instruction stream
    LANE_LOOP(e, nx + nu) {
      const TX* row;
      const TX* vq;
      int sr, len;
      TX acc;
      if (e < nx) {
        const int q = e / 12;
        row = Ab + q * 144 + (e - 12 * q);
        sr = 12;
        vq = pv + 12 * q;
        len = 12;
        acc = (TX)(-rct[row_dyn(d, k) + e]);
      } else {
        row = Kg + (e - nx) * nx;
        sr = 1;
        vq = pv;
        len = nx;
        acc = kf[e - nx];
      }
      for (int j = 0; j < len; ++j) acc += row[j * sr] * vq[j];
      if (e < nx) {
        wv[e] = acc;
      } else {
        gv[e - nx] = acc;
        ox[off_u(d, k) + e - nx] = (double)acc;
      }
    }
    team_sync(c);
    // xi = A dx + B du + d~
    LANE_LOOP(i, nx) {
      int q = i / 12, ri = i - 12 * q;
      TX acc = wv[i];
      for (int j = 0; j < 4; ++j) acc += Bb[q * 48 + j * 12 + ri] * gv[4 * q + j];
      wv[i] = acc;
    }
    team_sync(c);
    const TX* Pt = F.Pt + (long long)(k + 1) * nx * nx;
    const TX* ptk = F.ptv + (long long)(k + 1) * nx;
    LANE_LOOP(i, nx) {
      TX acc = ptk[i];
      for (int j = 0; j < nx; ++j) acc += Pt[i * nx + j] * wv[j];
      tv[i] = acc;
    }
    team_sync(c);
    LANE_LOOP(i, nx) {
      double lam = (double)tv[i];
      double dxn = (double)wv[i] - (resto ? dv[row_dyn(d, k) + i] * lam : 0.0);
      pv[i] = (TX)dxn;
      ox[off_x(d, k + 1) + i] = dxn;
      oy[row_dyn(d, k) + i] = -lam;
    }
    team_sync(c);
  }
  // inequality multipliers and slacks
  #pragma unroll 1
  for (int t = lane; t < N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, rr = t - (t / d.ni) * d.ni;
    const IneqGrad g = ineq_grad_tab(d, igr, t, rr);
    double gdx = 0.0;
    const double* dxk = ox + off_x(d, k);
    for (int comp = 0; comp < g.ncomp; ++comp) {
      gdx += g.g[comp] * dxk[12 * g.q0 + comp];
      if (g.q1 >= 0) gdx -= g.g[comp] * dxk[12 * g.q1 + comp];
    }
    double rs = rx[off_s(d, k) + rr];
    // E (g dx + r_s / D_s + r~_g) with E / D_s = evr
    double dyi = ev[t] * (gdx + rct[row_ineq(d, k) + rr]) + evr[t] * rs;
    oy[row_ineq(d, k) + rr] = dyi;
    ox[off_s(d, k) + rr] = (dyi - rs) * rds[t];
  }
  if (resto) {
    team_sync(c);
    LANE_LOOP(i, m) {
      op[i] = (oy[i] - rp[i]) * ipv[i];
      on[i] = (-oy[i] - rn[i]) * inv[i];
    }
  }
  team_sync(c);
}

// ---------------------------------------------------- KKT mat-vec (FP64)
// out = K v for the matrix that `factor` condensed (same dw, same phase),
// K-sized layout as in `solve`.  Used for iterative refinement.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void kkt_matvec(Ctx<TB, TF, NQ, TM>& c, const double* v, double* out, double dw,
                           const double* y) {
  const auto& d = c.d;
  const int lane = c.lane;
  const int nx = d.nx, nu = d.nu, N = d.N, n = d.n, m = d.m;
  const long long nwk = c.L.nw;
  const double* igr = c.f + c.L.igr;
  const double* vy = v + nwk;
  double* oy = out + nwk;
  const int flags = c.resto ? FF_RESTO : 0;
  // W-part diagonal terms and dynamics Hessian, and J^T v_y (dynamics)
  LANE_LOOP(i, c.nw) {
    double acc = 0.0;
    int kind = wkind(d, i);
    acc += (obj_hdiag(c, i, flags) + sigma_of(c, i) + dw) * v[i];
    (void)kind;
    out[i] = acc;
  }
  team_sync(c);
  #pragma unroll 1
  for (int t = lane; t < N * d.nq; t += c.T) {
    int k = t / d.nq, q = t - (t / d.nq) * d.nq;
    const TB* A = c.blk + c.L.A + ((long long)k * d.nq + q) * 144;
    const TB* B = c.blk + c.L.B + ((long long)k * d.nq + q) * 48;
    const TB* H = c.blk + c.L.H + ((long long)k * d.nq + q) * 100;
    int ox = off_x(d, k) + 12 * q, ou = off_u(d, k) + 4 * q;
    double vz[10];
    for (int j = 0; j < 6; ++j) vz[j] = v[ox + 6 + j];
    for (int j = 0; j < 4; ++j) vz[6 + j] = v[ou + j];
    const double* yd = vy + row_dyn(d, k) + 12 * q;
    const double* yp = vy + (k == 0 ? 0 : row_dyn(d, k - 1)) + 12 * q;
    for (int r = 0; r < 12; ++r) {
      double acc = yp[r];
      for (int j = 0; j < 12; ++j) acc -= (double)A[r * 12 + j] * yd[j];
      if (r >= 6)
        for (int j = 0; j < 10; ++j) acc += (double)H[j * 10 + (r - 6)] * vz[j];
      out[ox + r] += acc;
    }
    for (int a = 0; a < 4; ++a) {
      double acc = 0.0;
      for (int j = 0; j < 12; ++j) acc -= (double)B[a * 12 + j] * yd[j];
      for (int j = 0; j < 10; ++j) acc += (double)H[j * 10 + 6 + a] * vz[j];
      out[ou + a] += acc;
    }
  }
  team_sync(c);
  LANE_LOOP(i, nx) out[off_x(d, N) + i] += vy[row_dyn(d, N - 1) + i];
  team_sync(c);
  // inequality Hessian and G^T v_y on positions; -v_y on slacks
  #pragma unroll 1
  for (int t = lane; t < N * 3 * d.nq; t += c.T) {
    int k = 1 + t / (3 * d.nq);
    int pc = t - (t / (3 * d.nq)) * (3 * d.nq);
    int q = pc / 3, comp = pc - 3 * (pc / 3);
    int i = 12 * q + comp;
    const double* yi = y + row_ineq(d, k);
    const double* vyi = vy + row_ineq(d, k);
    const double* vx = v + off_x(d, k);
    double acc = 0.0;
    for (int r = 0; r < d.ni; ++r) {
      const IneqGrad g = ineq_grad_tab(d, igr, (k - 1) * d.ni + r, r);
      const double gi = grad_pos(g, q, comp);
      if (gi == 0.0 && q != g.q0 && q != g.q1) continue;
      acc += gi * vyi[r];
      // Hessian 2 I (pairs +-2 I) couples equal components of the row's quads
      double hv = hess_pos(g, q, comp, g.q0, comp) * vx[12 * g.q0 + comp];
      if (g.q1 >= 0) hv += hess_pos(g, q, comp, g.q1, comp) * vx[12 * g.q1 + comp];
      acc += yi[r] * hv;
    }
    out[off_x(d, k) + i] += acc;
  }
  #pragma unroll 1
  for (int t = lane; t < N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, r = t - (t / d.ni) * d.ni;
    out[off_s(d, k) + r] -= vy[row_ineq(d, k) + r];
  }
  if (c.resto) {
    LANE_LOOP(i, m) {
      out[n + i] -= vy[i];
      out[n + m + i] += vy[i];
    }
  }
  team_sync(c);
  // constraint part: J v_w (- v_p + v_n in restoration)
  LANE_LOOP(i, nx) oy[i] = v[i];
  #pragma unroll 1
  for (int t = lane; t < N * d.nq; t += c.T) {
    int k = t / d.nq, q = t - (t / d.nq) * d.nq;
    const TB* A = c.blk + c.L.A + ((long long)k * d.nq + q) * 144;
    const TB* B = c.blk + c.L.B + ((long long)k * d.nq + q) * 48;
    const double* vx = v + off_x(d, k) + 12 * q;
    const double* vu = v + off_u(d, k) + 4 * q;
    const double* vn = v + off_x(d, k + 1) + 12 * q;
    for (int r = 0; r < 12; ++r) {
      double acc = vn[r];
      for (int j = 0; j < 12; ++j) acc -= (double)A[j * 12 + r] * vx[j];
      for (int j = 0; j < 4; ++j) acc -= (double)B[j * 12 + r] * vu[j];
      oy[row_dyn(d, k) + 12 * q + r] = acc;
    }
  }
  #pragma unroll 1
  for (int t = lane; t < N * d.ni; t += c.T) {
    int k = 1 + t / d.ni, r = t - (t / d.ni) * d.ni;
    const IneqGrad g = ineq_grad_tab(d, igr, t, r);
    const double* vx = v + off_x(d, k);
    double acc = -v[off_s(d, k) + r];
    for (int comp = 0; comp < g.ncomp; ++comp) {
      acc += g.g[comp] * vx[12 * g.q0 + comp];
      if (g.q1 >= 0) acc -= g.g[comp] * vx[12 * g.q1 + comp];
    }
    oy[row_ineq(d, k) + r] = acc;
  }
  team_sync(c);
  if (c.resto) {
    LANE_LOOP(i, m) oy[i] += -v[n + i] + v[n + m + i];
  }
  team_sync(c);
  (void)nu;
}

}  // namespace bipm
