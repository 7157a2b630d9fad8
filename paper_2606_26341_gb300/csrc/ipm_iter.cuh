// The interior-point iteration of one problem (one warp): convergence test,
// monotone barrier update, inertia-corrected factorisation, Newton step with
// optional FP64 iterative refinement, fraction-to-boundary rule, tiny-step
// rule, backtracking filter line search with second-order correction, and the
// entry to and return from the l1 feasibility-restoration phase.
//
// The branch structure follows the paper's Table I and the IPOPT algorithm it
// reviews (Sec. IV); restoration is a per-problem mode in which the same code
// works on the restoration problem (variables x, p, n).
#pragma once

#include <type_traits>

#include "ipm_device.cuh"

namespace bipm {

enum Outcome : int { OUT_ACCEPTED = 0, OUT_LS_FAILED = 1 };

// ------------------------------------------------------------- reductions
template <class TB, class TF, int NQ, int TM>
__device__ double l1_norm(Ctx<TB, TF, NQ, TM>& c, const double* v, int len) {
  double a = 0.0;
  #pragma unroll 1
  for (int i = c.lane; i < len; i += c.T) a += fabs(v[i]);
  return team_sum(c, a);
}
template <class TB, class TF, int NQ, int TM>
__device__ double inf_norm(Ctx<TB, TF, NQ, TM>& c, const double* v, int len) {
  double a = 0.0;
  #pragma unroll 1
  for (int i = c.lane; i < len; i += c.T) a = fmax(a, fabs(v[i]));
  return team_max(c, a);
}
template <class TB, class TF, int NQ, int TM>
__device__ bool all_finite(Ctx<TB, TF, NQ, TM>& c, const double* v, int len) {
  int bad = 0;
  #pragma unroll 1
  for (int i = c.lane; i < len; i += c.T) bad |= !isfinite(v[i]);
  return !team_or(c, bad);
}

// barrier objective phi_mu (Eq. 3) with the one-sided damping term, over the
// first `len` entries of a W-sized point w; +inf outside the bounds
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double barrier_phi(Ctx<TB, TF, NQ, TM>& c, const double* w, double f, double mu, int len) {
  double acc = 0.0;
  int bad = 0;
  const int nb = n_bounded(c.d, len);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(c.d, b, kind);
    double sl = w[i];
    if (!(sl > 0.0)) bad = 1;
    acc -= mu * log(sl);
    if (kind == VK_BOX) {
      double su = kUmax - w[i];
      if (!(su > 0.0)) bad = 1;
      acc -= mu * log(su);
    } else {
      acc += kKappaD * mu * sl;
    }
  }
  if (team_or(c, bad)) return INFINITY;
  return f + team_sum(c, acc);
}

// scaled optimality error E_mu of Eq. 5 (IPOPT's scaling)
struct ErrParts {
  double dual, prim, y1, z1, nb;
};

template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ ErrParts err_parts(Ctx<TB, TF, NQ, TM>& c) {
  const double* gf = c.f + c.L.gf;
  const double* jty = c.f + c.L.jty;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  const double* y = c.f + c.L.y;
  const double* cv = c.f + c.L.c;
  double du = 0.0, z1 = 0.0, nb = 0.0;
  #pragma unroll 1
  for (int i = c.lane; i < c.nw; i += c.T) {
    int kind = wkind(c.d, i);
    double zli = has_lower(kind) ? zl[i] : 0.0;
    double zui = has_upper(kind) ? zu[i] : 0.0;
    du = fmax(du, fabs(gf[i] + jty[i] - zli + zui));
    z1 += fabs(zli) + fabs(zui);
    nb += (has_lower(kind) ? 1.0 : 0.0) + (has_upper(kind) ? 1.0 : 0.0);
  }
  double pr = 0.0, y1 = 0.0;
  #pragma unroll 1
  for (int i = c.lane; i < c.d.m; i += c.T) {
    pr = fmax(pr, fabs(cv[i]));
    y1 += fabs(y[i]);
  }
  ErrParts e;
  e.dual = team_max(c, du);
  e.prim = team_max(c, pr);
  e.y1 = team_sum(c, y1);
  e.z1 = team_sum(c, z1);
  e.nb = team_sum(c, nb);
  return e;
}

template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double opt_error(Ctx<TB, TF, NQ, TM>& c, const ErrParts& e, double mu) {
  const double* w = c.f + c.L.x;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  double comp = 0.0;
  const int nbnd = n_bounded(c.d, c.nw);
  #pragma unroll 1
  for (int b = c.lane; b < nbnd; b += c.T) {
    int kind;
    const int i = bnd_index(c.d, b, kind);
    comp = fmax(comp, fabs(w[i] * zl[i] - mu));
    if (kind == VK_BOX) comp = fmax(comp, fabs((kUmax - w[i]) * zu[i] - mu));
  }
  comp = team_max(c, comp);
  double nb = fmax(1.0, e.nb);
  double s_d = fmax(kSmax, (e.y1 + e.z1) / fmax(1.0, c.d.m + e.nb)) / kSmax;
  double s_c = fmax(kSmax, e.z1 / nb) / kSmax;
  return fmax(fmax(e.dual / s_d, e.prim), comp / s_c);
}

// largest alpha in (0, 1] keeping the bounded entries of w + alpha dw at least
// the fraction 1 - tau of their distance to the bounds
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double ftb_primal(Ctx<TB, TF, NQ, TM>& c, const double* w, const double* dw, double tau) {
  double a = 1.0;
  const int nb = n_bounded(c.d, c.nw);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(c.d, b, kind);
    if (dw[i] < 0.0) a = fmin(a, -tau * w[i] / dw[i]);
    if (kind == VK_BOX && dw[i] > 0.0) a = fmin(a, tau * (kUmax - w[i]) / dw[i]);
  }
  return team_min(c, a);
}

// bound-multiplier steps (text after Eq. 6) for the primal step dx at the
// current point
__device__ __forceinline__ double dz_lower(double sl, double zl, double mu, double dx) {
  return mu / sl - zl - zl / sl * dx;
}
__device__ __forceinline__ double dz_upper(double su, double zu, double mu, double dx) {
  return mu / su - zu + zu / su * dx;
}

// ---------------------------------------------------------------- filter
template <class C>
__device__ __forceinline__ bool in_filter(const C& c, const double* filt, int nf, double theta,
                                          double phi, double theta_max) {
  if (!(theta < theta_max)) return true;
  int hit = 0;
  #pragma unroll 1
  for (int j = c.lane; j < nf; j += c.T) hit |= (theta >= filt[2 * j] && phi >= filt[2 * j + 1]);
  return team_or(c, hit);
}

template <class C>
__device__ __forceinline__ void filter_add(const C& c, double* filt, int& nf, double theta,
                                           double phi) {
  int cnt = nf;
  if (c.lane == 0) {
    int w = 0;
    for (int j = 0; j < cnt; ++j) {
      double t = filt[2 * j], p = filt[2 * j + 1];
      if (!(t >= theta && p >= phi)) {
        filt[2 * w] = t;
        filt[2 * w + 1] = p;
        ++w;
      }
    }
    filt[2 * w] = theta;
    filt[2 * w + 1] = phi;
    ++w;
    if (w > kFilterCap) {
      for (int j = 1; j < w; ++j) {
        filt[2 * (j - 1)] = filt[2 * j];
        filt[2 * (j - 1) + 1] = filt[2 * j + 1];
      }
      --w;
    }
    cnt = w;
  }
  team_sync(c);
  nf = team_bcast0(c, cnt);
}

// -------------------------------------------------- factorisation and solve
// Largest barrier diagonal of the condensed system: Sigma of the inputs and
// the condensation weight E of the slacks.  Relative to the O(1) Hessian
// blocks it measures how much of FP32's 24-bit mantissa the factorisation
// loses in the position and input blocks.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double barrier_scale(Ctx<TB, TF, NQ, TM>& c) {
  const auto& d = c.d;
  const double* ev = c.f + c.L.ev;
  const double* sg = c.f + c.L.sig;
  double b = 0.0;
  #pragma unroll 1
  for (int t = c.lane; t < d.N * d.ni; t += c.T) b = fmax(b, ev[t]);
  #pragma unroll 1
  for (int t = c.lane; t < d.N * d.nu; t += c.T) {
    int k = t / d.nu, a = t - (t / d.nu) * d.nu;
    b = fmax(b, sg[off_u(d, k) + a]);
  }
  return team_max(c, b);
}

template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ bool factor_any(Ctx<TB, TF, NQ, TM>& c, double dw, bool force64) {
  const int flags = c.resto ? FF_RESTO : 0;
  const double* y = c.f + c.L.y;
  if (HighPrecision<TF>::value && !std::is_same<TF, double>::value && !c.resto && !force64) {
    // double-float factorisation: accurate enough to need no refinement
    c.use64 = 0;
    return factor<TB, TF, NQ, TM, TF>(c, c.fac, dw, flags, y) != 0;
  }
  if (sizeof(TF) == 4 && !c.resto && !force64) {
    // per-problem precision choice: FP32 only while the barrier terms leave
    // the refinement a well-conditioned preconditioned system
    compute_diag(c, dw, flags);
    if (c.P->opt.fp32_switch < 0.0 || barrier_scale(c) > c.P->opt.fp32_switch) {
      force64 = true;
      c.n_esc++;
    }
  }
  if (HighPrecision<TF>::value || c.resto || force64) {
    c.use64 = 1;
    return factor<TB, TF, NQ, TM, double>(c, c.fac64, dw, flags, y) != 0;
  }
  int r = factor<TB, TF, NQ, TM, TF>(c, c.fac, dw, flags, y);
  if (r == 0) return false;
  if (r == 2) {
    c.n_esc++;
    c.use64 = 1;
    return factor<TB, TF, NQ, TM, double>(c, c.fac64, dw, flags, y) != 0;
  }
  c.use64 = 0;
  return true;
}

// Solves K out = -r.  With an FP32 factorisation the step is refined in FP64
// by restarted GMRES on K, right-preconditioned with the FP32 factors (the
// GMRES form of iterative refinement): residuals and Krylov vectors are FP64,
// each preconditioner application is one FP32 solve.  It stops when IPOPT's
// residual ratio |K out + r| / (min(|out|, 1e6 |r|) + |r|) drops below 1e-10;
// if that fails within the restarts the matrix is refactorised in FP64.
// Returns false only if that FP64 refactorisation reports wrong inertia.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ bool solve_refined(Ctx<TB, TF, NQ, TM>& c, const double* r, double* out) {
  const int flags = c.resto ? FF_RESTO : 0;
  const double* y = c.f + c.L.y;
  if (c.use64) {
    solve<TB, TF, NQ, TM, double>(c, c.fac64, r, out, flags, y);
    return true;
  }
  if (HighPrecision<TF>::value) {  // double-float factors: no refinement needed
    solve<TB, TF, NQ, TM, TF>(c, c.fac, r, out, flags, y);
    return true;
  }
  const int lane = c.lane;
  const int nwk = (int)c.L.nw;
  const int nused = c.nw;
  const int len = nused + c.d.m;
  const long long nk = c.L.nk;
  double* res = c.f + c.L.res;
  double* corr = c.f + c.L.corr;
  double* V = c.f + c.L.gmv;
  auto at = [&](int i) { return i < nused ? i : nwk + (i - nused); };
  auto norm2 = [&](const double* v) {
    double a = 0.0;
    #pragma unroll 1
    for (int i = lane; i < len; i += c.T) {
      double t = v[at(i)];
      a += t * t;
    }
    return sqrt(team_sum(c, a));
  };
  auto norm_inf = [&](const double* v) {
    double a = 0.0;
    #pragma unroll 1
    for (int i = lane; i < len; i += c.T) a = fmax(a, fabs(v[at(i)]));
    return team_max(c, a);
  };
  // preconditioner: z = M^{-1} v  (solve(r') returns K z = -r', so r' = -v)
  auto precond = [&](const double* v, double* z) {
    #pragma unroll 1
    for (int i = lane; i < len; i += c.T) corr[at(i)] = -v[at(i)];
    team_sync(c);
    solve<TB, TF, NQ, TM, TF>(c, c.fac, corr, z, flags, y);
  };
  solve<TB, TF, NQ, TM, TF>(c, c.fac, r, out, flags, y);
  const double rnorm = norm_inf(r);
  if (rnorm == 0.0) return true;
  for (int rs = 0; rs <= kGmresRestarts; ++rs) {
    // residual of K out = -r
    kkt_matvec(c, out, res, c.dw, y);
    #pragma unroll 1
    for (int i = lane; i < len; i += c.T) res[at(i)] = -r[at(i)] - res[at(i)];
    team_sync(c);
    double ratio = norm_inf(res) / (fmin(norm_inf(out), 1e6 * rnorm) + rnorm);
    if (ratio <= kIrTol) return true;
    if (rs == kGmresRestarts) break;
    double beta = norm2(res);
    double H[kGmresM + 1][kGmresM], cs[kGmresM], sn[kGmresM], g[kGmresM + 1];
    const double ibeta = 1.0 / beta;
    #pragma unroll 1
    for (int i = lane; i < len; i += c.T) V[at(i)] = res[at(i)] * ibeta;
    g[0] = beta;
    team_sync(c);
    int jm = 0;
    for (int j = 0; j < kGmresM; ++j) {
      double* vj = V + (long long)j * nk;
      double* vn = V + (long long)(j + 1) * nk;
      precond(vj, res);           // res <- M^{-1} v_j
      kkt_matvec(c, res, vn, c.dw, y);  // v_{j+1} <- K M^{-1} v_j
      c.n_ir++;
      for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt
        const double* vi = V + (long long)i * nk;
        double h = 0.0;
        #pragma unroll 1
        for (int t = lane; t < len; t += c.T) h += vn[at(t)] * vi[at(t)];
        h = team_sum(c, h);
        #pragma unroll 1
        for (int t = lane; t < len; t += c.T) vn[at(t)] -= h * vi[at(t)];
        team_sync(c);
        H[i][j] = h;
      }
      double hn = norm2(vn);
      H[j + 1][j] = hn;
      if (hn > 0.0) {
        const double ihn = 1.0 / hn;
        #pragma unroll 1
        for (int t = lane; t < len; t += c.T) vn[at(t)] *= ihn;
        team_sync(c);
      }
      for (int i = 0; i < j; ++i) {  // previous Givens rotations
        double a = H[i][j], b = H[i + 1][j];
        H[i][j] = cs[i] * a + sn[i] * b;
        H[i + 1][j] = -sn[i] * a + cs[i] * b;
      }
      double a = H[j][j], b = H[j + 1][j];
      double rr = hypot(a, b);
      cs[j] = rr > 0.0 ? a / rr : 1.0;
      sn[j] = rr > 0.0 ? b / rr : 0.0;
      H[j][j] = rr;
      H[j + 1][j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      jm = j + 1;
      if (fabs(g[j + 1]) <= 1e-12 * beta || hn == 0.0) break;
    }
    // y = H^{-1} g, out += M^{-1} (V y)
    double yv[kGmresM];
    for (int i = jm - 1; i >= 0; --i) {
      double acc = g[i];
      for (int t = i + 1; t < jm; ++t) acc -= H[i][t] * yv[t];
      yv[i] = H[i][i] != 0.0 ? acc / H[i][i] : 0.0;
    }
    #pragma unroll 1
    for (int t = lane; t < len; t += c.T) {
      double acc = 0.0;
      for (int i = 0; i < jm; ++i) acc += yv[i] * V[(long long)i * nk + at(t)];
      res[at(t)] = acc;
    }
    team_sync(c);
    precond(res, res);
    #pragma unroll 1
    for (int t = lane; t < len; t += c.T) out[at(t)] += res[at(t)];
    team_sync(c);
  }
  // refinement did not converge: refactorise in FP64
  c.n_esc++;
  if (factor<TB, TF, NQ, TM, double>(c, c.fac64, c.dw, flags, y) == 0) return false;
  c.use64 = 1;
  solve<TB, TF, NQ, TM, double>(c, c.fac64, r, out, flags, y);
  // an FP64 step that is not finite cannot be used: the problem stops
  if (!all_finite(c, out, nused) || !all_finite(c, out + nwk, c.d.m)) c.esc_failed = 1;
  return true;
}

// Least-squares multipliers: [[I, J^T], [J, 0]] (w, y) = (-(grad f - z_L + z_U), 0);
// y = 0 if |y|_inf > y_max.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void ls_multipliers(Ctx<TB, TF, NQ, TM>& c) {
  const auto& d = c.d;
  const int lane = c.lane;
  double* w = c.f + c.L.x;
  double* y = c.f + c.L.y;
  const double* gf = c.f + c.L.gf;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  double* rhs = c.f + c.L.rhs;
  double* sol = c.f + c.L.sol;
  eval_blocks(c, w, y, false);
  LANE_LOOP(i, d.n) {
    int kind = var_kind(d, i);
    rhs[i] = gf[i] - (has_lower(kind) ? zl[i] : 0.0) + (has_upper(kind) ? zu[i] : 0.0);
  }
  LANE_LOOP(i, d.m) rhs[c.L.nw + i] = 0.0;
  team_sync(c);
  factor<TB, TF, NQ, TM, double>(c, c.fac64, 0.0, FF_IDENT, y);
  solve<TB, TF, NQ, TM, double>(c, c.fac64, rhs, sol, FF_IDENT, y);
  double ymax = inf_norm(c, sol + c.L.nw, d.m);
  LANE_LOOP(i, d.m) y[i] = ymax > kYmax ? 0.0 : sol[c.L.nw + i];
  team_sync(c);
}

// z <- max(min(z, kappa_Sigma mu / s), mu / (kappa_Sigma s)) over the first len entries
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void kappa_sigma_reset(Ctx<TB, TF, NQ, TM>& c, int len, double mu) {
  double* w = c.f + c.L.x;
  double* zl = c.f + c.L.zl;
  double* zu = c.f + c.L.zu;
  const int nb = n_bounded(c.d, len);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(c.d, b, kind);
    double s = w[i];
    zl[i] = fmax(fmin(zl[i], kKappaSigma * mu / s), mu / (kKappaSigma * s));
    if (kind == VK_BOX) {
      s = kUmax - w[i];
      zu[i] = fmax(fmin(zu[i], kKappaSigma * mu / s), mu / (kKappaSigma * s));
    }
  }
  team_sync(c);
}

// A barrier-parameter decrease or entering restoration ends an active
// watchdog and soft restoration and clears the shortened-step count.
__device__ __forceinline__ void end_globalization(SlotState& S) {
  S.wd_active = 0;
  S.wd_trials = 0;
  S.wd_short = 0;
  S.soft_active = 0;
  S.soft_iters = 0;
}

// Average and minimum of the complementarity products s_i z_i over all bounds
// of the original problem.
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void complementarity_stats(Ctx<TB, TF, NQ, TM>& c, double& avg, double& mn) {
  const auto& d = c.d;
  const double* w = c.f + c.L.x;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  double sum = 0.0, lo = INFINITY, cnt = 0.0;
  const int nb = n_bounded(d, d.n);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(d, b, kind);
    const double pl = w[i] * zl[i];
    sum += pl;
    lo = fmin(lo, pl);
    cnt += 1.0;
    if (kind == VK_BOX) {
      const double pu = (kUmax - w[i]) * zu[i];
      sum += pu;
      lo = fmin(lo, pu);
      cnt += 1.0;
    }
  }
  sum = team_sum(c, sum);
  cnt = team_sum(c, cnt);
  mn = team_min(c, lo);
  avg = cnt > 0.0 ? sum / cnt : 0.0;
  if (!(cnt > 0.0)) mn = 0.0;
}

// LOQO's centrality rule: sigma * average with sigma = 0.1 min(0.05 (1 - xi)/xi, 2)^3,
// xi = min / average
__device__ __forceinline__ double loqo_mu(double avg, double mn) {
  if (!(avg > 0.0)) return 0.0;
  const double xi = mn / avg;
  const double t = xi > 0.0 ? fmin(0.05 * (1.0 - xi) / xi, 2.0) : 2.0;
  return 0.1 * t * t * t * avg;
}

// 1-norm primal-dual error of the barrier problem at mu (original problem):
// |grad f + J^T y - z_L + z_U|_1 + |c|_1 + |S_L z_L - mu e|_1 + |S_U z_U - mu e|_1
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ double pd_error(Ctx<TB, TF, NQ, TM>& c, const double* w, const double* zl, const double* zu,
                                        const double* gf, const double* jty, const double* cv, double mu) {
  const auto& d = c.d;
  double a = 0.0;
  #pragma unroll 1
  for (int i = c.lane; i < d.n; i += c.T) {
    const int kind = wkind(d, i);
    a += fabs(gf[i] + jty[i] - (has_lower(kind) ? zl[i] : 0.0) + (has_upper(kind) ? zu[i] : 0.0));
  }
  #pragma unroll 1
  for (int i = c.lane; i < d.m; i += c.T) a += fabs(cv[i]);
  const int nb = n_bounded(d, d.n);
  #pragma unroll 1
  for (int b = c.lane; b < nb; b += c.T) {
    int kind;
    const int i = bnd_index(d, b, kind);
    a += fabs(w[i] * zl[i] - mu);
    if (kind == VK_BOX) a += fabs((kUmax - w[i]) * zu[i] - mu);
  }
  return team_sum(c, a);
}

// ------------------------------------------------------------- iteration
struct TrialVal {
  double theta, phi, f;
  bool finite;
};

// trial point w + alpha * dir: constraint violation and barrier objective of
// the current phase; the phase constraint vector goes to ct
template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ TrialVal trial_point(Ctx<TB, TF, NQ, TM>& c, double alpha, const double* dir) {
  const auto& d = c.d;
  const int lane = c.lane;
  const double* w = c.f + c.L.x;
  double* xt = c.f + c.L.xt;
  double* ct = c.f + c.L.ct;
  LANE_LOOP(i, c.nw) xt[i] = w[i] + alpha * dir[i];
  team_sync(c);
  c.n_trial++;
  double f = eval_values(c, xt, ct);
  if (c.resto) {
    LANE_LOOP(i, d.m) ct[i] += -xt[d.n + i] + xt[d.n + d.m + i];
    team_sync(c);
    f = resto_objective(c, xt);
  }
  TrialVal tv;
  tv.finite = isfinite(f) && all_finite(c, ct, d.m);
  tv.theta = l1_norm(c, ct, d.m);
  tv.phi = tv.finite ? barrier_phi(c, xt, f, c.mu, c.nw) : INFINITY;
  tv.f = f;
  return tv;
}

template <class TB, class TF, int NQ, int TM>
__device__ __noinline__ void iterate(Ctx<TB, TF, NQ, TM>& c, SlotState& S) {
  const auto& d = c.d;
  const int lane = c.lane;
  const Options& opt = c.P->opt;
  const int n = d.n, m = d.m;
  const int nwk = (int)c.L.nw;
  double* w = c.f + c.L.x;
  double* zl = c.f + c.L.zl;
  double* zu = c.f + c.L.zu;
  double* y = c.f + c.L.y;
  double* cv = c.f + c.L.c;
  double* ct = c.f + c.L.ct;
  double* csoc = c.f + c.L.csoc;
  double* gf = c.f + c.L.gf;
  double* jty = c.f + c.L.jty;
  double* gphi = c.f + c.L.gphi;
  double* rhs = c.f + c.L.rhs;
  double* sol = c.f + c.L.sol;
  double* rhs2 = c.f + c.L.rhs2;
  double* sol2 = c.f + c.L.sol2;
  double* xr = c.f + c.L.xr;

  c.resto = S.mode == MODE_RESTO;
  c.nw = c.resto ? n + 2 * m : n;
  c.zeta = S.zeta;
  c.n_ir = 0;
  c.n_esc = 0;
  c.n_fact = 0;
  c.n_solve = 0;
  c.n_trial = 0;
  c.n_fact32 = 0;
  c.n_solve32 = 0;
  double& mu = c.resto ? S.mu_r : S.mu;
  double& dw_last = c.resto ? S.dw_last_r : S.dw_last;
  double& th_max = c.resto ? S.theta_max_r : S.theta_max;
  double& th_min = c.resto ? S.theta_min_r : S.theta_min;
  int& tiny = c.resto ? S.tiny_r : S.tiny;
  int& nf = c.resto ? S.n_filt_r : S.n_filt;
  double* filt = c.f + (c.resto ? c.L.filt_r : c.L.filt);

  const long long t_start = clock64();
  long long t_mark = t_start;
  auto lap = [&](int ph) {
    long long now = clock64();
    S.cyc[ph] += now - t_mark;
    t_mark = now;
  };
  // ---- evaluation at the current point: c(x), f(x) and J^T y in one sweep
  double f_orig = eval_values(c, w, cv, false);
  eval_jty(c, w, y, jty, cv);
  double fph = f_orig;
  if (c.resto) {
    LANE_LOOP(i, m) cv[i] += -w[n + i] + w[n + m + i];
    team_sync(c);
    fph = resto_objective(c, w);
  }
  eval_grad(c, w, gf);
  if (d.ni > 0) fill_ineq_grad(c, w);
  lap(PH_EVAL);
  if (!(isfinite(fph) && all_finite(c, cv, m) && all_finite(c, gf, c.nw))) {
    S.status = BIPM_EVAL_ERROR;
    return;
  }
  if (S.iter >= opt.max_iter) {
    if (!c.resto) {
      if (S.need_y_ls) ls_multipliers(c);
      eval_jty(c, w, y, jty);
      ErrParts e = err_parts(c);
      S.status = opt_error(c, e, 0.0) <= opt.tol ? BIPM_CONVERGED : BIPM_MAX_ITER;
      S.need_y_ls = 0;
    } else {
      S.status = BIPM_MAX_ITER;
    }
    return;
  }
  if (!c.resto && S.need_y_ls) {
    ls_multipliers(c);
    eval_jty(c, w, y, jty);
    lap(PH_LSQ);
  }
  double theta = l1_norm(c, cv, m);
  if (!c.resto && S.need_init) {
    th_max = 1e4 * fmax(1.0, theta);
    th_min = 1e-4 * fmax(1.0, theta);
  }
  if (!c.resto) {
    S.need_init = 0;
    S.need_y_ls = 0;
  }

  // ---- overall convergence (Eq. 5 with mu = 0)
  ErrParts ep = err_parts(c);
  if (opt_error(c, ep, 0.0) <= opt.tol) {
    S.status = c.resto ? BIPM_RESTO_FAILED : BIPM_CONVERGED;
    return;
  }

  // ---- barrier update (Table I row 7): adaptive on the original problem, if chosen
  bool mu_done = false;
  if (!c.resto && opt.mu_strategy == 1) {
    const double err0 = opt_error(c, ep, 0.0);
    double avg, mn;
    complementarity_stats(c, avg, mn);
    if (S.mu_max == 0.0) S.mu_max = kMuMaxFact * fmax(avg, opt.tol);
    double mu_new = mu;
    bool progress = S.n_refs == 0;
    {
      double rmax = 0.0;
      for (int i = 0; i < S.n_refs; ++i) rmax = fmax(rmax, S.mu_refs[i]);
      if (S.n_refs > 0) progress = err0 <= kRefsRedFact * rmax;
    }
    if (S.mu_free) {
      mu_done = true;
      if (progress && !tiny) {
        if (S.n_refs == kNumRefs) {
          for (int i = 1; i < kNumRefs; ++i) S.mu_refs[i - 1] = S.mu_refs[i];
          S.n_refs--;
        }
        S.mu_refs[S.n_refs++] = err0;
        mu_new = fmax(kMuMinFree, fmin(S.mu_max, loqo_mu(avg, mn)));
      } else {
        S.mu_free = 0;
        mu_new = fmax(opt.tol / 10.0, kMuMonoInit * avg);
      }
    } else if (opt_error(c, ep, mu) <= kKappaEps * mu && progress) {
      mu_done = true;
      S.mu_free = 1;
      S.mu_refs[0] = err0;
      S.n_refs = 1;
      mu_new = fmax(kMuMinFree, fmin(S.mu_max, loqo_mu(avg, mn)));
    }
    if (mu_done && mu_new != mu) {
      mu = mu_new;
      nf = 0;
      tiny = 0;
      end_globalization(S);
    }
  }
  // ---- monotone barrier update (Table I row 7)
  if (!mu_done) {
    const double mu_floor = opt.tol / 10.0;
    bool first = true;
    while (true) {
      double e_mu = opt_error(c, ep, mu);
      if ((e_mu <= kKappaEps * mu) || (first && tiny)) {
        if (mu <= mu_floor) {
          if (first && tiny) {
            S.status = c.resto ? BIPM_RESTO_FAILED : BIPM_TINY_STEP;
            return;
          }
          break;
        }
        mu = fmax(mu_floor, fmin(kKappaMu * mu, pow(mu, kThetaMu)));
        nf = 0;
        first = false;
        tiny = 0;
        if (!c.resto) end_globalization(S);
        continue;
      }
      break;
    }
  }
  c.mu = mu;
  const double tau = fmax(kTauMin, 1.0 - mu);

  // ---- derivatives and the right-hand side of Eq. 7
  lap(PH_MISC);
  eval_blocks(c, w, y, true);
  lap(PH_DERIV);
  LANE_LOOP(i, c.nw) gphi[i] = gf[i];
  team_sync(c);
  {
    const int nb = n_bounded(d, c.nw);
    #pragma unroll 1
    for (int b = lane; b < nb; b += c.T) {
      int kind;
      const int i = bnd_index(d, b, kind);
      double g = gf[i] - mu / w[i];
      if (kind == VK_BOX)
        g += mu / (kUmax - w[i]);
      else
        g += kKappaD * mu;
      gphi[i] = g;
    }
  }
  team_sync(c);
  LANE_LOOP(i, c.nw) {
    double g = gphi[i] + jty[i];
    rhs[i] = g;
    rhs2[i] = g;
  }
  LANE_LOOP(i, m) rhs[nwk + i] = cv[i];
  team_sync(c);

  // ---- inertia correction (IPOPT Algorithm IC) and the Newton step
  fill_sigma(c);
  lap(PH_MISC);
  bool force64 = false;
  double dwc = 0.0;
  bool ls_fail = false;
  while (true) {
    dwc = 0.0;
    c.dw = 0.0;
    bool ok = factor_any(c, 0.0, force64);
    if (!ok) {
      dwc = dw_last == 0.0 ? kDwInit : fmax(kDwMin, kKwMinus * dw_last);
      while (true) {
        S.n_inertia_corr++;
        c.dw = dwc;
        ok = factor_any(c, dwc, force64);
        if (ok) break;
        dwc *= dw_last == 0.0 ? kKwPlusBar : kKwPlus;
        if (dwc > kDwMax) break;
      }
      if (!ok) {
        ls_fail = true;
        break;
      }
      dw_last = dwc;
    }
    c.dw = dwc;
    lap(PH_FACTOR);
    c.esc_failed = 0;
    bool solved = solve_refined(c, rhs, sol);
    lap(PH_SOLVE);
    if (solved && c.esc_failed) {
      // no accurate Newton step even in FP64: the problem stops here
      S.n_ir_steps += c.n_ir;
      S.n_escalations += c.n_esc;
      S.n_fact += c.n_fact;
      S.n_solve += c.n_solve;
      S.n_fact32 += c.n_fact32;
      S.n_solve32 += c.n_solve32;
      S.cyc[PH_TOTAL] += clock64() - t_start;
      S.status = BIPM_FP64_ESCALATION_FAILED;
      return;
    }
    if (solved) break;
    // FP64 refactorisation after failed refinement reported wrong inertia:
    // redo the correction in FP64
    if (force64) {
      ls_fail = true;
      break;
    }
    force64 = true;
  }

  Outcome outcome = OUT_LS_FAILED;
  double theta0 = theta, phi0 = 0.0, gdx = 0.0;
  bool wd_restored = false;  // the watchdog returned the iterate to its stored point
  if (!ls_fail) {
    const double* dx = sol;
    double a_max = ftb_primal(c, w, dx, tau);

    // accept a step (alpha, dir) with dir K-sized; the z step follows from dir
    // fraction-to-boundary step of the bound multipliers along the z step of dir
    auto dual_max = [&](const double* ddx) {
      double az = 1.0;
      const int nb = n_bounded(d, c.nw);
      #pragma unroll 1
      for (int b = lane; b < nb; b += c.T) {
        int kind;
        const int i = bnd_index(d, b, kind);
        double dzl = dz_lower(w[i], zl[i], mu, ddx[i]);
        if (dzl < 0.0) az = fmin(az, -tau * zl[i] / dzl);
        if (kind == VK_BOX) {
          double dzu = dz_upper(kUmax - w[i], zu[i], mu, ddx[i]);
          if (dzu < 0.0) az = fmin(az, -tau * zu[i] / dzu);
        }
      }
      return team_min(c, az);
    };
    // accept a step (alpha, dir) with dir K-sized; the z step follows from dir
    // (az_fixed >= 0: that dual step size instead of its fraction to the boundary)
    auto accept = [&](double alpha, const double* dir, bool augment, double az_fixed = -1.0) {
      const double* ddx = dir;
      const double* ddy = dir + nwk;
      const double az = az_fixed >= 0.0 ? az_fixed : dual_max(ddx);
      const int nb = n_bounded(d, c.nw);
      // bound multipliers from the step at the current point, then the primal step
      #pragma unroll 1
      for (int b = lane; b < nb; b += c.T) {
        int kind;
        const int i = bnd_index(d, b, kind);
        zl[i] += az * dz_lower(w[i], zl[i], mu, ddx[i]);
        if (kind == VK_BOX) zu[i] += az * dz_upper(kUmax - w[i], zu[i], mu, ddx[i]);
      }
      team_sync(c);
      LANE_LOOP(i, c.nw) w[i] += alpha * ddx[i];
      LANE_LOOP(i, m) y[i] += alpha * ddy[i];
      team_sync(c);
      kappa_sigma_reset(c, c.nw, mu);
      if (augment) filter_add(c, filt, nf, (1.0 - kGammaTheta) * theta0, phi0 - kGammaPhi * theta0);
      S.last_alpha = alpha;
    };

    // tiny step (Table I row 4)
    // max_i |dx_i| / (1 + |w_i|) < 10 eps, tested without a division per entry
    int big = 0;
    #pragma unroll 1
    for (int i = lane; i < c.nw; i += c.T) big |= fabs(dx[i]) >= 10.0 * kEpsMach * (1.0 + fabs(w[i]));
    if (!team_or(c, big)) {
      accept(a_max, sol, false);
      tiny = 1;
      S.n_tiny++;
      if (!c.resto) S.wd_short = 0;
      outcome = OUT_ACCEPTED;
    } else {
      tiny = 0;
      phi0 = barrier_phi(c, w, fph, mu, c.nw);
      double gd = 0.0;
      #pragma unroll 1
      for (int i = lane; i < c.nw; i += c.T) gd += gphi[i] * dx[i];
      gdx = team_sum(c, gd);
      double a_min;
      if (gdx < 0.0 && theta <= th_min)
        a_min = kGammaAlpha * fmin(kGammaTheta, fmin(kGammaPhi * theta / (-gdx),
                                                     kDelta * pow(theta, kSTheta) / pow(-gdx, kSPhi)));
      else if (gdx < 0.0)
        a_min = kGammaAlpha * fmin(kGammaTheta, kGammaPhi * theta / (-gdx));
      else
        a_min = kGammaAlpha * kGammaTheta;

      auto switching = [&](double alpha) {
        return gdx < 0.0 && alpha * pow(-gdx, kSPhi) > kDelta * pow(theta, kSTheta);
      };
      auto acceptable = [&](double th_t, double ph_t, double alpha) {
        if (!isfinite(ph_t) || in_filter(c, filt, nf, th_t, ph_t, th_max)) return false;
        if (switching(alpha) && theta <= th_min) return ph_t <= phi0 + kEtaPhi * alpha * gdx;
        return th_t <= (1.0 - kGammaTheta) * theta || ph_t <= phi0 - kGammaPhi * theta;
      };
      auto needs_augment = [&](double alpha, double ph_t) {
        return !(switching(alpha) && ph_t <= phi0 + kEtaPhi * alpha * gdx);
      };
      const bool globalize = !c.resto;  // watchdog and soft restoration: original problem only

      // soft restoration (Table I row 5): one primal-dual step alpha_s = min(alpha_max,
      // alpha_z_max); accepted if it passes the original tests (the soft phase ends)
      // or lowers the primal-dual error E_pd by the factor 1 - kappa_soft
      auto soft_step = [&]() {
        const double a_s = fmin(a_max, dual_max(dx));
        TrialVal tv = trial_point(c, a_s, dx);
        if (!tv.finite) return false;
        if (acceptable(tv.theta, tv.phi, 0.0)) {
          accept(a_s, sol, true, a_s);
          S.soft_active = 0;
          S.soft_iters = 0;
          return true;
        }
        // errors at the current point and at the trial (y and z moved by a_s too)
        const double e0 = pd_error(c, w, zl, zu, gf, jty, cv, mu);
        const double* xt = c.f + c.L.xt;
        double* gt = c.f + c.L.sft_g;
        double* jt = c.f + c.L.sft_j;
        double* yt = c.f + c.L.sft_y;
        double* zlt = c.f + c.L.res;
        double* zut = c.f + c.L.corr;
        LANE_LOOP(i, m) yt[i] = y[i] + a_s * dx[nwk + i];
        LANE_LOOP(i, n) {
          zlt[i] = zl[i];
          zut[i] = zu[i];
        }
        team_sync(c);
        {
          const int nb = n_bounded(d, n);
          #pragma unroll 1
          for (int b = lane; b < nb; b += c.T) {
            int kind;
            const int i = bnd_index(d, b, kind);
            zlt[i] = zl[i] + a_s * dz_lower(w[i], zl[i], mu, dx[i]);
            if (kind == VK_BOX) zut[i] = zu[i] + a_s * dz_upper(kUmax - w[i], zu[i], mu, dx[i]);
          }
        }
        team_sync(c);
        eval_grad(c, xt, gt);
        eval_jty(c, xt, yt, jt);
        if (!all_finite(c, gt, n) || !all_finite(c, jt, n)) return false;
        const double e1 = pd_error(c, xt, zlt, zut, gt, jt, ct, mu);
        if (!(e1 <= (1.0 - kKappaSoft) * e0)) return false;
        accept(a_s, sol, true, a_s);
        S.soft_active = 1;
        S.soft_iters++;
        return true;
      };

      // filter tests against the reference values stored when the watchdog started
      auto switching_ref = [&](double alpha) {
        return S.wd_gdx < 0.0 && alpha * pow(-S.wd_gdx, kSPhi) > kDelta * pow(S.wd_theta, kSTheta);
      };
      auto acceptable_ref = [&](double th_t, double ph_t, double alpha) {
        if (!isfinite(ph_t) || in_filter(c, filt, nf, th_t, ph_t, th_max)) return false;
        if (switching_ref(alpha) && S.wd_theta <= th_min) return ph_t <= S.wd_phi + kEtaPhi * alpha * S.wd_gdx;
        return th_t <= (1.0 - kGammaTheta) * S.wd_theta || ph_t <= S.wd_phi - kGammaPhi * S.wd_theta;
      };
      auto needs_augment_ref = [&](double alpha, double ph_t) {
        return !(switching_ref(alpha) && ph_t <= S.wd_phi + kEtaPhi * alpha * S.wd_gdx);
      };

      bool handled = false;
      if (globalize && opt.soft_resto && S.soft_active) {
        // in the soft restoration phase the soft step replaces the line search
        handled = true;
        if (S.soft_iters < kSoftMax && soft_step()) outcome = OUT_ACCEPTED;
      }
      if (!handled && globalize && opt.watchdog && !S.wd_active && S.wd_short >= kWdTrigger) {
        // watchdog (Table I row 3) starts: store the iterate, its step and references
        double* sx = c.f + c.L.wd_x;
        double* szl = c.f + c.L.wd_zl;
        double* szu = c.f + c.L.wd_zu;
        double* sy = c.f + c.L.wd_y;
        double* sd = c.f + c.L.wd_dir;
        LANE_LOOP(i, n) {
          sx[i] = w[i];
          szl[i] = zl[i];
          szu[i] = zu[i];
          sd[i] = dx[i];
        }
        LANE_LOOP(i, m) {
          sy[i] = y[i];
          sd[nwk + i] = dx[nwk + i];
        }
        team_sync(c);
        S.wd_active = 1;
        S.wd_trials = 0;
        S.wd_short = 0;
        S.wd_theta = theta;
        S.wd_phi = phi0;
        S.wd_gdx = gdx;
        S.wd_amax = a_max;
        S.wd_amin = a_min;
      }
      if (!handled && globalize && opt.watchdog && S.wd_active) {
        // the full step, judged against the stored iterate
        handled = true;
        TrialVal tv = trial_point(c, a_max, dx);
        if (tv.finite && acceptable_ref(tv.theta, tv.phi, a_max)) {
          theta0 = S.wd_theta;
          phi0 = S.wd_phi;
          accept(a_max, sol, needs_augment_ref(a_max, tv.phi));
          S.wd_active = 0;
          S.wd_trials = 0;
          outcome = OUT_ACCEPTED;
        } else if (++S.wd_trials <= kWdTrialMax) {
          accept(a_max, sol, false);  // unconditionally
          outcome = OUT_ACCEPTED;
        } else {
          // give up: back to the stored iterate, backtracking along its step from
          // half its full step (no second-order correction: its factors are gone)
          S.wd_active = 0;
          S.wd_trials = 0;
          const double* sd = c.f + c.L.wd_dir;
          LANE_LOOP(i, n) {
            w[i] = c.f[c.L.wd_x + i];
            zl[i] = c.f[c.L.wd_zl + i];
            zu[i] = c.f[c.L.wd_zu + i];
          }
          LANE_LOOP(i, m) y[i] = c.f[c.L.wd_y + i];
          team_sync(c);
          wd_restored = true;
          theta0 = S.wd_theta;
          phi0 = S.wd_phi;
          int n_try = 0;
          for (double alpha = 0.5 * S.wd_amax; alpha >= S.wd_amin && n_try < kLsMaxTrials; alpha *= 0.5) {
            ++n_try;
            TrialVal tv2 = trial_point(c, alpha, sd);
            if (tv2.finite && acceptable_ref(tv2.theta, tv2.phi, alpha)) {
              accept(alpha, sd, needs_augment_ref(alpha, tv2.phi));
              outcome = OUT_ACCEPTED;
              break;
            }
          }
        }
      }

      double alpha = a_max;
      int n_trial = 0;
      while (!handled) {
        ++n_trial;
        TrialVal tv = trial_point(c, alpha, dx);
        if (tv.finite) {
          if (acceptable(tv.theta, tv.phi, alpha)) {
            accept(alpha, sol, needs_augment(alpha, tv.phi));
            if (globalize) S.wd_short = alpha < a_max ? S.wd_short + 1 : 0;
            outcome = OUT_ACCEPTED;
            break;
          }
          if (n_trial == 1 && !(tv.theta < theta)) {
            // second-order correction (Table I row 2)
            LANE_LOOP(i, m) csoc[i] = alpha * cv[i] + ct[i];
            team_sync(c);
            double theta_old = theta;
            bool soc_ok = false;
            for (int p = 1; p <= kPmax; ++p) {
              S.n_soc++;
              LANE_LOOP(i, m) rhs2[nwk + i] = csoc[i];
              team_sync(c);
              c.esc_failed = 0;
              if (!solve_refined(c, rhs2, sol2) || c.esc_failed) break;  // no usable correction
              double a_soc = ftb_primal(c, w, sol2, tau);
              TrialVal sv = trial_point(c, a_soc, sol2);
              if (!sv.finite) break;
              if (acceptable(sv.theta, sv.phi, alpha)) {
                accept(a_soc, sol2, needs_augment(alpha, sv.phi));
                soc_ok = true;
                break;
              }
              if (p == kPmax || sv.theta > kKappaSoc * theta_old) break;
              LANE_LOOP(i, m) csoc[i] = a_soc * csoc[i] + ct[i];
              team_sync(c);
              theta_old = sv.theta;
            }
            if (soc_ok) {
              if (globalize) S.wd_short = 0;
              outcome = OUT_ACCEPTED;
              break;
            }
          }
        }
        alpha *= 0.5;
        if (alpha < a_min || n_trial >= kLsMaxTrials) {
          if (globalize && opt.soft_resto && soft_step()) outcome = OUT_ACCEPTED;
          break;
        }
      }
    }
  }
  lap(PH_LS);
  S.n_ir_steps += c.n_ir;
  S.n_escalations += c.n_esc;
  S.n_fact += c.n_fact;
  S.n_solve += c.n_solve;
  S.n_trial += c.n_trial;
  S.n_fact32 += c.n_fact32;
  S.n_solve32 += c.n_solve32;

  if (outcome == OUT_ACCEPTED) {
    S.cyc[PH_TOTAL] += clock64() - t_start;
    S.iter++;
    if (c.resto) {
      S.n_resto_iter++;
      // return test: enough reduction of the original infeasibility and
      // acceptable to the original filter at the original barrier parameter
      double f_o = eval_values(c, w, ct);
      double th_o = l1_norm(c, ct, m);
      double ph_o = barrier_phi(c, w, f_o, S.mu, n);
      const double* filt_o = c.f + c.L.filt;
      if (isfinite(ph_o) && th_o <= kKappaResto * S.theta_ref &&
          !in_filter(c, filt_o, S.n_filt, th_o, ph_o, S.theta_max)) {
        kappa_sigma_reset(c, n, S.mu);
        LANE_LOOP(i, 2 * m) {
          w[n + i] = 0.0;
          zl[n + i] = 0.0;
          zu[n + i] = 0.0;
        }
        team_sync(c);
        S.mode = MODE_NORMAL;
        S.need_y_ls = 1;
      }
    }
    return;
  }

  // ---- line search failed (or no regularisation gave the right inertia)
  S.cyc[PH_TOTAL] += clock64() - t_start;
  if (c.resto) {
    S.status = BIPM_RESTO_FAILED;
    return;
  }
  if (wd_restored) {
    // the failed search ran from the watchdog's stored iterate: restoration starts there
    f_orig = eval_values(c, w, cv);
    theta = l1_norm(c, cv, m);
  }
  if (theta <= opt.tol) {
    S.status = BIPM_RESTO_FAILED;
    return;
  }
  // enter restoration (IPOPT Sec. 3.3 reading)
  end_globalization(S);
  {
    double phi = barrier_phi(c, w, f_orig, S.mu, n);
    filter_add(c, filt, nf, (1.0 - kGammaTheta) * theta, phi - kGammaPhi * theta);
    double cmax = inf_norm(c, cv, m);
    double mu_r = fmax(S.mu, cmax);
    S.zeta = sqrt(S.mu);
    S.theta_ref = theta;
    LANE_LOOP(i, n) {
      xr[i] = w[i];
      int kind = var_kind(d, i);
      if (has_lower(kind)) zl[i] = fmin(kRho, zl[i]);
      if (has_upper(kind)) zu[i] = fmin(kRho, zu[i]);
    }
    double acc = 0.0;
    LANE_LOOP(i, m) {
      double ci = cv[i];
      double a = (mu_r - kRho * ci) / (2.0 * kRho);
      double nn = a + sqrt(a * a + mu_r * ci / (2.0 * kRho));
      double pp = ci + nn;
      w[n + i] = pp;
      w[n + m + i] = nn;
      zl[n + i] = mu_r / pp;
      zl[n + m + i] = mu_r / nn;
      zu[n + i] = 0.0;
      zu[n + m + i] = 0.0;
      y[i] = 0.0;
      acc += fabs(ci - pp + nn);
    }
    double th_r = team_sum(c, acc);
    team_sync(c);
    S.mu_r = mu_r;
    S.theta_max_r = 1e4 * fmax(1.0, th_r);
    S.theta_min_r = 1e-4 * fmax(1.0, th_r);
    S.n_filt_r = 0;
    S.dw_last_r = 0.0;
    S.tiny_r = 0;
    S.mode = MODE_RESTO;
    S.iter++;
  }
}

}  // namespace bipm
