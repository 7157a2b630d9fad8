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

#include "ipm_device.cuh"

namespace bipm {

enum Outcome : int { OUT_ACCEPTED = 0, OUT_LS_FAILED = 1 };

// ------------------------------------------------------------- reductions
template <class TB, class TF>
__device__ double l1_norm(Ctx<TB, TF>& c, const double* v, int len) {
  double a = 0.0;
  for (int i = c.lane; i < len; i += 32) a += fabs(v[i]);
  return warp_sum(a);
}
template <class TB, class TF>
__device__ double inf_norm(Ctx<TB, TF>& c, const double* v, int len) {
  double a = 0.0;
  for (int i = c.lane; i < len; i += 32) a = fmax(a, fabs(v[i]));
  return warp_max(a);
}
template <class TB, class TF>
__device__ bool all_finite(Ctx<TB, TF>& c, const double* v, int len) {
  int bad = 0;
  for (int i = c.lane; i < len; i += 32) bad |= !isfinite(v[i]);
  return !warp_or(bad);
}

// barrier objective phi_mu (Eq. 3) with the one-sided damping term, over the
// first `len` entries of a W-sized point w; +inf outside the bounds
template <class TB, class TF>
__device__ double barrier_phi(Ctx<TB, TF>& c, const double* w, double f, double mu, int len) {
  double acc = 0.0;
  int bad = 0;
  for (int i = c.lane; i < len; i += 32) {
    int kind = wkind(c.d, i);
    if (kind == VK_FREE) continue;
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
  if (warp_or(bad)) return INFINITY;
  return f + warp_sum(acc);
}

// scaled optimality error E_mu of Eq. 5 (IPOPT's scaling)
struct ErrParts {
  double dual, prim, y1, z1, nb;
};

template <class TB, class TF>
__device__ ErrParts err_parts(Ctx<TB, TF>& c) {
  const double* gf = c.f + c.L.gf;
  const double* jty = c.f + c.L.jty;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  const double* y = c.f + c.L.y;
  const double* cv = c.f + c.L.c;
  double du = 0.0, z1 = 0.0, nb = 0.0;
  for (int i = c.lane; i < c.nw; i += 32) {
    int kind = wkind(c.d, i);
    double zli = has_lower(kind) ? zl[i] : 0.0;
    double zui = has_upper(kind) ? zu[i] : 0.0;
    du = fmax(du, fabs(gf[i] + jty[i] - zli + zui));
    z1 += fabs(zli) + fabs(zui);
    nb += (has_lower(kind) ? 1.0 : 0.0) + (has_upper(kind) ? 1.0 : 0.0);
  }
  double pr = 0.0, y1 = 0.0;
  for (int i = c.lane; i < c.d.m; i += 32) {
    pr = fmax(pr, fabs(cv[i]));
    y1 += fabs(y[i]);
  }
  ErrParts e;
  e.dual = warp_max(du);
  e.prim = warp_max(pr);
  e.y1 = warp_sum(y1);
  e.z1 = warp_sum(z1);
  e.nb = warp_sum(nb);
  return e;
}

template <class TB, class TF>
__device__ double opt_error(Ctx<TB, TF>& c, const ErrParts& e, double mu) {
  const double* w = c.f + c.L.x;
  const double* zl = c.f + c.L.zl;
  const double* zu = c.f + c.L.zu;
  double comp = 0.0;
  for (int i = c.lane; i < c.nw; i += 32) {
    int kind = wkind(c.d, i);
    if (has_lower(kind)) comp = fmax(comp, fabs(w[i] * zl[i] - mu));
    if (has_upper(kind)) comp = fmax(comp, fabs((kUmax - w[i]) * zu[i] - mu));
  }
  comp = warp_max(comp);
  double nb = fmax(1.0, e.nb);
  double s_d = fmax(kSmax, (e.y1 + e.z1) / fmax(1.0, c.d.m + e.nb)) / kSmax;
  double s_c = fmax(kSmax, e.z1 / nb) / kSmax;
  return fmax(fmax(e.dual / s_d, e.prim), comp / s_c);
}

// largest alpha in (0, 1] keeping the bounded entries of w + alpha dw at least
// the fraction 1 - tau of their distance to the bounds
template <class TB, class TF>
__device__ double ftb_primal(Ctx<TB, TF>& c, const double* w, const double* dw, double tau) {
  double a = 1.0;
  for (int i = c.lane; i < c.nw; i += 32) {
    int kind = wkind(c.d, i);
    if (kind == VK_FREE) continue;
    if (dw[i] < 0.0) a = fmin(a, -tau * w[i] / dw[i]);
    if (kind == VK_BOX && dw[i] > 0.0) a = fmin(a, tau * (kUmax - w[i]) / dw[i]);
  }
  return warp_min(a);
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
__device__ __forceinline__ bool in_filter(const double* filt, int nf, double theta, double phi,
                                          double theta_max, int lane) {
  if (!(theta < theta_max)) return true;
  int hit = 0;
  for (int j = lane; j < nf; j += 32) hit |= (theta >= filt[2 * j] && phi >= filt[2 * j + 1]);
  return warp_or(hit);
}

__device__ __forceinline__ void filter_add(double* filt, int& nf, double theta, double phi,
                                           int lane) {
  int cnt = nf;
  if (lane == 0) {
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
  __syncwarp();
  nf = __shfl_sync(0xffffffffu, cnt, 0);
}

// -------------------------------------------------- factorisation and solve
template <class TB, class TF>
__device__ bool factor_any(Ctx<TB, TF>& c, double dw, bool force64) {
  const int flags = c.resto ? FF_RESTO : 0;
  const double* y = c.f + c.L.y;
  if (sizeof(TF) == 8 || c.resto || force64) {
    c.use64 = 1;
    return factor<TB, TF, double>(c, c.fac64, dw, flags, y) != 0;
  }
  int r = factor<TB, TF, TF>(c, c.fac, dw, flags, y);
  if (r == 0) return false;
  if (r == 2) {
    c.n_esc++;
    c.use64 = 1;
    return factor<TB, TF, double>(c, c.fac64, dw, flags, y) != 0;
  }
  c.use64 = 0;
  return true;
}

// Solves K out = -r.  With an FP32 factorisation the step is refined in FP64
// (residual with the FP64 KKT mat-vec, correction with the FP32 factors) until
// IPOPT's residual ratio drops below 1e-10; if that fails within 10 steps the
// matrix is refactorised in FP64.  Returns false only if that FP64
// refactorisation reports wrong inertia.
template <class TB, class TF>
__device__ bool solve_refined(Ctx<TB, TF>& c, const double* r, double* out) {
  const int flags = c.resto ? FF_RESTO : 0;
  const double* y = c.f + c.L.y;
  if (c.use64) {
    solve<TB, TF, double>(c, c.fac64, r, out, flags, y);
    return true;
  }
  solve<TB, TF, TF>(c, c.fac, r, out, flags, y);
  const int nwk = (int)c.L.nw;
  const int nused = c.nw;
  const int mm = c.d.m;
  double* res = c.f + c.L.res;
  double* corr = c.f + c.L.corr;
  // norms over the used entries: [0, nw) and [nwk, nwk + m)
  auto norm_used = [&](const double* v) {
    double a = 0.0;
    for (int i = c.lane; i < nused + mm; i += 32) {
      int j = i < nused ? i : nwk + (i - nused);
      a = fmax(a, fabs(v[j]));
    }
    return warp_max(a);
  };
  double rnorm = norm_used(r);
  if (rnorm == 0.0) return true;
  for (int it = 0; it <= kIrMaxSteps; ++it) {
    kkt_matvec(c, out, res, c.dw, y);
    for (int i = c.lane; i < nused + mm; i += 32) {
      int j = i < nused ? i : nwk + (i - nused);
      res[j] = -r[j] - res[j];
    }
    __syncwarp();
    double nres = norm_used(res);
    double snorm = norm_used(out);
    double ratio = nres / (fmin(snorm, 1e6 * rnorm) + rnorm);
    if (ratio <= kIrTol) return true;
    if (it == kIrMaxSteps) break;
    for (int i = c.lane; i < nused + mm; i += 32) {
      int j = i < nused ? i : nwk + (i - nused);
      res[j] = -res[j];
    }
    __syncwarp();
    solve<TB, TF, TF>(c, c.fac, res, corr, flags, y);
    for (int i = c.lane; i < nused + mm; i += 32) {
      int j = i < nused ? i : nwk + (i - nused);
      out[j] += corr[j];
    }
    __syncwarp();
    c.n_ir++;
  }
  // refinement did not converge: refactorise in FP64
  c.n_esc++;
  if (factor<TB, TF, double>(c, c.fac64, c.dw, flags, y) == 0) return false;
  c.use64 = 1;
  solve<TB, TF, double>(c, c.fac64, r, out, flags, y);
  return true;
}

// Least-squares multipliers: [[I, J^T], [J, 0]] (w, y) = (-(grad f - z_L + z_U), 0);
// y = 0 if |y|_inf > y_max.
template <class TB, class TF>
__device__ void ls_multipliers(Ctx<TB, TF>& c) {
  const Dims& d = c.d;
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
  __syncwarp();
  factor<TB, TF, double>(c, c.fac64, 0.0, FF_IDENT, y);
  solve<TB, TF, double>(c, c.fac64, rhs, sol, FF_IDENT, y);
  double ymax = inf_norm(c, sol + c.L.nw, d.m);
  LANE_LOOP(i, d.m) y[i] = ymax > kYmax ? 0.0 : sol[c.L.nw + i];
  __syncwarp();
}

// z <- max(min(z, kappa_Sigma mu / s), mu / (kappa_Sigma s)) over the first len entries
template <class TB, class TF>
__device__ void kappa_sigma_reset(Ctx<TB, TF>& c, int len, double mu) {
  double* w = c.f + c.L.x;
  double* zl = c.f + c.L.zl;
  double* zu = c.f + c.L.zu;
  for (int i = c.lane; i < len; i += 32) {
    int kind = wkind(c.d, i);
    if (has_lower(kind)) {
      double s = w[i];
      zl[i] = fmax(fmin(zl[i], kKappaSigma * mu / s), mu / (kKappaSigma * s));
    }
    if (has_upper(kind)) {
      double s = kUmax - w[i];
      zu[i] = fmax(fmin(zu[i], kKappaSigma * mu / s), mu / (kKappaSigma * s));
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------- iteration
template <class TB, class TF>
struct TrialVal {
  double theta, phi, f;
  bool finite;
};

// trial point w + alpha * dir: constraint violation and barrier objective of
// the current phase; the phase constraint vector goes to ct
template <class TB, class TF>
__device__ TrialVal<TB, TF> trial_point(Ctx<TB, TF>& c, double alpha, const double* dir) {
  const Dims& d = c.d;
  const int lane = c.lane;
  const double* w = c.f + c.L.x;
  double* xt = c.f + c.L.xt;
  double* ct = c.f + c.L.ct;
  LANE_LOOP(i, c.nw) xt[i] = w[i] + alpha * dir[i];
  __syncwarp();
  c.n_trial++;
  double f = eval_values(c, xt, ct);
  if (c.resto) {
    LANE_LOOP(i, d.m) ct[i] += -xt[d.n + i] + xt[d.n + d.m + i];
    __syncwarp();
    f = resto_objective(c, xt);
  }
  TrialVal<TB, TF> tv;
  tv.finite = isfinite(f) && all_finite(c, ct, d.m);
  tv.theta = l1_norm(c, ct, d.m);
  tv.phi = tv.finite ? barrier_phi(c, xt, f, c.mu, c.nw) : INFINITY;
  tv.f = f;
  return tv;
}

template <class TB, class TF>
__device__ void iterate(Ctx<TB, TF>& c, SlotState& S) {
  const Dims& d = c.d;
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
  double& mu = c.resto ? S.mu_r : S.mu;
  double& dw_last = c.resto ? S.dw_last_r : S.dw_last;
  double& th_max = c.resto ? S.theta_max_r : S.theta_max;
  double& th_min = c.resto ? S.theta_min_r : S.theta_min;
  int& tiny = c.resto ? S.tiny_r : S.tiny;
  int& nf = c.resto ? S.n_filt_r : S.n_filt;
  double* filt = c.f + (c.resto ? c.L.filt_r : c.L.filt);

  // ---- evaluation at the current point
  double f_orig = eval_values(c, w, cv);
  double fph = f_orig;
  if (c.resto) {
    LANE_LOOP(i, m) cv[i] += -w[n + i] + w[n + m + i];
    __syncwarp();
    fph = resto_objective(c, w);
  }
  eval_grad(c, w, gf);
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
  if (!c.resto && S.need_y_ls) ls_multipliers(c);
  eval_jty(c, w, y, jty);
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

  // ---- monotone barrier update (Table I row 7)
  {
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
        continue;
      }
      break;
    }
  }
  c.mu = mu;
  const double tau = fmax(kTauMin, 1.0 - mu);

  // ---- derivatives and the right-hand side of Eq. 7
  eval_blocks(c, w, y, true);
  LANE_LOOP(i, c.nw) {
    int kind = wkind(d, i);
    double g = gf[i];
    if (has_lower(kind)) g -= mu / w[i];
    if (has_upper(kind)) g += mu / (kUmax - w[i]);
    if (kind == VK_LOWER) g += kKappaD * mu;
    gphi[i] = g;
    rhs[i] = g + jty[i];
    rhs2[i] = g + jty[i];
  }
  LANE_LOOP(i, m) rhs[nwk + i] = cv[i];
  __syncwarp();

  // ---- inertia correction (IPOPT Algorithm IC) and the Newton step
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
    if (solve_refined(c, rhs, sol)) break;
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
  if (!ls_fail) {
    const double* dx = sol;
    double a_max = ftb_primal(c, w, dx, tau);

    // accept a step (alpha, dir) with dir K-sized; the z step follows from dir
    auto accept = [&](double alpha, const double* dir, bool augment) {
      const double* ddx = dir;
      const double* ddy = dir + nwk;
      double az = 1.0;
      for (int i = lane; i < c.nw; i += 32) {
        int kind = wkind(d, i);
        if (has_lower(kind)) {
          double dzl = dz_lower(w[i], zl[i], mu, ddx[i]);
          if (dzl < 0.0) az = fmin(az, -tau * zl[i] / dzl);
        }
        if (has_upper(kind)) {
          double dzu = dz_upper(kUmax - w[i], zu[i], mu, ddx[i]);
          if (dzu < 0.0) az = fmin(az, -tau * zu[i] / dzu);
        }
      }
      az = warp_min(az);
      for (int i = lane; i < c.nw; i += 32) {
        int kind = wkind(d, i);
        double dzl = has_lower(kind) ? dz_lower(w[i], zl[i], mu, ddx[i]) : 0.0;
        double dzu = has_upper(kind) ? dz_upper(kUmax - w[i], zu[i], mu, ddx[i]) : 0.0;
        w[i] += alpha * ddx[i];
        if (has_lower(kind)) zl[i] += az * dzl;
        if (has_upper(kind)) zu[i] += az * dzu;
      }
      LANE_LOOP(i, m) y[i] += alpha * ddy[i];
      __syncwarp();
      kappa_sigma_reset(c, c.nw, mu);
      if (augment) filter_add(filt, nf, (1.0 - kGammaTheta) * theta0, phi0 - kGammaPhi * theta0, lane);
      S.last_alpha = alpha;
    };

    // tiny step (Table I row 4)
    double rel = 0.0;
    for (int i = lane; i < c.nw; i += 32) rel = fmax(rel, fabs(dx[i]) / (1.0 + fabs(w[i])));
    rel = warp_max(rel);
    if (rel < 10.0 * kEpsMach) {
      accept(a_max, sol, false);
      tiny = 1;
      S.n_tiny++;
      outcome = OUT_ACCEPTED;
    } else {
      tiny = 0;
      phi0 = barrier_phi(c, w, fph, mu, c.nw);
      double gd = 0.0;
      for (int i = lane; i < c.nw; i += 32) gd += gphi[i] * dx[i];
      gdx = warp_sum(gd);
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
        if (!isfinite(ph_t) || in_filter(filt, nf, th_t, ph_t, th_max, lane)) return false;
        if (switching(alpha) && theta <= th_min) return ph_t <= phi0 + kEtaPhi * alpha * gdx;
        return th_t <= (1.0 - kGammaTheta) * theta || ph_t <= phi0 - kGammaPhi * theta;
      };
      auto needs_augment = [&](double alpha, double ph_t) {
        return !(switching(alpha) && ph_t <= phi0 + kEtaPhi * alpha * gdx);
      };

      double alpha = a_max;
      int n_trial = 0;
      while (true) {
        ++n_trial;
        TrialVal<TB, TF> tv = trial_point(c, alpha, dx);
        if (tv.finite) {
          if (acceptable(tv.theta, tv.phi, alpha)) {
            accept(alpha, sol, needs_augment(alpha, tv.phi));
            outcome = OUT_ACCEPTED;
            break;
          }
          if (n_trial == 1 && !(tv.theta < theta)) {
            // second-order correction (Table I row 2)
            LANE_LOOP(i, m) csoc[i] = alpha * cv[i] + ct[i];
            __syncwarp();
            double theta_old = theta;
            bool soc_ok = false;
            for (int p = 1; p <= kPmax; ++p) {
              S.n_soc++;
              LANE_LOOP(i, m) rhs2[nwk + i] = csoc[i];
              __syncwarp();
              if (!solve_refined(c, rhs2, sol2)) break;
              double a_soc = ftb_primal(c, w, sol2, tau);
              TrialVal<TB, TF> sv = trial_point(c, a_soc, sol2);
              if (!sv.finite) break;
              if (acceptable(sv.theta, sv.phi, alpha)) {
                accept(a_soc, sol2, needs_augment(alpha, sv.phi));
                soc_ok = true;
                break;
              }
              if (p == kPmax || sv.theta > kKappaSoc * theta_old) break;
              LANE_LOOP(i, m) csoc[i] = a_soc * csoc[i] + ct[i];
              __syncwarp();
              theta_old = sv.theta;
            }
            if (soc_ok) {
              outcome = OUT_ACCEPTED;
              break;
            }
          }
        }
        alpha *= 0.5;
        if (alpha < a_min || n_trial >= kLsMaxTrials) break;
      }
    }
  }
  S.n_ir_steps += c.n_ir;
  S.n_escalations += c.n_esc;
  S.n_fact += c.n_fact;
  S.n_solve += c.n_solve;
  S.n_trial += c.n_trial;

  if (outcome == OUT_ACCEPTED) {
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
          !in_filter(filt_o, S.n_filt, th_o, ph_o, S.theta_max, lane)) {
        kappa_sigma_reset(c, n, S.mu);
        LANE_LOOP(i, 2 * m) {
          w[n + i] = 0.0;
          zl[n + i] = 0.0;
          zu[n + i] = 0.0;
        }
        __syncwarp();
        S.mode = MODE_NORMAL;
        S.need_y_ls = 1;
      }
    }
    return;
  }

  // ---- line search failed (or no regularisation gave the right inertia)
  if (c.resto) {
    S.status = BIPM_RESTO_FAILED;
    return;
  }
  if (theta <= opt.tol) {
    S.status = BIPM_RESTO_FAILED;
    return;
  }
  // enter restoration (IPOPT Sec. 3.3 reading)
  {
    double phi = barrier_phi(c, w, f_orig, S.mu, n);
    filter_add(filt, nf, (1.0 - kGammaTheta) * theta, phi - kGammaPhi * theta, lane);
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
    double th_r = warp_sum(acc);
    __syncwarp();
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
