// seed_device.cuh -- the scalar part of the Sec. 3 recurrence, shared by the
// step-by-step kernels (krylov.cu) and the persistent kernels (persistent.cu).
// It runs in thread 0 of a block that holds the reduced sums.  G = true: the
// state (SeedState, eta) is in global memory and the block is whichever block
// finished a reduction last, on any SM, so state is read with L2 loads (never
// from a stale L1 line written by another SM), all issued before their values
// are used so that their round trips overlap.  G = false: the state is the
// block's own shared-memory copy (the persistent kernels keep one per block).
// History arrays that are NULL are not written.
#pragma once
#include <math.h>

#include "device_common.cuh"
#include "seed_internal.h"

namespace seedk {

template <bool G, class P> SEED_DEV P sld(const P *p) {
  if constexpr (G) return __ldcg(p);
  else return *p;
}

// The LU update (delta_i, gamma_{i-1}, zeta_i) and the seeding scalars (eta^j) from alpha_i and
// g^j = v_i^H r_0^j (sums[j], j = 1..nrhs-1); beta_{i-1} is st->beta_prev.
template <class T, bool G = true>
SEED_DEV void seed_step_scalars(const SeedBufs<T> &b, int i, double a, const double2 *sums) {
  SeedState *st = b.st;
  const double bp = sld<G>(&st->beta_prev), inv_dprev = sld<G>(&st->inv_delta), zprev = sld<G>(&st->zeta),
               beta0 = sld<G>(&st->beta0);
  const int nr = b.Wb == nullptr ? b.nrhs : 1;
  double2 e[kMaxRhs];
#pragma unroll 16
  for (int j = 1; j < nr; ++j) e[j] = sld<G>(b.eta + j);
  double gam, del, zet;
  if (i == 1) {           // first step: delta_1 = alpha_1, zeta_1 = beta_0
    gam = 0.0;
    del = a;
    zet = beta0;
  } else {                // later steps (gamma_{i-1} = beta_{i-1} / delta_{i-1}, by the stored reciprocal:
                          // a division costs this part's FP64 pipe about as much as 20 multiplies)
    gam = bp * inv_dprev;
    del = a - gam * bp;
    zet = -gam * zprev;
  }
  if (b.Wb == nullptr) {
#pragma unroll 16
    for (int j = 1; j < nr; ++j) {   // seeding of systems 2..p
      const double2 g = sums[j];
      b.eta[j] = (i == 1) ? g : c2(g.x - gam * e[j].x, g.y - gam * e[j].y);
    }
  } else if (b.gamma_hist) {         // blocked seeding: eta^j at the block's flush
    b.gamma_hist[i] = gam;
  }
  st->alpha = a;
  st->gamma = gam;
  st->delta = del;
  st->inv_delta = 1.0 / del;
  st->zeta = zet;
  if (b.alpha_hist) b.alpha_hist[i] = a;
  if (b.delta_hist) b.delta_hist[i] = del;
  if (!(del > 0.0) || !isfinite(del)) {
    st->active = 0;
    st->stop_reason = STOP_NOTSPD;
  }
}

// Sec. 3, end of a step: beta_i = ||f||, residual estimate and the stopping test.
template <class T, bool G = true>
SEED_DEV void seed_finish(const SeedBufs<T> &b, double sumsq) {
  SeedState *st = b.st;
  const int i = sld<G>(&st->i);
  const double alpha = sld<G>(&st->alpha), bp = sld<G>(&st->beta_prev), tnorm = sld<G>(&st->tnorm),
               zeta = sld<G>(&st->zeta), inv_delta = sld<G>(&st->inv_delta), tol_abs = sld<G>(&st->tol_abs),
               brel = sld<G>(&st->breakdown_rel);
  int converged_at = sld<G>(&st->converged_at), stop_at = sld<G>(&st->stop_at);
  const int extra = sld<G>(&st->extra_iters), m_max = sld<G>(&st->m_max);
  const double beta = sqrt(sumsq);
  if (b.beta_hist) b.beta_hist[i] = beta;
  const double row = fabs(alpha) + (i > 1 ? bp : 0.0) + beta;
  const double tn = row > tnorm ? row : tnorm;
  const double rho = beta * fabs(zeta) * inv_delta;
  if (converged_at < 0 && rho <= tol_abs) {
    converged_at = i;
    stop_at = i + extra;
  }
  int stop = STOP_RUNNING;
  if (beta <= brel * tn) stop = STOP_BREAKDOWN;
  else if (stop_at >= 0 && i >= stop_at) stop = STOP_CONVERGED;
  else if (i >= m_max) stop = STOP_MMAX;
  st->tnorm = tn;
  st->rho = rho;
  st->beta = beta;
  st->converged_at = converged_at;
  st->stop_at = stop_at;
  if (stop != STOP_RUNNING) {
    st->active = 0;
    st->stop_reason = stop;
  } else {
    st->beta_prev = beta;
    st->inv_beta = 1.0 / beta;
    st->i = i + 1;
  }
}

// Lockstep CG, after x += alpha p, r -= alpha q and rr = ||r||^2 (thread 0 of
// the block that reduced column col): count the iteration, stop the column
// when ||r|| <= tol ||b|| (or at the iteration cap; the true residual is
// checked afterwards), else beta = rr / rho and rho = rr.
SEED_DEV void cg_update_tail(const CgCols &c, int col, double rr) {
  const double rn = sqrt(rr), bn = c.bnorm[col];
  c.iters[col] += 1;
  c.mvps[col] += 1;
  c.relres[col] = bn > 0.0 ? rn / bn : 0.0;
  if (rn <= c.tol * bn) {
    c.active[col] = 0;
    c.reached[col] = 1;
    c.needs_check[col] = 1;
  } else if (c.iters[col] >= c.maxit || !isfinite(rr)) {
    // a NaN or infinite residual (non-finite input, or p^H A p <= 0 on an
    // operator that is not positive definite) ends the column unconverged
    c.active[col] = 0;
    c.needs_check[col] = 1;
  } else {
    c.beta[col] = rr / c.rho[col];
    c.rho[col] = rr;
  }
}

}  // namespace seedk
