// Scheme set-up shared by gbs_set_weights and gbs_step_noalloc (host only, no heap use):
// the dependent weights from the free ones and the order constraints, in double-double.
//
// Sec. 3.2 eq. "vander" and Sec. 3.7 eqs. "order_constraints" / "cdep_computation": with
// x_k = 1 / N_k^2 the weights satisfy sum_k c_k x_k^j = [j == 0] for j = 0 .. p/2 - 1.  The
// p/2 dependent weights solve V_dep c_dep = b - V_free c_free, a transposed Vandermonde system
// solved by the Bjorck-Pereyra algorithm (its dual form) in double-double, then rounded to
// FP64.  The rounded weights must still satisfy every constraint to 64 ulp of
// sum_k |c_k| x_k^j, else the scheme is refused (GBS_ERR_ORDER).
#pragma once

#include <cmath>
#include <cstdio>

#include "gbs.h"
#include "gbs_dd.h"

namespace gbs {

inline dd inv_sq(int n) { return dd_from(1.0) / dd_from(double(n) * double(n)); }

// Solve the transposed Vandermonde system sum_i x_i^j c_i = b_j (j = 0..n) in place in b
// (Bjorck & Pereyra 1970, dual algorithm).
inline void bjorck_pereyra_dual(const dd* x, dd* b, int q) {
  const int n = q - 1;
  for (int k = 0; k < n; ++k)
    for (int i = n; i > k; --i) b[i] = b[i] - x[k] * b[i - 1];
  for (int k = n - 1; k >= 0; --k) {
    for (int i = k + 1; i <= n; ++i) b[i] = b[i] / (x[i] - x[i - k - 1]);
    for (int i = k; i < n; ++i) b[i] = b[i] - b[i + 1];
  }
}

// Residual check of the order constraints for weights c of the m step counts `steps`.
inline gbs_status check_order_constraints(int order_p, int m, const int* steps, const double* c, char* msg,
                                          size_t msglen) {
  for (int j = 0; j < order_p / 2; ++j) {
    dd sum = dd_from(j == 0 ? -1.0 : 0.0);
    double scale = 0.0;
    for (int k = 0; k < m; ++k) {
      dd pw = dd_from(1.0);
      const dd hx = inv_sq(steps[k]);
      for (int e = 0; e < j; ++e) pw = pw * hx;
      sum = sum + dd_from(c[k]) * pw;
      scale += std::fabs(c[k]) * (pw.hi + pw.lo);
    }
    const double res = std::fabs(sum.hi + sum.lo);
    if (!(res <= 64.0 * 2.220446049250313e-16 * scale)) {
      std::snprintf(msg, msglen, "order constraint j=%d violated: residual %.3e > 64 ulp of %.3e", j, res, scale);
      return GBS_ERR_ORDER;
    }
  }
  return GBS_OK;
}

// Weights c[0 .. n_dep + n_free) of the scheme whose first n_dep = order_p / 2 step counts are
// dependent: c_dep from c_free (non-finite free weights: GBS_ERR_INVALID), then the residual
// check.  `steps` holds the dependent counts followed by the free ones.
inline gbs_status scheme_weights(int order_p, int n_dep, int n_free, const int* steps, const double* c_free,
                                 double* c, char* msg, size_t msglen) {
  dd x[GBS_MAX_SEQ], r[GBS_MAX_SEQ];
  for (int i = 0; i < n_free; ++i)
    if (!std::isfinite(c_free[i])) {
      std::snprintf(msg, msglen, "free weight %d is not finite", i);
      return GBS_ERR_INVALID;
    }
  for (int i = 0; i < n_dep; ++i) x[i] = inv_sq(steps[i]);
  for (int j = 0; j < n_dep; ++j) {
    dd rj = dd_from(j == 0 ? 1.0 : 0.0);
    for (int i = 0; i < n_free; ++i) {
      dd pw = dd_from(1.0);
      const dd hx = inv_sq(steps[n_dep + i]);
      for (int e = 0; e < j; ++e) pw = pw * hx;
      rj = rj - dd_from(c_free[i]) * pw;
    }
    r[j] = rj;
  }
  bjorck_pereyra_dual(x, r, n_dep);
  for (int i = 0; i < n_dep; ++i) c[i] = r[i].hi + r[i].lo;
  for (int i = 0; i < n_free; ++i) c[n_dep + i] = c_free[i];
  for (int k = 0; k < n_dep + n_free; ++k)
    if (!std::isfinite(c[k])) {
      std::snprintf(msg, msglen, "weight %d is not finite", k);
      return GBS_ERR_ORDER;
    }
  return check_order_constraints(order_p, n_dep + n_free, steps, c, msg, msglen);
}

}  // namespace gbs
