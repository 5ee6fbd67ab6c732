// mma.cpp -- the design update of Alg. 3 on the host: the Method of Moving Asymptotes
// (Svanberg 1987) for min f0(x) subject to one constraint f1(x) <= 0 and x_min <= x <= x_max.
// The paper uses a variant for large projection sharpness that it does not give; this is the
// plain method.
//
// One step from the iterate x (objective f0, constraint f1, their gradients df0, df1):
//   asymptotes  L, U = x -/+ (x_max - x_min) / 2 in the first two steps; afterwards
//               L = x - g (x' - L'), U = x + g (U' - x') with the previous iterate x' and
//               asymptotes L', U', where g = 0.7 if the component oscillated over the last two
//               steps, 1.2 if it moved the same way twice, 1 otherwise;
//   box         a = max(x_min, L + 0.1 (x - L), x - move), b = min(x_max, U - 0.1 (U - x), x + move);
//   models      f_i ~ r_i + sum_j p_ij / (U_j - x_j) + q_ij / (x_j - L_j) with
//               p_ij = (U_j - x_j)^2 (max(0, d_j f_i) + e_ij), q_ij = (x_j - L_j)^2 (max(0, -d_j f_i) + e_ij),
//               e_ij = 1e-3 |d_j f_i| + 1e-6 / (x_max - x_min) (strict convexity);
//   subproblem  minimise the f0 model subject to the f1 model <= 0 and a <= x <= b through the
//               dual in the multiplier lam >= 0: each x_j(lam) minimises
//               (p0j + lam p1j) / (U_j - x) + (q0j + lam q1j) / (x - L_j) over [a_j, b_j], which is
//               (L_j sqrt(P) + U_j sqrt(Q)) / (sqrt(P) + sqrt(Q)) clipped; the f1 model at x(lam)
//               decreases in lam: lam = 0 if it holds there, else its root by bisection.
// Host FP64; the result does not depend on thread count or timing.
#include <cmath>
#include <cstddef>
#include <new>
#include <vector>
#include "../../include/ptg.h"

struct ptg_mma {
  int n = 0;
  double x_min = 0, x_max = 1, move = 0.2;
  long k = 0;
  std::vector<double> x1, x2, L, U;                 // previous two iterates, previous asymptotes
  std::vector<double> a, b, p0, q0, p1, q1, Lc, Uc;  // work arrays of one step
};

namespace {

// the f1 model at x(lam); writes x(lam) to xo
double constraint_at(const ptg_mma& m, double lam, double r1, double* xo) {
  double g = r1;
  for (int j = 0; j < m.n; ++j) {
    const double P = m.p0[j] + lam * m.p1[j], Q = m.q0[j] + lam * m.q1[j];
    const double sP = std::sqrt(P), sQ = std::sqrt(Q);
    double x = (m.Lc[j] * sP + m.Uc[j] * sQ) / (sP + sQ);
    if (x < m.a[j]) x = m.a[j];
    if (x > m.b[j]) x = m.b[j];
    xo[j] = x;
    g += m.p1[j] / (m.Uc[j] - x) + m.q1[j] / (x - m.Lc[j]);
  }
  return g;
}

}  // namespace

extern "C" {

int ptg_mma_create(int n, double x_min, double x_max, double move, ptg_mma** out) {
  if (!out) return PTG_EINVAL;
  *out = nullptr;
  if (n < 1 || !(x_max > x_min) || !(move > 0.0)) return PTG_EINVAL;
  ptg_mma* m = new (std::nothrow) ptg_mma();
  if (!m) return PTG_ENOMEM;
  try {
    m->n = n;
    m->x_min = x_min;
    m->x_max = x_max;
    m->move = move;
    for (auto* v : {&m->x1, &m->x2, &m->L, &m->U, &m->a, &m->b, &m->p0, &m->q0, &m->p1, &m->q1, &m->Lc, &m->Uc})
      v->assign(n, 0.0);
  } catch (...) {
    delete m;
    return PTG_ENOMEM;
  }
  *out = m;
  return PTG_OK;
}

void ptg_mma_destroy(ptg_mma* m) { delete m; }

int ptg_mma_update(ptg_mma* m, const double* x, double f0, const double* df0, double f1, const double* df1,
                   double* x_new) {
  if (!m || !x || !df0 || !df1 || !x_new) return PTG_EINVAL;
  (void)f0;   // the model of f0 needs only its gradient (its constant does not move the minimiser)
  const int n = m->n;
  const double span = m->x_max - m->x_min;
  double r1 = f1;
  for (int j = 0; j < n; ++j) {
    const double xj = x[j];
    double L, U;
    if (m->k < 2) {
      L = xj - 0.5 * span;
      U = xj + 0.5 * span;
    } else {
      const double s = (xj - m->x1[j]) * (m->x1[j] - m->x2[j]);
      const double g = s < 0.0 ? 0.7 : (s > 0.0 ? 1.2 : 1.0);
      L = xj - g * (m->x1[j] - m->L[j]);
      U = xj + g * (m->U[j] - m->x1[j]);
    }
    m->Lc[j] = L;
    m->Uc[j] = U;
    double a = L + 0.1 * (xj - L), b = U - 0.1 * (U - xj);
    if (a < m->x_min) a = m->x_min;
    if (a < xj - m->move) a = xj - m->move;
    if (b > m->x_max) b = m->x_max;
    if (b > xj + m->move) b = xj + m->move;
    m->a[j] = a;
    m->b[j] = b;
    const double u2 = (U - xj) * (U - xj), l2 = (xj - L) * (xj - L);
    const double d0 = df0[j], d1 = df1[j];
    const double e0 = 1e-3 * std::fabs(d0) + 1e-6 / span, e1 = 1e-3 * std::fabs(d1) + 1e-6 / span;
    m->p0[j] = u2 * ((d0 > 0.0 ? d0 : 0.0) + e0);
    m->q0[j] = l2 * ((d0 < 0.0 ? -d0 : 0.0) + e0);
    m->p1[j] = u2 * ((d1 > 0.0 ? d1 : 0.0) + e1);
    m->q1[j] = l2 * ((d1 < 0.0 ? -d1 : 0.0) + e1);
    r1 -= m->p1[j] / (U - xj) + m->q1[j] / (xj - L);
  }
  // the dual in lam: bisection on the decreasing f1 model at x(lam)
  if (constraint_at(*m, 0.0, r1, x_new) > 0.0) {
    double lo = 0.0, hi = 1.0;
    while (constraint_at(*m, hi, r1, x_new) > 0.0 && hi < 1e30) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (constraint_at(*m, mid, r1, x_new) > 0.0)
        lo = mid;
      else
        hi = mid;
      if (hi - lo <= 1e-14 * hi) break;
    }
    constraint_at(*m, hi, r1, x_new);
  }
  m->x2 = m->x1;
  m->x1.assign(x, x + n);
  m->L = m->Lc;
  m->U = m->Uc;
  ++m->k;
  return PTG_OK;
}

int ptg_mma_get_state(const ptg_mma* m, long long* k, double* x1, double* x2, double* L, double* U) {
  if (!m || !k || !x1 || !x2 || !L || !U) return PTG_EINVAL;
  *k = m->k;
  for (int j = 0; j < m->n; ++j) {
    x1[j] = m->x1[j];
    x2[j] = m->x2[j];
    L[j] = m->L[j];
    U[j] = m->U[j];
  }
  return PTG_OK;
}

int ptg_mma_set_state(ptg_mma* m, long long k, const double* x1, const double* x2, const double* L, const double* U) {
  if (!m || k < 0 || !x1 || !x2 || !L || !U) return PTG_EINVAL;
  m->k = (long)k;
  m->x1.assign(x1, x1 + m->n);
  m->x2.assign(x2, x2 + m->n);
  m->L.assign(L, L + m->n);
  m->U.assign(U, U + m->n);
  return PTG_OK;
}

}  // extern "C"
