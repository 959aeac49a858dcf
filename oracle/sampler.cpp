// Oracle sampler: leapfrog with boundary maps, multinomial NUTS, adaptive
// tempering, systematic resampling, weighted covariance and the full SMC run.
// TEST INFRASTRUCTURE ONLY (see oracle.h).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "oracle.h"

namespace oracle {
void uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[2]);
void normal2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[2]);
void loglike_one(const ref_model* m, const ref_event* ev, const double* theta, double* lnl, double* grad);
double prior_logpdf_one(const ref_model* m, const double* x, double* g);

// Philox counter word 2 ("purpose") of every random draw.
enum { P_PRIOR = 1, P_MOMENTUM = 2, P_DIRECTION = 3, P_LEAF = 4, P_TOP = 5, P_RESAMPLE = 6 };

const int kMaxDepth = 12;
const double kDivergence = 1000.0;

static double logaddexp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double m = a > b ? a : b;
  return m + std::log(std::exp(a - m) + std::exp(b - m));
}

// One point of a Hamiltonian trajectory.
struct Point {
  double th[REF_MAX_DIM];
  double r[REF_MAX_DIM];
  double gl[REF_MAX_DIM];  // grad ln L
  double gu[REF_MAX_DIM];  // grad U, U = -beta ln L - ln pi
  double lnl, lp, u;
};

struct Sampler {
  const ref_model* m;
  const ref_event* ev;
  int D;
  double beta;
  double minv[REF_MAX_DIM][REF_MAX_DIM];  // inverse mass matrix (metric)
  double chol[REF_MAX_DIM][REF_MAX_DIM];  // lower factor: minv = L L^T

  void velocity(const double* r, double* v) const {
    for (int i = 0; i < D; ++i) {
      double s = 0.0;
      for (int j = 0; j < D; ++j) s += minv[i][j] * r[j];
      v[i] = s;
    }
  }
  double kinetic(const double* r) const {
    double v[REF_MAX_DIM];
    velocity(r, v);
    double s = 0.0;
    for (int i = 0; i < D; ++i) s += r[i] * v[i];
    return 0.5 * s;
  }
  // rho . M^{-1} r
  double sharp_dot(const double* rho, const double* r) const {
    double v[REF_MAX_DIM];
    velocity(r, v);
    double s = 0.0;
    for (int i = 0; i < D; ++i) s += rho[i] * v[i];
    return s;
  }
  bool no_uturn(const double* rho, const double* ra, const double* rb) const {
    return sharp_dot(rho, ra) > 0.0 && sharp_dot(rho, rb) > 0.0;
  }

  // Evaluate ln L, grad ln L, ln pi, grad ln pi, U and grad U at p.th.
  void evaluate(Point& p) const {
    double glp[REF_MAX_DIM];
    loglike_one(m, ev, p.th, &p.lnl, p.gl);
    p.lp = prior_logpdf_one(m, p.th, glp);
    for (int i = 0; i < D; ++i) p.gu[i] = -beta * p.gl[i] - glp[i];
    p.u = -beta * p.lnl - p.lp;
  }

  // Boundary maps after a drift. Reflective: mirror the coordinate into the
  // box, and for each mirror flip the velocity component normal to the wall
  // (momentum update r_i -= 2 v_i / Minv_ii, which keeps the kinetic energy).
  // Periodic: wrap into [lo, hi), momentum unchanged. Returns false if a
  // coordinate cannot be brought back (non-finite).
  bool boundary(double* th, double* r) const {
    for (int i = 0; i < D; ++i) {
      double lo = m->lo[i], hi = m->hi[i];
      if (!std::isfinite(th[i])) return false;
      if (m->boundary[i] == REF_BOUND_PERIODIC) {
        double w = hi - lo;
        double t = std::fmod(th[i] - lo, w);
        if (t < 0.0) t += w;
        th[i] = lo + t;
      } else {
        int flips = 0;
        while ((th[i] < lo || th[i] > hi) && flips < 100) {
          th[i] = th[i] < lo ? 2.0 * lo - th[i] : 2.0 * hi - th[i];
          ++flips;
        }
        if (th[i] < lo || th[i] > hi) return false;
        if (flips & 1) {
          double v[REF_MAX_DIM];
          velocity(r, v);
          r[i] = r[i] - 2.0 * v[i] / minv[i][i];
        }
      }
    }
    return true;
  }

  // Leapfrog step of signed size h (Sec. 4, Eqs. (11)-(13)).
  bool leapfrog(const Point& a, double h, Point& b) const {
    double v[REF_MAX_DIM];
    for (int i = 0; i < D; ++i) b.r[i] = a.r[i] - 0.5 * h * a.gu[i];
    velocity(b.r, v);
    for (int i = 0; i < D; ++i) b.th[i] = a.th[i] + h * v[i];
    if (!boundary(b.th, b.r)) return false;
    evaluate(b);
    for (int i = 0; i < D; ++i) b.r[i] = b.r[i] - 0.5 * h * b.gu[i];
    return true;
  }

  // One multinomial NUTS transition of particle `pid` at step counter `step`.
  void transition(Point& cur, uint64_t key, uint32_t pid, uint32_t step, double eps, int max_depth,
                  ref_nuts_stats* st) const {
    // momentum r ~ N(0, M), M = minv^{-1}: solve L^T r = z
    double z[REF_MAX_DIM + 1];
    for (int p = 0; 2 * p < D; ++p) normal2(key, pid, step, P_MOMENTUM, (uint32_t)p, z + 2 * p);
    Point left = cur;
    for (int i = D - 1; i >= 0; --i) {
      double s = z[i];
      for (int j = i + 1; j < D; ++j) s -= chol[j][i] * left.r[j];
      left.r[i] = s / chol[i][i];
    }
    Point right = left;
    double H0 = left.u + kinetic(left.r);
    Point prop = left;
    double logw = 0.0;
    double rho[REF_MAX_DIM];
    for (int i = 0; i < D; ++i) rho[i] = left.r[i];

    int depth = 0, n_leaf = 0;
    uint32_t leaf_ctr = 0;
    double acc = 0.0;
    bool divergent = false;
    while (depth < max_depth) {
      double ud[2];
      uniform2(key, pid, step, P_DIRECTION, (uint32_t)depth, ud);
      int dir = ud[0] < 0.5 ? -1 : 1;
      Point edge = dir > 0 ? right : left;
      Point prop_sub = edge;
      double logw_sub = -INFINITY;
      double rho_sub[REF_MAX_DIM] = {0};
      double rho_start[kMaxDepth + 1][REF_MAX_DIM];
      double r_first[kMaxDepth + 1][REF_MAX_DIM];
      bool ok = true;
      long n_sub = 1L << depth;
      for (long n = 0; n < n_sub && ok; ++n) {
        Point nxt;
        bool fin = leapfrog(edge, dir * eps, nxt);
        ++n_leaf;
        double dH = fin ? nxt.u + kinetic(nxt.r) - H0 : NAN;
        acc += (dH == dH) ? std::fmin(1.0, std::exp(-dH)) : 0.0;
        if (!(dH <= kDivergence)) {
          divergent = true;
          ok = false;
          break;
        }
        edge = nxt;
        double lw = -dH;
        double lw_new = logaddexp(logw_sub, lw);
        double ul[2];
        uniform2(key, pid, step, P_LEAF, leaf_ctr++, ul);
        if (ul[0] < std::exp(lw - lw_new)) prop_sub = nxt;
        logw_sub = lw_new;
        for (int lvl = 1; lvl <= depth; ++lvl)
          if (n % (1L << lvl) == 0) {
            for (int i = 0; i < D; ++i) {
              rho_start[lvl][i] = rho_sub[i];
              r_first[lvl][i] = nxt.r[i];
            }
          }
        for (int i = 0; i < D; ++i) rho_sub[i] += nxt.r[i];
        for (int lvl = 1; lvl <= depth; ++lvl)
          if ((n + 1) % (1L << lvl) == 0) {
            double rb[REF_MAX_DIM];
            for (int i = 0; i < D; ++i) rb[i] = rho_sub[i] - rho_start[lvl][i];
            if (!no_uturn(rb, r_first[lvl], nxt.r)) {
              ok = false;
              break;
            }
          }
      }
      if (!ok) break;
      double ut[2];
      uniform2(key, pid, step, P_TOP, (uint32_t)depth, ut);
      if (ut[0] < std::exp(logw_sub - logw)) prop = prop_sub;
      logw = logaddexp(logw, logw_sub);
      for (int i = 0; i < D; ++i) rho[i] += rho_sub[i];
      if (dir > 0)
        right = edge;
      else
        left = edge;
      ++depth;
      if (!no_uturn(rho, left.r, right.r)) break;
    }
    cur = prop;
    if (st) {
      st->accept_sum += n_leaf > 0 ? acc / n_leaf : 0.0;
      st->depth_sum += depth;
      st->n_leapfrog += n_leaf;
      st->n_divergent += divergent ? 1 : 0;
    }
  }
};

// Cholesky of the metric; falls back to its diagonal when not positive definite.
static void set_metric(Sampler& s, const double* inv_mass) {
  int D = s.D;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) s.minv[i][j] = inv_mass ? inv_mass[i * D + j] : (i == j ? 1.0 : 0.0);
  bool ok = true;
  for (int j = 0; j < D && ok; ++j) {
    for (int i = 0; i < D; ++i) s.chol[i][j] = 0.0;
    double d = s.minv[j][j];
    for (int k = 0; k < j; ++k) d -= s.chol[j][k] * s.chol[j][k];
    if (!(d > 0.0) || !std::isfinite(d)) {
      ok = false;
      break;
    }
    s.chol[j][j] = std::sqrt(d);
    for (int i = j + 1; i < D; ++i) {
      double t = s.minv[i][j];
      for (int k = 0; k < j; ++k) t -= s.chol[i][k] * s.chol[j][k];
      s.chol[i][j] = t / s.chol[j][j];
    }
  }
  if (!ok) {
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        double dii = s.minv[i][i] > 0.0 && std::isfinite(s.minv[i][i]) ? s.minv[i][i] : 1.0;
        s.minv[i][j] = i == j ? dii : 0.0;
        s.chol[i][j] = i == j ? std::sqrt(dii) : 0.0;
      }
  }
}

}  // namespace oracle

using namespace oracle;

extern "C" {

int ref_nuts_mutate_ids(const ref_model* m, const ref_event* ev, int64_t n, const int64_t* ids, double beta,
                        double* theta, double* lnl, double* grad, const double* inv_mass, double step,
                        int max_depth, int n_steps, uint64_t key, uint32_t ctr, ref_nuts_stats* stats) {
  if (max_depth < 0 || max_depth > kMaxDepth) return -1;
  if (ids)
    for (int64_t i = 0; i < n; ++i)
      if (ids[i] < 0 || ids[i] > 0xffffffffLL) return -1;
  Sampler s;
  s.m = m;
  s.ev = ev;
  s.D = m->n_dim;
  s.beta = beta;
  set_metric(s, inv_mass);
  int D = s.D;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    // the transition's random numbers are named by the particle's index in
    // the ensemble, so any subset can be run on its own
    const uint32_t pid = (uint32_t)(ids ? ids[i] : i);
    Point cur;
    for (int j = 0; j < D; ++j) cur.th[j] = theta[i * D + j];
    s.evaluate(cur);  // U and grad U at the current position (ln L recomputed: plain)
    ref_nuts_stats st = {0.0, 0, 0, 0};
    for (int t = 0; t < n_steps; ++t)
      s.transition(cur, key, pid, ctr + (uint32_t)t, step, max_depth, &st);
    for (int j = 0; j < D; ++j) {
      theta[i * D + j] = cur.th[j];
      grad[i * D + j] = cur.gl[j];
    }
    lnl[i] = cur.lnl;
    if (stats) stats[i] = st;
  }
  return 0;
}

int ref_nuts_mutate(const ref_model* m, const ref_event* ev, int64_t n, double beta, double* theta,
                    double* lnl, double* grad, const double* inv_mass, double step, int max_depth,
                    int n_steps, uint64_t key, uint32_t ctr, ref_nuts_stats* stats) {
  return ref_nuts_mutate_ids(m, ev, n, nullptr, beta, theta, lnl, grad, inv_mass, step, max_depth, n_steps, key,
                             ctr, stats);
}

// As ref_nuts_mutate_ids, each particle with its own inverse mass matrix
// (inv_mass [N][D][D]): the local metric of Sec. 5, fixed through the call.
int ref_nuts_mutate_local_ids(const ref_model* m, const ref_event* ev, int64_t n, const int64_t* ids,
                              double beta, double* theta, double* lnl, double* grad, const double* inv_mass,
                              double step, int max_depth, int n_steps, uint64_t key, uint32_t ctr,
                              ref_nuts_stats* stats) {
  if (max_depth < 0 || max_depth > kMaxDepth || !inv_mass) return -1;
  if (ids)
    for (int64_t i = 0; i < n; ++i)
      if (ids[i] < 0 || ids[i] > 0xffffffffLL) return -1;
  Sampler s;
  s.m = m;
  s.ev = ev;
  s.D = m->n_dim;
  s.beta = beta;
  const int D = s.D;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) {
    Sampler sp = s;
    set_metric(sp, inv_mass + i * D * D);
    Point cur;
    for (int j = 0; j < D; ++j) cur.th[j] = theta[i * D + j];
    sp.evaluate(cur);
    ref_nuts_stats st = {0.0, 0, 0, 0};
    const uint32_t pid = (uint32_t)(ids ? ids[i] : i);
    for (int t = 0; t < n_steps; ++t)
      sp.transition(cur, key, pid, ctr + (uint32_t)t, step, max_depth, &st);
    for (int j = 0; j < D; ++j) {
      theta[i * D + j] = cur.th[j];
      grad[i * D + j] = cur.gl[j];
    }
    lnl[i] = cur.lnl;
    if (stats) stats[i] = st;
  }
  return 0;
}

int ref_nuts_mutate_local(const ref_model* m, const ref_event* ev, int64_t n, double beta, double* theta,
                          double* lnl, double* grad, const double* inv_mass, double step, int max_depth,
                          int n_steps, uint64_t key, uint32_t ctr, ref_nuts_stats* stats) {
  return ref_nuts_mutate_local_ids(m, ev, n, nullptr, beta, theta, lnl, grad, inv_mass, step, max_depth, n_steps,
                                   key, ctr, stats);
}

// Inverse of a symmetric positive-definite matrix through its Cholesky
// factor (in place; the diagonal if the factorisation fails).
static void spd_inverse(int D, double* a) {
  std::vector<double> c(a, a + D * D), ci(D * D, 0.0);
  bool ok = true;
  for (int j = 0; j < D && ok; ++j) {
    double d = c[j * D + j];
    for (int k = 0; k < j; ++k) d -= c[j * D + k] * c[j * D + k];
    if (!(d > 0.0) || !std::isfinite(d)) {
      ok = false;
      break;
    }
    c[j * D + j] = std::sqrt(d);
    for (int i = j + 1; i < D; ++i) {
      double t = c[i * D + j];
      for (int k = 0; k < j; ++k) t -= c[i * D + k] * c[j * D + k];
      c[i * D + j] = t / c[j * D + j];
    }
  }
  if (!ok) {
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) a[i * D + j] = i == j ? 1.0 / a[i * D + i] : 0.0;
    return;
  }
  for (int j = 0; j < D; ++j) {  // C^-1 column by column (forward substitution)
    ci[j * D + j] = 1.0 / c[j * D + j];
    for (int i = j + 1; i < D; ++i) {
      double t = 0.0;
      for (int k = j; k < i; ++k) t -= c[i * D + k] * ci[k * D + j];
      ci[i * D + j] = t / c[i * D + i];
    }
  }
  for (int i = 0; i < D; ++i)  // M^-1 = C^-T C^-1
    for (int j = 0; j < D; ++j) {
      double t = 0.0;
      for (int k = (i > j ? i : j); k < D; ++k) t += ci[k * D + i] * ci[k * D + j];
      a[i * D + j] = t;
    }
}

// Eq. (5)-(6): ESS of w_i = exp(dbeta (lnL_i - max)); bisection on dbeta.
static double ess_at(int64_t n, const double* x, double db) {
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double w = x[i] == -INFINITY ? 0.0 : std::exp(db * x[i]);
    s1 += w;
    s2 += w * w;
  }
  return s1 * s1 / s2;
}

int ref_smc_reweight(int64_t n, const double* lnl, double beta_prev, double alpha, double* beta_next,
                     double* dlnz, double* ess, double* w) {
  if (n <= 0) return -1;
  std::vector<double> x(n);
  double mx = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (lnl[i] > mx) mx = lnl[i];
  if (!std::isfinite(mx)) return -1;
  for (int64_t i = 0; i < n; ++i) x[i] = std::isfinite(lnl[i]) ? lnl[i] - mx : -INFINITY;
  double target = alpha * (double)n;
  double hi = 1.0 - beta_prev;
  double db;
  if (hi <= 0.0) {
    db = 0.0;
    *beta_next = 1.0;
  } else if (ess_at(n, x.data(), hi) >= target) {
    db = hi;
    *beta_next = 1.0;
  } else {
    double lo = 0.0;
    for (int it = 0; it < 100; ++it) {
      double mid = 0.5 * (lo + hi);
      if (ess_at(n, x.data(), mid) >= target)
        lo = mid;
      else
        hi = mid;
    }
    db = lo;
    *beta_next = beta_prev + db;
  }
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    w[i] = x[i] == -INFINITY ? 0.0 : std::exp(db * x[i]);
    s1 += w[i];
    s2 += w[i] * w[i];
  }
  *ess = s1 * s1 / s2;
  *dlnz = db * mx + std::log(s1) - std::log((double)n);
  return 0;
}

// q_i = floor(W_i 2^32); C = inclusive prefix sums; U = floor(u 2^32);
// p_m = floor((m 2^32 + U) C_N / (N 2^32)); ancestor(m) = min{ j : C_j > p_m }.
int ref_systematic_resample(int64_t n, const double* w, double u, int32_t* anc) {
  if (n <= 0 || !(u >= 0.0 && u < 1.0)) return -1;
  std::vector<uint64_t> c(n);
  uint64_t run = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!(w[i] >= 0.0 && w[i] <= 1.0)) return -1;
    run += (uint64_t)std::floor(w[i] * 4294967296.0);
    c[i] = run;
  }
  if (run == 0) return -1;
  uint64_t U = (uint64_t)std::floor(u * 4294967296.0);
  unsigned __int128 den = (unsigned __int128)n << 32;
  for (int64_t mm = 0; mm < n; ++mm) {
    unsigned __int128 x = ((unsigned __int128)mm << 32) + U;
    uint64_t p = (uint64_t)((x * run) / den);
    int64_t j = 0;
    while (!(c[j] > p)) ++j;  // linear scan: plain
    anc[mm] = (int32_t)j;
  }
  return 0;
}

int ref_weighted_cov(int d, int64_t n, const double* theta, const double* w, double* cov) {
  double sw = 0.0;
  double mu[REF_MAX_DIM] = {0};
  for (int64_t i = 0; i < n; ++i) {
    sw += w[i];
    for (int a = 0; a < d; ++a) mu[a] += w[i] * theta[i * d + a];
  }
  for (int a = 0; a < d; ++a) mu[a] /= sw;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) {
      double s = 0.0;
      for (int64_t i = 0; i < n; ++i) s += w[i] * (theta[i * d + a] - mu[a]) * (theta[i * d + b] - mu[b]);
      cov[a * d + b] = s / sw;
    }
  return 0;
}

int ref_smc_run(const ref_model* m, const ref_event* ev, const ref_smc_opts* o, uint64_t key, double* lnz,
                int* n_stages, double* theta_out, double* lnl_out, ref_stage* stages) {
  int64_t n = o->n_particles;
  int D = m->n_dim;
  std::vector<double> th(n * D), th2(n * D), l(n), l2(n), g(n * D), g2(n * D), w(n), cov(D * D);
  std::vector<int32_t> anc(n);
  std::vector<ref_nuts_stats> st(n);
  ref_prior_sample(m, n, th.data(), key, 0u);
  ref_loglike(m, ev, n, th.data(), l.data(), g.data());
  double beta = 0.0, z = 0.0;
  int t = 0;
  while (beta < 1.0 && t < o->max_stages) {
    ++t;
    double bn, dl, ess;
    ref_smc_reweight(n, l.data(), beta, o->alpha, &bn, &dl, &ess, w.data());
    z += dl;
    ref_weighted_cov(D, n, th.data(), w.data(), cov.data());
    double u[2];
    uniform2(key, 0u, (uint32_t)t, P_RESAMPLE, 0u, u);
    ref_systematic_resample(n, w.data(), u[0], anc.data());
    for (int64_t i = 0; i < n; ++i) {
      int64_t a = anc[i];
      for (int j = 0; j < D; ++j) {
        th2[i * D + j] = th[a * D + j];
        g2[i * D + j] = g[a * D + j];
      }
      l2[i] = l[a];
    }
    th.swap(th2);
    g.swap(g2);
    l.swap(l2);
    double eps;
    const double* minv = nullptr;
    if (o->metric == 1 || o->metric == 2) {
      eps = o->eps_scale;
      minv = cov.data();
    } else {
      double smin = INFINITY;
      for (int j = 0; j < D; ++j) smin = std::fmin(smin, std::sqrt(cov[j * D + j]));
      eps = o->eps_scale * smin;
    }
    if (o->metric == 2) {
      // local metric of each resampled particle at the new temperature (Sec. 5)
      std::vector<double> pm((size_t)n * D * D);
      ref_local_metric(m, ev, n, th.data(), bn, pm.data());
      for (int64_t i = 0; i < n; ++i) spd_inverse(D, pm.data() + i * D * D);
      ref_nuts_mutate_local(m, ev, n, bn, th.data(), l.data(), g.data(), pm.data(), eps, o->max_depth, o->n_mut,
                            key, (uint32_t)t << 8, st.data());
    } else {
      ref_nuts_mutate(m, ev, n, bn, th.data(), l.data(), g.data(), minv, eps, o->max_depth, o->n_mut, key,
                      (uint32_t)t << 8, st.data());
    }
    if (stages) {
      ref_stage& s = stages[t - 1];
      s.beta = bn;
      s.dbeta = bn - beta;
      s.ess = ess;
      s.dlnz = dl;
      s.eps = eps;
      double a = 0.0, dsum = 0.0;
      int64_t lf = 0;
      int dv = 0;
      for (int64_t i = 0; i < n; ++i) {
        a += st[i].accept_sum;
        dsum += st[i].depth_sum;
        lf += st[i].n_leapfrog;
        dv += st[i].n_divergent;
      }
      s.accept_mean = a / (double)(n * o->n_mut);
      s.depth_mean = dsum / (double)(n * o->n_mut);
      s.n_leapfrog = lf;
      s.n_divergent = dv;
    }
    beta = bn;
  }
  *lnz = z;
  *n_stages = t;
  if (theta_out) std::memcpy(theta_out, th.data(), sizeof(double) * n * D);
  if (lnl_out) std::memcpy(lnl_out, l.data(), sizeof(double) * n);
  return beta >= 1.0 ? 0 : 1;
}

// The inverse mass matrices ref_smc_run's metric 2 mutates with: the local
// metric of each particle at beta, each inverted by spd_inverse.
int ref_local_inv_mass(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double beta,
                       double* inv_mass) {
  const int rc = ref_local_metric(m, ev, n, theta, beta, inv_mass);
  if (rc) return rc;
  const int D = m->n_dim;
  for (int64_t i = 0; i < n; ++i) spd_inverse(D, inv_mass + i * D * D);
  return 0;
}

}  // extern "C"

// Sample recycling (Sec. 5): mixture weights of the pooled particles for the
// final target, then rejection sampling to i.i.d. draws.
int ref_recycle_weights(int64_t m, int t, const double* lnl, const double* beta, const double* lnz_t,
                        double* log_w) {
  if (m < 0 || t < 1) return -1;
  const double lnz_final = lnz_t[t - 1];
  for (int64_t i = 0; i < m; ++i) {
    // ln sum_t exp(beta_t ln L_i - ln Z_t), with its largest term factored out
    double mx = -INFINITY;
    for (int s = 0; s < t; ++s) mx = std::fmax(mx, beta[s] * lnl[i] - lnz_t[s]);
    double acc = 0.0;
    for (int s = 0; s < t; ++s) acc += std::exp(beta[s] * lnl[i] - lnz_t[s] - mx);
    const double ln_mix = mx + std::log(acc) - std::log((double)t);
    log_w[i] = lnl[i] - lnz_final - ln_mix;
  }
  return 0;
}

int ref_rejection_sample(int64_t m, const double* log_w, uint64_t key, int32_t* keep) {
  if (m < 0) return -1;
  double mx = -INFINITY;
  for (int64_t i = 0; i < m; ++i) mx = std::fmax(mx, log_w[i]);
  for (int64_t i = 0; i < m; ++i) {
    double u[2];
    ref_uniform2(key, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), 7u, 0u, u);
    keep[i] = (u[0] < std::exp(log_w[i] - mx)) ? 1 : 0;
  }
  return 0;
}
