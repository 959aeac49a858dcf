// Persistent multinomial NUTS (Sec. 4; Hoffman & Gelman 2014, multinomial
// variant with biased progressive sampling at the top level and the
// generalised U-turn criterion on every completed sub-tree).
//
// One CTA of kNutsWarps warps owns SLOTS (8, 16 or 32) particles for the whole
// call; SLOTS is chosen from N so that the CTAs about fill the GPU in one wave
// while warp 0's per-particle phase runs on as many lanes as possible (an FP64
// warp instruction costs the same pipe time whatever its active-lane count).
// Lane s of warp 0 runs the NUTS state machine of slot s: the trajectory is grown one
// leapfrog at a time (iteratively, no recursion), and every leapfrog needs one
// likelihood+gradient evaluation. Each "tick" of the CTA: warp 0 computes the
// prologue of every pending evaluation (lane-parallel), each warp sweeps the
// bins of one pending particle, warp 0 runs the epilogues and advances the
// state machines to their next evaluation. Particles with shallow trees finish
// early and leave their lane idle; the tree state of every slot lives in shared
// memory ([field][dim][slot], conflict-free across lanes).
//
// Leaf order and random draws (Philox4x32-10, counter = (particle, step,
// purpose, index)): per transition the momentum (purpose 2, one normal pair
// per index), per doubling j the direction (purpose 3, index j) and the
// top-level acceptance (purpose 5, index j), per leaf the in-subtree
// progressive acceptance (purpose 4, running leaf index).
#pragma once
#include <cmath>

#include "context.cuh"
#include "sweep.cuh"

namespace sharpy {

constexpr int kNutsWarps = 8;
constexpr int kMaxDepth = SHARPY_MAX_DEPTH;
constexpr double kDivergence = 1000.0;

// Shared-memory vector fields of the tree state.
enum {
  F_LTH, F_LR, F_LGU, F_LV,  // left end: theta, momentum, grad U, velocity Minv r
  F_RTH, F_RR, F_RGU, F_RV,  // right end
  F_PTH, F_PGL,              // proposal (also the current point between transitions)
  F_STH, F_SGL,              // sub-tree proposal
  F_RHO, F_RHOS,             // momentum sums: whole tree, current sub-tree
  F_NTH, F_NR,               // pending leaf: position, half-step momentum
  F_RS0,                     // rho_start[1..kMaxDepth]
  F_RF0 = F_RS0 + kMaxDepth, // velocity of the first leaf of each open block [1..kMaxDepth]
  F_COUNT = F_RF0 + kMaxDepth
};

struct NutsArgs {
  DevModel m;
  DevEvent ev;
  int64_t n;
  double* theta;
  double* lnl;
  double* grad;
  const double* beta_ptr;
  double beta;
  const double* minv;      // [D][D] or null
  const double* cov_step;  // identity metric with step = eps_scale * min sqrt(diag cov)
  double step;
  int max_depth;
  int n_steps;
  uint64_t key;
  uint32_t ctr;
  sharpy_nuts_stats* stats;
  int* status;
};

enum { METRIC_IDENTITY = 0, METRIC_DIAGONAL = 1, METRIC_DENSE = 2 };

template <int SLOTS>
struct NutsShared {
  double vec[F_COUNT][kMaxDim][SLOTS];
  double minv[kMaxDim][kMaxDim];
  double chol[kMaxDim][kMaxDim];
  double eps, beta;
  double lp_const;  // sum of the prior's constant log terms
  int metric_kind;
  int alive;
  int pending[SLOTS];
};

__device__ __forceinline__ double logaddexp(double a, double b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  double mx = fmax(a, b);
  return mx + log(exp(a - mx) + exp(b - mx));
}

// Per-slot state machine (registers of lane s of warp 0).
struct Slot {
  int64_t pid;
  int t;           // transition index
  int depth;       // completed doublings
  long n;          // leaf index within the current sub-tree
  int dir;
  uint32_t leaf_ctr;
  double h0, logw, logw_sub, lnl_p, lnl_s, acc;
  int n_leaf, divergent;
  int done;
  double u_cur, lnl_new;
  // stats
  double st_acc, st_bins;
  int st_depth, st_leap, st_div;
};

template <int PREC, int NDET, int SLOTS>
struct Nuts {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  const NutsArgs& A;
  NutsShared<SLOTS>& S;
  int s;  // slot
  int D;
  __device__ Nuts(const NutsArgs& a, NutsShared<SLOTS>& sh, int slot) : A(a), S(sh), s(slot), D(a.m.n_dim) {}
  __device__ double& V(int f, int d) { return S.vec[f][d][s]; }

  // v = Minv r for the momentum stored in field f
  __device__ void velocity(int f, double* v) {
    if (S.metric_kind == METRIC_IDENTITY) {
      for (int i = 0; i < D; ++i) v[i] = V(f, i);
    } else if (S.metric_kind == METRIC_DIAGONAL) {
      for (int i = 0; i < D; ++i) v[i] = S.minv[i][i] * V(f, i);
    } else {
      for (int i = 0; i < D; ++i) {
        double acc = 0.0;
        for (int j = 0; j < D; ++j) acc += S.minv[i][j] * V(f, j);
        v[i] = acc;
      }
    }
  }
  __device__ double dot(const double* a, int f) {
    double k = 0.0;
    for (int i = 0; i < D; ++i) k += a[i] * V(f, i);
    return k;
  }
  __device__ double dotv(const double* a, const double* b) {
    double k = 0.0;
    for (int i = 0; i < D; ++i) k += a[i] * b[i];
    return k;
  }
  // ln pi and grad ln pi with the constant terms precomputed
  __device__ double prior(const double* x, double* g) {
    const DevModel& m = A.m;
    double lp = S.lp_const;
    bool inside = true;
    for (int i = 0; i < D; ++i) {
      g[i] = 0.0;
      if (!(x[i] >= m.lo[i] && x[i] <= m.hi[i])) inside = false;
      if (m.prior[i] == SHARPY_PRIOR_POWER2) {
        lp += 2.0 * log(x[i]);
        g[i] = 2.0 / x[i];
      }
    }
    return inside ? lp : -INFINITY;
  }

  // Boundary maps on the pending leaf (F_NTH, F_NR). False if not finite.
  __device__ bool boundary() {
    const DevModel& m = A.m;
    for (int i = 0; i < D; ++i) {
      double x = V(F_NTH, i);
      if (!isfinite(x)) return false;
      double lo = m.lo[i], hi = m.hi[i];
      if (m.boundary[i] == SHARPY_BOUND_PERIODIC) {
        // lo + ((x - lo) mod w): for |x - lo| < 2w one exact subtraction or
        // addition gives fmod's result; fmod only for larger excursions
        const double w = hi - lo;
        double t = x - lo;
        if (t >= w)
          t = t < 2.0 * w ? t - w : fmod(t, w);
        else if (t < 0.0)
          t = t >= -w ? t : fmod(t, w);
        if (t < 0.0) t += w;
        V(F_NTH, i) = lo + t;
      } else {
        int flips = 0;
        while ((x < lo || x > hi) && flips < 100) {
          x = x < lo ? 2.0 * lo - x : 2.0 * hi - x;
          ++flips;
        }
        if (x < lo || x > hi) return false;
        V(F_NTH, i) = x;
        if (flips & 1) {
          double v[kMaxDim];
          velocity(F_NR, v);
          V(F_NR, i) = V(F_NR, i) - 2.0 * v[i] / S.minv[i][i];
        }
      }
    }
    return true;
  }

  // First half of a leapfrog from the end of the tree in direction dir.
  __device__ bool begin_leapfrog(int dir) {
    const int fth = dir > 0 ? F_RTH : F_LTH, fr = dir > 0 ? F_RR : F_LR, fgu = dir > 0 ? F_RGU : F_LGU;
    const double h = dir * S.eps;
    for (int i = 0; i < D; ++i) V(F_NR, i) = V(fr, i) - 0.5 * h * V(fgu, i);
    double v[kMaxDim];
    velocity(F_NR, v);
    for (int i = 0; i < D; ++i) V(F_NTH, i) = V(fth, i) + h * v[i];
    return boundary();
  }

  __device__ void draw_direction(Slot& sl) {
    double u0, u1;
    uniform2(A.key, (uint32_t)sl.pid, A.ctr + (uint32_t)sl.t, RNG_DIRECTION, (uint32_t)sl.depth, &u0, &u1);
    sl.dir = u0 < 0.5 ? -1 : 1;
    sl.n = 0;
    sl.logw_sub = -INFINITY;
    for (int i = 0; i < D; ++i) V(F_RHOS, i) = 0.0;
  }

  // Start transition sl.t from the current point (F_PTH, F_PGL, lnl_p).
  __device__ void start_transition(Slot& sl) {
    const uint32_t step = A.ctr + (uint32_t)sl.t;
    double z[kMaxDim + 1];
    for (int p = 0; 2 * p < D; ++p) {
      double u0, u1;
      uniform2(A.key, (uint32_t)sl.pid, step, RNG_MOMENTUM, (uint32_t)p, &u0, &u1);
      double r = sqrt(-2.0 * log(u0));
      double sn, cs;
      sincospi(2.0 * u1, &sn, &cs);
      z[2 * p] = r * cs;
      z[2 * p + 1] = r * sn;
    }
    // r ~ N(0, M), M = Minv^{-1} = (L L^T)^{-1}: solve L^T r = z
    for (int i = D - 1; i >= 0; --i) {
      double acc = z[i];
      for (int j = i + 1; j < D; ++j) acc -= S.chol[j][i] * V(F_LR, j);
      V(F_LR, i) = acc / S.chol[i][i];
    }
    // U and grad U at the current point
    double x[kMaxDim], glp[kMaxDim], v0[kMaxDim];
    for (int i = 0; i < D; ++i) x[i] = V(F_PTH, i);
    double lp = prior(x, glp);
    sl.u_cur = -S.beta * sl.lnl_p - lp;
    velocity(F_LR, v0);
    for (int i = 0; i < D; ++i) {
      V(F_LTH, i) = x[i];
      V(F_LGU, i) = -S.beta * V(F_PGL, i) - glp[i];
      V(F_LV, i) = v0[i];
      V(F_RTH, i) = x[i];
      V(F_RR, i) = V(F_LR, i);
      V(F_RGU, i) = V(F_LGU, i);
      V(F_RV, i) = v0[i];
      V(F_RHO, i) = V(F_LR, i);
    }
    sl.h0 = sl.u_cur + 0.5 * dot(v0, F_LR);
    sl.logw = 0.0;
    sl.depth = 0;
    sl.leaf_ctr = 0;
    sl.acc = 0.0;
    sl.n_leaf = 0;
    sl.divergent = 0;
  }

  __device__ void end_transition(Slot& sl) {
    sl.st_acc += sl.n_leaf > 0 ? sl.acc / sl.n_leaf : 0.0;
    sl.st_depth += sl.depth;
    sl.st_leap += sl.n_leaf;
    sl.st_div += sl.divergent;
    sl.t += 1;
  }

  // Advance until the next evaluation is pending (true) or the slot is done.
  // `have_leaf` : a leaf evaluation just finished (F_NTH/F_NR hold the leaf with
  // full-step momentum, gl in F_SGL? no: passed in), process it first.
  __device__ bool advance(Slot& sl, bool have_leaf, const double* gl_new, double lp_new, const double* glp_new) {
    if (have_leaf) {
      // complete the leapfrog
      const double h = sl.dir * S.eps;
      double gu[kMaxDim];
      for (int i = 0; i < D; ++i) {
        gu[i] = -S.beta * gl_new[i] - glp_new[i];
        V(F_NR, i) = V(F_NR, i) - 0.5 * h * gu[i];
      }
      double u_new = -S.beta * sl.lnl_new - lp_new;
      double vn[kMaxDim];
      velocity(F_NR, vn);
      double dH = u_new + 0.5 * dot(vn, F_NR) - sl.h0;
      sl.n_leaf += 1;
      sl.acc += (dH == dH) ? fmin(1.0, exp(-dH)) : 0.0;
      if (!(dH <= kDivergence)) {
        sl.divergent = 1;
        end_transition(sl);
        goto next_transition;
      }
      {
        // the leaf becomes the end of the tree in direction dir
        const int fth = sl.dir > 0 ? F_RTH : F_LTH, fr = sl.dir > 0 ? F_RR : F_LR, fgu = sl.dir > 0 ? F_RGU : F_LGU;
        const int fv = sl.dir > 0 ? F_RV : F_LV;
        for (int i = 0; i < D; ++i) {
          V(fth, i) = V(F_NTH, i);
          V(fr, i) = V(F_NR, i);
          V(fgu, i) = gu[i];
          V(fv, i) = vn[i];
        }
        double lw = -dH;
        double lw_new = logaddexp(sl.logw_sub, lw);
        double u0, u1;
        uniform2(A.key, (uint32_t)sl.pid, A.ctr + (uint32_t)sl.t, RNG_LEAF, sl.leaf_ctr++, &u0, &u1);
        if (u0 < exp(lw - lw_new)) {
          for (int i = 0; i < D; ++i) {
            V(F_STH, i) = V(F_NTH, i);
            V(F_SGL, i) = gl_new[i];
          }
          sl.lnl_s = sl.lnl_new;
        }
        sl.logw_sub = lw_new;
        for (int lvl = 1; lvl <= sl.depth; ++lvl)
          if ((sl.n & ((1L << lvl) - 1)) == 0)
            for (int i = 0; i < D; ++i) {
              V(F_RS0 + lvl - 1, i) = V(F_RHOS, i);
              V(F_RF0 + lvl - 1, i) = vn[i];
            }
        for (int i = 0; i < D; ++i) V(F_RHOS, i) += V(F_NR, i);
        bool ok = true;
        for (int lvl = 1; lvl <= sl.depth && ok; ++lvl)
          if (((sl.n + 1) & ((1L << lvl) - 1)) == 0) {
            double rb[kMaxDim];
            for (int i = 0; i < D; ++i) rb[i] = V(F_RHOS, i) - V(F_RS0 + lvl - 1, i);
            if (!(dot(rb, F_RF0 + lvl - 1) > 0.0 && dotv(rb, vn) > 0.0)) ok = false;
          }
        if (!ok) {
          end_transition(sl);
          goto next_transition;
        }
        sl.n += 1;
        if (sl.n < (1L << sl.depth)) {
          if (begin_leapfrog(sl.dir)) return true;
          sl.n_leaf += 1;
          sl.divergent = 1;
          end_transition(sl);
          goto next_transition;
        }
        // sub-tree complete: biased progressive sampling at the top level
        uniform2(A.key, (uint32_t)sl.pid, A.ctr + (uint32_t)sl.t, RNG_TOP, (uint32_t)sl.depth, &u0, &u1);
        if (u0 < exp(sl.logw_sub - sl.logw)) {
          for (int i = 0; i < D; ++i) {
            V(F_PTH, i) = V(F_STH, i);
            V(F_PGL, i) = V(F_SGL, i);
          }
          sl.lnl_p = sl.lnl_s;
        }
        sl.logw = logaddexp(sl.logw, sl.logw_sub);
        double rho[kMaxDim];
        for (int i = 0; i < D; ++i) {
          V(F_RHO, i) += V(F_RHOS, i);
          rho[i] = V(F_RHO, i);
        }
        sl.depth += 1;
        if (!(dot(rho, F_LV) > 0.0 && dot(rho, F_RV) > 0.0) || sl.depth >= A.max_depth) {
          end_transition(sl);
          goto next_transition;
        }
        draw_direction(sl);
        if (begin_leapfrog(sl.dir)) return true;
        sl.n_leaf += 1;
        sl.divergent = 1;
        end_transition(sl);
      }
    }
  next_transition:
    while (sl.t < A.n_steps) {
      start_transition(sl);
      if (A.max_depth <= 0) {
        end_transition(sl);
        continue;
      }
      draw_direction(sl);
      if (begin_leapfrog(sl.dir)) return true;
      sl.n_leaf += 1;
      sl.divergent = 1;
      end_transition(sl);
    }
    sl.done = 1;
    return false;
  }
};

template <int PREC, int NDET, int SLOTS>
struct NutsSmem {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  using MT = typename MomType<PREC>::type;
  NutsShared<SLOTS> S;
  SweepCoef sc[SLOTS];
  EpiCoef<DT> ec[SLOTS];
  MT mom[SLOTS][NDET * kNMom * 2];
};

// Eight slots: registers capped for two CTAs per SM; wider CTAs run one per SM.
template <int SLOTS>
struct NutsMinBlocks {
  static constexpr int value = SLOTS == 8 ? 2 : 1;
};

template <int PREC, int NDET, int SLOTS>
__global__ void __launch_bounds__(kNutsWarps * 32, NutsMinBlocks<SLOTS>::value) nuts_kernel(NutsArgs A) {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  using MT = typename MomType<PREC>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NutsSmem<PREC, NDET, SLOTS>& SM = *reinterpret_cast<NutsSmem<PREC, NDET, SLOTS>*>(smem_raw);
  NutsShared<SLOTS>& S = SM.S;
  SweepCoef* sc = SM.sc;
  EpiCoef<DT>* ec = SM.ec;
  auto& mom = SM.mom;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int D = A.m.n_dim;
  const bool gw = A.m.model == SHARPY_MODEL_TAYLORF2;

  // metric, its Cholesky factor (diagonal fallback), step size, beta
  if (threadIdx.x == 0) {
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) S.minv[i][j] = A.minv ? A.minv[i * D + j] : (i == j ? 1.0 : 0.0);
    bool ok = true;
    for (int j = 0; j < D && ok; ++j) {
      for (int i = 0; i < D; ++i) S.chol[i][j] = 0.0;
      double d = S.minv[j][j];
      for (int k = 0; k < j; ++k) d -= S.chol[j][k] * S.chol[j][k];
      if (!(d > 0.0) || !isfinite(d)) {
        ok = false;
        break;
      }
      S.chol[j][j] = sqrt(d);
      for (int i = j + 1; i < D; ++i) {
        double t = S.minv[i][j];
        for (int k = 0; k < j; ++k) t -= S.chol[i][k] * S.chol[j][k];
        S.chol[i][j] = t / S.chol[j][j];
      }
    }
    if (!ok)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double dii = S.minv[i][i] > 0.0 && isfinite(S.minv[i][i]) ? S.minv[i][i] : 1.0;
          S.minv[i][j] = i == j ? dii : 0.0;
          S.chol[i][j] = i == j ? sqrt(dii) : 0.0;
        }
    bool ident = true, diag = true;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        if (i != j && S.minv[i][j] != 0.0) diag = false;
        if (S.minv[i][j] != (i == j ? 1.0 : 0.0)) ident = false;
      }
    S.metric_kind = ident ? METRIC_IDENTITY : (diag ? METRIC_DIAGONAL : METRIC_DENSE);
    double lpc = 0.0;
    for (int i = 0; i < D; ++i) {
      double lo = A.m.lo[i], hi = A.m.hi[i];
      lpc += A.m.prior[i] == SHARPY_PRIOR_POWER2 ? log(3.0 / (hi * hi * hi - lo * lo * lo)) : -log(hi - lo);
    }
    S.lp_const = lpc;
    double eps = A.step;
    if (A.cov_step) {
      double smin = INFINITY;
      for (int j = 0; j < D; ++j) smin = fmin(smin, sqrt(A.cov_step[j * D + j]));
      eps = A.step * smin;
    }
    S.eps = eps;
    S.beta = A.beta_ptr ? *A.beta_ptr : A.beta;
  }
  __syncthreads();

  Slot sl;
  bool active = false;
  if (warp == 0 && lane < SLOTS) {
    Nuts<PREC, NDET, SLOTS> nu(A, S, lane);
    sl.pid = (int64_t)blockIdx.x * SLOTS + lane;
    sl.t = 0;
    sl.done = 1;
    sl.st_acc = sl.st_bins = 0.0;
    sl.st_depth = sl.st_leap = sl.st_div = 0;
    if (sl.pid < A.n) {
      for (int i = 0; i < D; ++i) {
        nu.V(F_PTH, i) = A.theta[sl.pid * D + i];
        nu.V(F_PGL, i) = A.grad[sl.pid * D + i];
      }
      sl.lnl_p = A.lnl[sl.pid];
      sl.done = 0;
      active = nu.advance(sl, false, nullptr, 0.0, nullptr);
    }
    S.pending[lane] = active ? 1 : 0;
  }
  const long max_ticks = (long)A.n_steps * ((1L << A.max_depth) + 1) + 4;
  for (long tick = 0;; ++tick) {
    // warp 0: any pending evaluation left?
    if (warp == 0) {
      unsigned any = __ballot_sync(0xffffffffu, lane < SLOTS && S.pending[lane]);
      if (lane == 0) S.alive = any != 0u;
      if (tick > max_ticks && any) {
        if (lane == 0) set_status(A.status, SHARPY_ETIMEOUT);
        if (lane < SLOTS) S.pending[lane] = 0;
        if (lane == 0) S.alive = 0;
      }
    }
    __syncthreads();
    if (!S.alive) break;
    // (A) prologues (GW) or direct evaluations (Gaussian mixture)
    double gl_new[kMaxDim], glp_new[kMaxDim], lp_new = 0.0;
    if (warp == 0 && lane < SLOTS && S.pending[lane]) {
      Nuts<PREC, NDET, SLOTS> nu(A, S, lane);
      double x[kMaxDim];
      for (int i = 0; i < D; ++i) x[i] = nu.V(F_NTH, i);
      if (gw)
        prologue<DT, true, PREC == SHARPY_MIXED_SPLIT>(A.m, A.ev, x, sc[lane], ec[lane]);
      else
        gaussmix(A.m, x, &sl.lnl_new, gl_new);
    }
    __syncthreads();
    // (B) sweeps: warp w sweeps slot w
    if (gw) {
      for (int slot = warp; slot < SLOTS; slot += kNutsWarps) {
        MT* mw = mom[slot];
        for (int i = lane; i < NDET * kNMom * 2; i += 32) mw[i] = MT(0);
        __syncwarp();
        if (S.pending[slot] && sc[slot].ok) sweep<PREC, true, NDET>(A.ev, sc[slot], mw);
      }
    }
    __syncthreads();
    // (C) epilogues and state machines
    if (warp == 0 && lane < SLOTS && S.pending[lane]) {
      Nuts<PREC, NDET, SLOTS> nu(A, S, lane);
      double x[kMaxDim];
      for (int i = 0; i < D; ++i) x[i] = nu.V(F_NTH, i);
      if (gw) {
        double gph[SHARPY_NPHYS];
        sl.lnl_new = NAN;
        if (sc[lane].ok) {
          epilogue<DT, true>(A.ev, sc[lane], ec[lane], mom[lane], &sl.lnl_new, gph);
          sl.st_bins += (double)(sc[lane].kisco + 1) * A.ev.n_det;
        }
        for (int i = 0; i < D; ++i) gl_new[i] = sc[lane].ok ? gph[A.m.phys[i]] : NAN;
      }
      lp_new = nu.prior(x, glp_new);
      if (!isfinite(sl.lnl_new)) sl.lnl_new = -INFINITY;  // rejected leaf (U = +inf)
      for (int i = 0; i < D; ++i)
        if (!isfinite(gl_new[i])) gl_new[i] = 0.0;
      bool more = nu.advance(sl, true, gl_new, lp_new, glp_new);
      S.pending[lane] = more ? 1 : 0;
    }
  }
  // write back
  if (warp == 0 && lane < SLOTS && sl.pid < A.n) {
    Nuts<PREC, NDET, SLOTS> nu(A, S, lane);
    for (int i = 0; i < D; ++i) {
      A.theta[sl.pid * D + i] = nu.V(F_PTH, i);
      A.grad[sl.pid * D + i] = nu.V(F_PGL, i);
    }
    A.lnl[sl.pid] = sl.lnl_p;
    if (A.stats) {
      sharpy_nuts_stats st;
      st.accept_sum = sl.st_acc;
      st.active_bins = sl.st_bins;
      st.depth_sum = sl.st_depth;
      st.n_leapfrog = sl.st_leap;
      st.n_divergent = sl.st_div;
      st.pad = 0;
      A.stats[sl.pid] = st;
    }
  }
}


// Launch helper for one (precision, detector count); the slot count is picked
// by the caller. Defined in nuts_inst.cu, compiled once per combination.
int launch_nuts(int precision, int ndet, int slots, const NutsArgs& A, cudaStream_t s);

template <int P, int ND>
int launch_nuts_impl(int slots, const NutsArgs& A, cudaStream_t s) {
  auto go = [&](auto kernel, int sl, size_t bytes) -> int {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return SHARPY_ECUDA;
    dim3 grid((unsigned)((A.n + sl - 1) / sl));
    kernel<<<grid, kNutsWarps * 32, bytes, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
  };
  if (slots == 32) return go(nuts_kernel<P, ND, 32>, 32, sizeof(NutsSmem<P, ND, 32>));
  if (slots == 16) return go(nuts_kernel<P, ND, 16>, 16, sizeof(NutsSmem<P, ND, 16>));
  return go(nuts_kernel<P, ND, 8>, 8, sizeof(NutsSmem<P, ND, 8>));
}

}  // namespace sharpy
