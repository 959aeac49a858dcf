// Persistent multinomial NUTS (Sec. 4; Hoffman & Gelman 2014, multinomial
// variant with biased progressive sampling at the top level and the
// generalised U-turn criterion on every completed sub-tree).
//
// One CTA of kNutsWarps warps owns SLOTS (8, 16 or 32) particles for the
// whole call; the slot count is autotuned (about two CTAs share each SM, so
// their serial per-particle phases overlap with each other's sweeps). Every
// slot's trajectory is grown one leapfrog at a time (iteratively, no
// recursion), and every leapfrog needs one likelihood+gradient evaluation.
// Each "tick" of the CTA has three phases between barriers:
//   A  the prologue of every pending evaluation, lane = slot: the phase half
//      (PN coefficients, k_ISCO; FP64, or double-float on the mixed paths) on
//      the control warp, the sky half (responses, delays, amplitude) on its
//      neighbour, a warp on another SM sub-partition;
//   B  each warp sweeps the bins of the next pending particle, longest first;
//   C  each pending slot's epilogue, tree update and first half of the next
//      leapfrog, on a lane group of 32/(SLOTS/4) lanes (one or more dimensions
//      per lane), the pending slots dealt out one per warp first.
// An FP64 warp instruction costs the same pipe time whatever its active-lane
// count, and a warp runs the union of its lanes' branches of the state
// machine: spreading both over the sub-partitions shortens the serial part of
// a tick. Particles with shallow trees finish early and leave their slot idle;
// the tree state of every slot lives in shared memory ([field][slot][dim]: a
// slot's lane group reads consecutive words).
//
// Precision of the tree state (template VT): positions theta and the potential
// energy are FP64 on every path. The FP64 path keeps momenta, velocities,
// momentum sums, gradients, log-weights and random draws in FP64 too. The
// mixed paths keep those in FP32: a dependent FP64 operation costs ~64 cycles
// on this GPU (FP32: ~4) and an FP64 exp ~1200, and this state machine is a
// serial chain per particle; FP32 resolves the momenta and weights far below
// the mixed likelihood's own error.
//
// Leaf order and random draws (Philox4x32-10, counter = (particle, step,
// purpose, index)): per transition the momentum (purpose 2, one normal pair
// per index), per doubling j the direction (purpose 3, index j) and the
// top-level acceptance (purpose 5, index j), per leaf the in-subtree
// progressive acceptance (purpose 4, running leaf index). FP64 draws use 53
// bits of the first two words; FP32 draws use the top 24 bits of the first.
#pragma once
#include <cmath>

#include "context.cuh"
#include "sweep.cuh"

namespace sharpy {

constexpr int kNutsWarps = 4;  // warps per CTA; two CTAs share an SM so their serial phases interleave
constexpr int kMaxDepth = SHARPY_MAX_DEPTH;
constexpr double kDivergence = 1000.0;

// Position fields (FP64).
enum { P_L, P_R, P_P, P_S, P_N, P_COUNT };  // left end, right end, proposal, sub-tree proposal, pending leaf
// Momentum-like fields (type VT).
enum {
  F_LR, F_LGU, F_LV,          // left end: momentum, grad U, velocity Minv r
  F_RR, F_RGU, F_RV,          // right end
  F_PGL, F_SGL,               // grad ln L of the proposal / sub-tree proposal
  F_RHO, F_RHOS,              // momentum sums: whole tree, current sub-tree
  F_NR,                       // pending leaf: half-step momentum
  F_RS0,                      // rho_start[1..kMaxDepth]
  F_RF0 = F_RS0 + kMaxDepth,  // velocity of the first leaf of each open block [1..kMaxDepth]
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
  const double* pminv;     // [n][D][D] per-particle metric (with pchol), or null
  const double* pchol;
  int local_metric;        // 1: per-particle metric (pminv, pchol); sizes the shared memory
  const double* cov_step;  // identity metric with step = eps_scale * min sqrt(diag cov)
  double step;
  int max_depth;
  int n_steps;
  uint64_t key;
  uint32_t ctr;
  sharpy_nuts_stats* stats;
  int* status;
  int64_t tick_limit;      // > 0: lowered tick bound (failure-detection tests); 0: the default
  int64_t id_offset;       // ensemble index of row 0: names the rows' random numbers (a shard of an ensemble)
  // long signals (null otherwise): per-stream moment sums of every slot,
  // [CTA][slot][kStreams][64] doubles, so that a sweep's streams can run on
  // several warps of the tick
  double* stream_part;
  // batched driver (null otherwise): CTA b runs block cta_map[b].y of event
  // cta_map[b].x, whose arguments are batch[cta_map[b].x]; an event's CTAs
  // return at once while *active == 0, and its counter is *stage << 8
  const NutsArgs* batch;
  const int2* cta_map;
  const int* active;
  const int* stage;
};

enum { METRIC_IDENTITY = 0, METRIC_DIAGONAL = 1, METRIC_DENSE = 2 };

// Per-slot state machine scalars: kept in shared memory between ticks and in
// the registers of the lane group that advances the slot in a tick (identical
// in all its lanes).
template <class VT>
struct Slot {
  int64_t pid;
  int t;           // transition index
  int depth;       // completed doublings
  long n;          // leaf index within the current sub-tree
  int dir;
  uint32_t leaf_ctr;
  double h0;       // Hamiltonian at the start of the transition
  double lnl_p, lnl_s, lnl_new;
  VT logw, logw_sub, acc;
  int n_leaf, divergent;
  int done;
  // stats
  double st_acc;
  long long st_bins;  // active (bin, detector) pairs, summed exactly in integers
  int st_depth, st_leap, st_div;
};

template <int SLOTS, class VT>
struct NutsShared {
  double pos[P_COUNT][SLOTS][kMaxDim];  // [field][slot][dim]: a slot's lanes read consecutive words
  VT vec[F_COUNT][SLOTS][kMaxDim];
  // metric: minv and its Cholesky factor, [kMaxDim][kMaxDim][mstride] each, after
  // NutsSmem in dynamic shared memory: one copy (shared metric, mstride = 1) or
  // one per slot (per-particle metric, mstride = SLOTS)
  VT* mmin;
  VT* mchol;
  int mstride;
  long long lokey[kMaxDim], hikey[kMaxDim];  // order keys of the prior box (see okey)
  double eps, beta;
  VT epsv;          // eps in the state machine's type
  double lp_const;  // sum of the prior's constant log terms
  int metric_kind;
  int alive;
  int pending[SLOTS];
  int order[SLOTS];  // this tick's sweeps, longest (largest k_ISCO) first
  int n_order;
  int next;          // next entry of order (or of items) to claim
  // long signals: the tick's sweep work items in claiming order, slot * 16 +
  // stream + 1 (stream -1: the slot's whole sweep)
  short items[SLOTS * kStreams];
  int n_items;
  int cslot[SLOTS];  // this tick's state machine of lane group g: slot cslot[g], or -1
  Slot<VT> sstate[SLOTS];
};

// Elementary functions in the state machine's precision.
__device__ __forceinline__ double vexp(double x) { return exp(x); }
__device__ __forceinline__ float vexp(float x) { return expf(x); }
__device__ __forceinline__ double vlog(double x) { return log(x); }
__device__ __forceinline__ float vlog(float x) { return logf(x); }
__device__ __forceinline__ double vsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float vsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ void vsincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void vsincospi(float x, float* s, float* c) { sincospif(x, s, c); }

// Order key of a double: for non-NaN x, y, okey(x) < okey(y) implies x < y
// (and x < y implies okey(x) < okey(y) except for -0 < +0). Lets the box test
// run on the integer pipes instead of the FP64 one.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

template <class VT>
__device__ __forceinline__ VT logaddexp(VT a, VT b) {
  if (a == -INFINITY) return b;
  if (b == -INFINITY) return a;
  VT mx = a > b ? a : b;
  return mx + vlog(vexp(a - mx) + vexp(b - mx));
}

// Two uniforms in (0, 1) from one Philox block, in the state machine's precision.
__device__ __forceinline__ void draw2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double* u0,
                                      double* u1) {
  uniform2(key, c0, c1, c2, c3, u0, u1);
}
__device__ __forceinline__ void draw2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, float* u0,
                                      float* u1) {
  uint32_t x[4];
  philox4x32_10(c0, c1, c2, c3, (uint32_t)key, (uint32_t)(key >> 32), x);
  *u0 = ((float)(x[0] >> 8) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
  *u1 = ((float)(x[2] >> 8) + 0.5f) * 5.9604644775390625e-8f;
}

// Lanes per slot and dimensions per lane of the state machine: a slot's G
// lanes each own the dimensions t, t + G, ... (t < G) of its vectors, padded
// to kLaneDims. Sums over the dimensions follow one fixed tree over kLaneDims
// terms (pairs d, d + 8 first, then + 4, + 2, + 1) whatever G is, so a
// trajectory does not depend on the slot count.
constexpr int kLaneDims = 16;
static_assert(kMaxDim <= kLaneDims, "one fixed reduction tree over at most 16 dimensions");

template <int PREC, int NDET, int SLOTS>
struct Nuts {
  using VT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  static constexpr int SPW = SLOTS / kNutsWarps;  // slots per warp
  // lanes per slot: 16, 8, 4 (16 also for one slot per warp, whose group
  // leaves the upper half-warp out: the group size fixes the arithmetic)
  static constexpr int G = SPW == 1 ? 16 : 32 / SPW;
  static constexpr int DPL = kLaneDims / G;       // dimensions per lane: 1, 2, 4
  const NutsArgs& A;
  NutsShared<SLOTS, VT>& S;
  int s;        // slot
  int t;        // lane within the slot's group
  unsigned gm;  // the group's lanes
  int D;
  __device__ Nuts(const NutsArgs& a, NutsShared<SLOTS, VT>& sh, int slot, int lane_in_group, unsigned mask)
      : A(a), S(sh), s(slot), t(lane_in_group), gm(mask), D(a.m.n_dim) {}
  __device__ int dim(int k) const { return t + G * k; }
  __device__ bool has(int k) const { return t + G * k < D; }
  __device__ VT& V(int f, int d) { return S.vec[f][s][d]; }
  __device__ VT& MI(int i, int j) { return S.mmin[(i * kMaxDim + j) * S.mstride + (S.mstride > 1 ? s : 0)]; }
  __device__ VT& CH(int i, int j) { return S.mchol[(i * kMaxDim + j) * S.mstride + (S.mstride > 1 ? s : 0)]; }
  __device__ double& X(int f, int d) { return S.pos[f][s][d]; }
  __device__ void sync() { __syncwarp(gm); }

  // Sum over the slot's dimensions of this lane's partial terms p[0..DPL).
  template <class T>
  __device__ T gsum(const T* p) {
    T x;
    if constexpr (DPL == 1)
      x = p[0];
    else if constexpr (DPL == 2)
      x = p[0] + p[1];
    else
      x = (p[0] + p[2]) + (p[1] + p[3]);
#pragma unroll
    for (int m = G / 2; m >= 1; m >>= 1) x += __shfl_xor_sync(gm, x, m);
    return x;
  }

  // v = Minv r for the momentum stored in field f (this lane's dimensions)
  __device__ void velocity(int f, VT* v) {
    const int kind = S.metric_kind;
    if (kind == METRIC_DENSE) sync();  // every lane reads the whole momentum
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = dim(k);
      v[k] = VT(0);
      if (!has(k)) continue;
      if (kind == METRIC_IDENTITY) {
        v[k] = V(f, d);
      } else if (kind == METRIC_DIAGONAL) {
        v[k] = MI(d, d) * V(f, d);
      } else {
        VT acc = VT(0);
        for (int j = 0; j < D; ++j) acc += MI(d, j) * V(f, j);
        v[k] = acc;
      }
    }
  }
  __device__ VT dot(const VT* a, int f) {
    VT p[DPL];
#pragma unroll
    for (int k = 0; k < DPL; ++k) p[k] = has(k) ? a[k] * V(f, dim(k)) : VT(0);
    return gsum(p);
  }
  __device__ VT dotv(const VT* a, const VT* b) {
    VT p[DPL];
#pragma unroll
    for (int k = 0; k < DPL; ++k) p[k] = has(k) ? a[k] * b[k] : VT(0);
    return gsum(p);
  }
  // ln pi (FP64 total) and grad ln pi with the constant terms precomputed.
  // CHECK = false: x is known to lie in the box (it came out of boundary()).
  template <bool CHECK = true>
  __device__ double prior(const double* x, VT* g) {
    const DevModel& m = A.m;
    VT p[DPL];  // the log terms in the state machine's type (FP32 ones are exact: one is nonzero in practice)
    bool inside = true;
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = dim(k);
      g[k] = VT(0);
      p[k] = VT(0);
      if (!has(k)) continue;
      if (CHECK && !(x[k] >= m.lo[d] && x[k] <= m.hi[d])) inside = false;
      if (m.prior[d] == SHARPY_PRIOR_POWER2) {
        const VT xi = (VT)x[k];
        p[k] = VT(2) * vlog(xi);
        g[k] = VT(2) / xi;
      }
    }
    const double lp = S.lp_const + (double)gsum(p);
    if (CHECK) inside = __all_sync(gm, inside);
    return inside ? lp : -INFINITY;
  }

  // Boundary maps on the pending leaf (P_N, F_NR). False if not finite.
  // Periodic dimensions wrap lane-parallel (no momentum change). Reflections
  // also run lane-parallel with an identity or diagonal metric, where a
  // reflection changes only its own dimension's momentum; with a dense metric
  // the momentum update reads the whole velocity, so they run dimension by
  // dimension in order.
  __device__ bool boundary() {
    const DevModel& m = A.m;
    bool ok = true, reflect = false;
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = dim(k);
      if (!has(k)) continue;
      double x = X(P_N, d);
      const long long b = __double_as_longlong(x);
      if ((b & 0x7ff0000000000000LL) == 0x7ff0000000000000LL) {  // not finite
        ok = false;
        continue;
      }
      const long long q = okey(x);
      if (m.boundary[d] != SHARPY_BOUND_PERIODIC) {
        if (q < S.lokey[d] || q > S.hikey[d]) reflect = true;
        continue;
      }
      // lo = +0 and +0 <= x < hi: the wrap below returns x itself (x - 0 = x,
      // 0 + x = x); skip its FP64 arithmetic
      if (S.lokey[d] == 0 && q >= 0 && q < S.hikey[d]) continue;
      // lo + ((x - lo) mod w): for |x - lo| < 2w one exact subtraction or
      // addition gives fmod's result; fmod only for larger excursions
      const double lo = m.lo[d], w = m.hi[d] - lo;
      double r = x - lo;
      if (r >= w)
        r = r < 2.0 * w ? r - w : fmod(r, w);
      else if (r < 0.0)
        r = r >= -w ? r : fmod(r, w);
      if (r < 0.0) r += w;
      X(P_N, d) = lo + r;
    }
    if (!__all_sync(gm, ok)) return false;
    if (!__any_sync(gm, reflect)) return true;
    if (S.metric_kind != METRIC_DENSE) {
      bool bad = false;
#pragma unroll
      for (int k = 0; k < DPL; ++k) {
        const int d = dim(k);
        if (!has(k) || m.boundary[d] == SHARPY_BOUND_PERIODIC) continue;
        const double lo = m.lo[d], hi = m.hi[d];
        double x = X(P_N, d);
        int flips = 0;
        while ((x < lo || x > hi) && flips < 100) {
          x = x < lo ? 2.0 * lo - x : 2.0 * hi - x;
          ++flips;
        }
        if (x < lo || x > hi) {
          bad = true;  // the leaf is discarded as divergent: nothing written matters
          continue;
        }
        X(P_N, d) = x;
        if (flips & 1) {
          const VT vi = S.metric_kind == METRIC_IDENTITY ? V(F_NR, d) : MI(d, d) * V(F_NR, d);
          V(F_NR, d) = V(F_NR, d) - VT(2) * vi / MI(d, d);
        }
      }
      if (__any_sync(gm, bad)) return false;
      sync();
      return true;
    }
    for (int i = 0; i < D; ++i) {
      if (m.boundary[i] == SHARPY_BOUND_PERIODIC) continue;
      const double lo = m.lo[i], hi = m.hi[i];
      int flips = 0;
      if (t == i % G) {
        double x = X(P_N, i);
        while ((x < lo || x > hi) && flips < 100) {
          x = x < lo ? 2.0 * lo - x : 2.0 * hi - x;
          ++flips;
        }
        if (x < lo || x > hi) flips = -1;
        else X(P_N, i) = x;
      }
      flips = __shfl_sync(gm, flips, i % G, G);
      if (flips < 0) return false;
      if (flips & 1) {
        sync();
        VT vi;
        if (S.metric_kind == METRIC_IDENTITY) {
          vi = V(F_NR, i);
        } else if (S.metric_kind == METRIC_DIAGONAL) {
          vi = MI(i, i) * V(F_NR, i);
        } else {
          VT acc = VT(0);
          for (int j = 0; j < D; ++j) acc += MI(i, j) * V(F_NR, j);
          vi = acc;
        }
        sync();
        if (t == i % G) V(F_NR, i) = V(F_NR, i) - VT(2) * vi / MI(i, i);
      }
    }
    sync();
    return true;
  }

  // First half of a leapfrog from the end of the tree in direction dir.
  __device__ bool begin_leapfrog(int dir) {
    const int pth = dir > 0 ? P_R : P_L, fr = dir > 0 ? F_RR : F_LR, fgu = dir > 0 ? F_RGU : F_LGU;
    const VT hv = dir > 0 ? S.epsv : -S.epsv;  // = (VT)(dir * eps)
#pragma unroll
    for (int k = 0; k < DPL; ++k)
      if (has(k)) V(F_NR, dim(k)) = V(fr, dim(k)) - VT(0.5) * hv * V(fgu, dim(k));
    VT v[DPL];
    velocity(F_NR, v);
    // x + (dir eps) v as x + eps (dir v): the same exact product, so the same
    // rounding, without forming -eps in FP64
#pragma unroll
    for (int k = 0; k < DPL; ++k)
      if (has(k)) X(P_N, dim(k)) = X(pth, dim(k)) + S.eps * (double)(dir > 0 ? v[k] : -v[k]);
    return boundary();
  }

  __device__ void draw_direction(Slot<VT>& sl) {
    VT u0, u1;
    draw2(A.key, (uint32_t)(sl.pid + A.id_offset), A.ctr + (uint32_t)sl.t, RNG_DIRECTION, (uint32_t)sl.depth, &u0, &u1);
    sl.dir = u0 < VT(0.5) ? -1 : 1;
    sl.n = 0;
    sl.logw_sub = -INFINITY;
#pragma unroll
    for (int k = 0; k < DPL; ++k)
      if (has(k)) V(F_RHOS, dim(k)) = VT(0);
  }

  // Start transition sl.t from the current point (P_P, F_PGL, lnl_p).
  __device__ void start_transition(Slot<VT>& sl) {
    const uint32_t step = A.ctr + (uint32_t)sl.t;
    // z ~ N(0, I): dimensions 2p and 2p + 1 from the normal pair p
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = dim(k);
      if (!has(k)) continue;
      VT u0, u1;
      draw2(A.key, (uint32_t)(sl.pid + A.id_offset), step, RNG_MOMENTUM, (uint32_t)(d >> 1), &u0, &u1);
      const VT r = vsqrt(VT(-2) * vlog(u0));
      VT sn, cs;
      vsincospi(VT(2) * u1, &sn, &cs);
      V(F_LR, d) = (d & 1) ? r * sn : r * cs;
    }
    // r ~ N(0, M), M = Minv^{-1} = (L L^T)^{-1}: solve L^T r = z (identity: r = z)
    if (S.metric_kind == METRIC_DIAGONAL) {
#pragma unroll
      for (int k = 0; k < DPL; ++k)
        if (has(k)) V(F_LR, dim(k)) = V(F_LR, dim(k)) / CH(dim(k), dim(k));
    } else if (S.metric_kind == METRIC_DENSE) {
      sync();
      if (t == 0)
        for (int i = D - 1; i >= 0; --i) {
          VT acc = V(F_LR, i);
          for (int j = i + 1; j < D; ++j) acc -= CH(j, i) * V(F_LR, j);
          V(F_LR, i) = acc / CH(i, i);
        }
      sync();
    }
    // U and grad U at the current point
    double x[DPL];
    VT glp[DPL], v0[DPL];
#pragma unroll
    for (int k = 0; k < DPL; ++k) x[k] = has(k) ? X(P_P, dim(k)) : 0.0;
    const double lp = prior(x, glp);
    const double u_cur = -S.beta * sl.lnl_p - lp;
    const VT bv = (VT)S.beta;
    velocity(F_LR, v0);
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      const int d = dim(k);
      if (!has(k)) continue;
      X(P_L, d) = x[k];
      X(P_R, d) = x[k];
      V(F_LGU, d) = -bv * V(F_PGL, d) - glp[k];
      V(F_LV, d) = v0[k];
      V(F_RR, d) = V(F_LR, d);
      V(F_RGU, d) = V(F_LGU, d);
      V(F_RV, d) = v0[k];
      V(F_RHO, d) = V(F_LR, d);
    }
    sl.h0 = u_cur + (double)(VT(0.5) * dot(v0, F_LR));
    sl.logw = VT(0);
    sl.depth = 0;
    sl.leaf_ctr = 0;
    sl.acc = VT(0);
    sl.n_leaf = 0;
    sl.divergent = 0;
  }

  __device__ void end_transition(Slot<VT>& sl) {
    sl.st_acc += sl.n_leaf > 0 ? (double)(sl.acc / (VT)sl.n_leaf) : 0.0;
    sl.st_depth += sl.depth;
    sl.st_leap += sl.n_leaf;
    sl.st_div += sl.divergent;
    sl.t += 1;
  }

  // Advance until the next evaluation is pending (true) or the slot is done.
  // have_leaf: a leaf evaluation just finished (P_N, F_NR hold its position and
  // half-step momentum; lnl_new, gl_new, lp_new, glp_new its values, gl_new
  // and glp_new for this lane's dimensions).
  __device__ bool advance(Slot<VT>& sl, bool have_leaf, const VT* gl_new, double lp_new, const VT* glp_new) {
    if (have_leaf) {
      // complete the leapfrog
      const VT h = sl.dir > 0 ? S.epsv : -S.epsv;  // = (VT)(dir * eps)
      const VT bv = (VT)S.beta;
      VT gu[DPL];
#pragma unroll
      for (int k = 0; k < DPL; ++k) {
        gu[k] = VT(0);
        if (!has(k)) continue;
        gu[k] = -bv * gl_new[k] - glp_new[k];
        V(F_NR, dim(k)) = V(F_NR, dim(k)) - VT(0.5) * h * gu[k];
      }
      const double u_new = -S.beta * sl.lnl_new - lp_new;
      VT vn[DPL];
      velocity(F_NR, vn);
      // energy error: U_new - H0 in FP64 (the two are ~beta ln L, large and
      // close), the kinetic part added in the state machine's type
      VT dH;
      if constexpr (std::is_same<VT, float>::value)
        dH = (float)(u_new - sl.h0) + VT(0.5) * dot(vn, F_NR);
      else
        dH = u_new + (double)(VT(0.5) * dot(vn, F_NR)) - sl.h0;
      sl.n_leaf += 1;
      sl.acc += (dH == dH) ? (dH <= VT(0) ? VT(1) : vexp(-dH)) : VT(0);
      if (!(dH <= VT(kDivergence))) {
        sl.divergent = 1;
        end_transition(sl);
        goto next_transition;
      }
      {
        // the leaf becomes the end of the tree in direction dir
        const int pth = sl.dir > 0 ? P_R : P_L, fr = sl.dir > 0 ? F_RR : F_LR, fgu = sl.dir > 0 ? F_RGU : F_LGU;
        const int fv = sl.dir > 0 ? F_RV : F_LV;
#pragma unroll
        for (int k = 0; k < DPL; ++k) {
          const int d = dim(k);
          if (!has(k)) continue;
          X(pth, d) = X(P_N, d);
          V(fr, d) = V(F_NR, d);
          V(fgu, d) = gu[k];
          V(fv, d) = vn[k];
        }
        const VT lw = -dH;
        const VT lw_new = logaddexp(sl.logw_sub, lw);
        VT u0, u1;
        draw2(A.key, (uint32_t)(sl.pid + A.id_offset), A.ctr + (uint32_t)sl.t, RNG_LEAF, sl.leaf_ctr++, &u0, &u1);
        if (u0 < vexp(lw - lw_new)) {
#pragma unroll
          for (int k = 0; k < DPL; ++k) {
            if (!has(k)) continue;
            X(P_S, dim(k)) = X(P_N, dim(k));
            V(F_SGL, dim(k)) = gl_new[k];
          }
          sl.lnl_s = sl.lnl_new;
        }
        sl.logw_sub = lw_new;
        for (int lvl = 1; lvl <= sl.depth; ++lvl)
          if ((sl.n & ((1L << lvl) - 1)) == 0)
#pragma unroll
            for (int k = 0; k < DPL; ++k) {
              if (!has(k)) continue;
              V(F_RS0 + lvl - 1, dim(k)) = V(F_RHOS, dim(k));
              V(F_RF0 + lvl - 1, dim(k)) = vn[k];
            }
#pragma unroll
        for (int k = 0; k < DPL; ++k)
          if (has(k)) V(F_RHOS, dim(k)) += V(F_NR, dim(k));
        bool ok = true;
        for (int lvl = 1; lvl <= sl.depth && ok; ++lvl)
          if (((sl.n + 1) & ((1L << lvl) - 1)) == 0) {
            VT rb[DPL];
#pragma unroll
            for (int k = 0; k < DPL; ++k) rb[k] = has(k) ? V(F_RHOS, dim(k)) - V(F_RS0 + lvl - 1, dim(k)) : VT(0);
            if (!(dot(rb, F_RF0 + lvl - 1) > VT(0) && dotv(rb, vn) > VT(0))) ok = false;
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
        draw2(A.key, (uint32_t)(sl.pid + A.id_offset), A.ctr + (uint32_t)sl.t, RNG_TOP, (uint32_t)sl.depth, &u0, &u1);
        if (u0 < vexp(sl.logw_sub - sl.logw)) {
#pragma unroll
          for (int k = 0; k < DPL; ++k) {
            if (!has(k)) continue;
            X(P_P, dim(k)) = X(P_S, dim(k));
            V(F_PGL, dim(k)) = V(F_SGL, dim(k));
          }
          sl.lnl_p = sl.lnl_s;
        }
        sl.logw = logaddexp(sl.logw, sl.logw_sub);
        VT rho[DPL];
#pragma unroll
        for (int k = 0; k < DPL; ++k) {
          rho[k] = VT(0);
          if (!has(k)) continue;
          V(F_RHO, dim(k)) += V(F_RHOS, dim(k));
          rho[k] = V(F_RHO, dim(k));
        }
        sl.depth += 1;
        if (!(dot(rho, F_LV) > VT(0) && dot(rho, F_RV) > VT(0)) || sl.depth >= A.max_depth) {
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
struct NutsSmem;

// Byte offset of the metric arrays in dynamic shared memory and the total size.
template <int PREC, int NDET, int SLOTS>
__host__ __device__ constexpr size_t nuts_metric_offset() {
  return (sizeof(NutsSmem<PREC, NDET, SLOTS>) + 15) / 16 * 16;
}
template <int PREC, int NDET, int SLOTS>
__host__ __device__ constexpr size_t nuts_smem_bytes(bool local) {
  using VT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  return nuts_metric_offset<PREC, NDET, SLOTS>() + 2 * kMaxDim * kMaxDim * (local ? SLOTS : 1) * sizeof(VT);
}

template <int PREC, int NDET, int SLOTS>
struct NutsSmem {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  using MT = typename MomType<PREC>::type;
  NutsShared<SLOTS, DT> S;
  SweepCoef sc[SLOTS];
  EpiCoef<DT> ec[SLOTS];
  MT mom[SLOTS][NDET * kNMom * 2];
};

// Mixed paths: registers for three CTAs per SM (168 a thread, no spills),
// which the 8- and 16-slot launches can use (9 % on 16384 particles); FP64:
// two.
template <int PREC, int NDET, int SLOTS>
__global__ void __launch_bounds__(kNutsWarps * 32, PREC == SHARPY_FP64 ? 2 : (SLOTS == 4 ? 4 : 3))
    nuts_kernel(const __grid_constant__ NutsArgs P) {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  using VT = DT;
  using MT = typename MomType<PREC>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // this CTA's arguments (its event's, in a batched launch) in shared memory
  __shared__ __align__(16) NutsArgs A;
  __shared__ int s_block, s_skip;
  {
    const int2 cm = P.batch ? P.cta_map[blockIdx.x] : make_int2(0, (int)blockIdx.x);
    const NutsArgs* src = P.batch ? P.batch + cm.x : &P;
    static_assert(sizeof(NutsArgs) % 8 == 0, "NutsArgs is copied as 8-byte words");
    const unsigned long long* s8 = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d8 = reinterpret_cast<unsigned long long*>(&A);
    for (int i = threadIdx.x; i < (int)(sizeof(NutsArgs) / 8); i += blockDim.x) d8[i] = s8[i];
    __syncthreads();
    if (threadIdx.x == 0) {
      s_block = cm.y;
      s_skip = (A.active && *A.active == 0) ? 1 : 0;
      if (A.stage) A.ctr = (uint32_t)(*A.stage) << 8;
    }
    __syncthreads();
    if (s_skip) return;
  }
  NutsSmem<PREC, NDET, SLOTS>& SM = *reinterpret_cast<NutsSmem<PREC, NDET, SLOTS>*>(smem_raw);
  NutsShared<SLOTS, VT>& S = SM.S;
  SweepCoef* sc = SM.sc;
  EpiCoef<DT>* ec = SM.ec;
  auto& mom = SM.mom;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // control warp: warp 0 or 2 by CTA parity, so the serial (FP64-heavy) phases
  // of two CTAs sharing an SM run on different SM sub-partitions
  const int cw = (blockIdx.x & 1) << 1;
  const int D = A.m.n_dim;
  const bool gw = A.m.model == SHARPY_MODEL_TAYLORF2;

  // metric, its Cholesky factor (diagonal fallback; computed in FP64), step size, beta
  if (threadIdx.x == 0) {
    S.mstride = A.local_metric ? SLOTS : 1;
    S.mmin = reinterpret_cast<VT*>(smem_raw + nuts_metric_offset<PREC, NDET, SLOTS>());
    S.mchol = S.mmin + kMaxDim * kMaxDim * S.mstride;
    double mi[kMaxDim][kMaxDim], ch[kMaxDim][kMaxDim];
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) mi[i][j] = A.minv ? A.minv[i * D + j] : (i == j ? 1.0 : 0.0);
    bool ok = true;
    for (int j = 0; j < D && ok; ++j) {
      for (int i = 0; i < D; ++i) ch[i][j] = 0.0;
      double d = mi[j][j];
      for (int k = 0; k < j; ++k) d -= ch[j][k] * ch[j][k];
      if (!(d > 0.0) || !isfinite(d)) {
        ok = false;
        break;
      }
      ch[j][j] = sqrt(d);
      for (int i = j + 1; i < D; ++i) {
        double t = mi[i][j];
        for (int k = 0; k < j; ++k) t -= ch[i][k] * ch[j][k];
        ch[i][j] = t / ch[j][j];
      }
    }
    if (!ok)
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
          double dii = mi[i][i] > 0.0 && isfinite(mi[i][i]) ? mi[i][i] : 1.0;
          mi[i][j] = i == j ? dii : 0.0;
          ch[i][j] = i == j ? sqrt(dii) : 0.0;
        }
    bool ident = true, diag = true;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        if (i != j && mi[i][j] != 0.0) diag = false;
        if (mi[i][j] != (i == j ? 1.0 : 0.0)) ident = false;
        S.mmin[i * kMaxDim + j] = (VT)mi[i][j];  // the one copy (or slot 0's)
        S.mchol[i * kMaxDim + j] = (VT)ch[i][j];
      }
    S.metric_kind = A.pminv ? METRIC_DENSE : ident ? METRIC_IDENTITY : (diag ? METRIC_DIAGONAL : METRIC_DENSE);
    for (int i = 0; i < D; ++i) {
      S.lokey[i] = okey(A.m.lo[i]);
      S.hikey[i] = okey(A.m.hi[i]);
    }
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
    S.epsv = (VT)eps;
    S.beta = A.beta_ptr ? *A.beta_ptr : A.beta;
  }
  __syncthreads();

  // Slot ownership: warp w runs the state machines of slots w SPW ..
  // w SPW + SPW - 1, each on a group of G = 32 / SPW lanes that share its
  // vectors' dimensions, so the per-slot phases of a tick (epilogue, tree
  // update, next leapfrog) run on all four SM sub-partitions at once.
  using NT = Nuts<PREC, NDET, SLOTS>;
  constexpr int SPW = NT::SPW, G = NT::G, DPL = NT::DPL;
  static_assert(SLOTS % kNutsWarps == 0, "slots are shared evenly by the warps");
  const bool in_group = lane / G < SPW;   // false: the idle half-warp of a one-slot warp
  const int my = in_group ? warp * SPW + lane / G : -1;  // this lane's slot
  const int tg = lane % G;                // its lane within the slot's group
  const unsigned gmask = (G == 32 ? 0xffffffffu : ((1u << G) - 1u)) << (lane - tg);
  if (in_group) {
    Slot<VT> sl;
    NT nu(A, S, my, tg, gmask);
    sl.pid = (int64_t)s_block * SLOTS + my;
    sl.t = 0;
    sl.done = 1;
    sl.st_acc = 0.0;
    sl.st_bins = 0;
    sl.st_depth = sl.st_leap = sl.st_div = 0;
    bool active = false;
    if (sl.pid < A.n) {
#pragma unroll
      for (int k = 0; k < DPL; ++k) {
        const int d = nu.dim(k);
        if (!nu.has(k)) continue;
        nu.X(P_P, d) = A.theta[sl.pid * D + d];
        nu.V(F_PGL, d) = (VT)A.grad[sl.pid * D + d];
        if (A.pminv) {
          const double* pm = A.pminv + sl.pid * D * D;
          const double* pc = A.pchol + sl.pid * D * D;
          for (int j = 0; j < D; ++j) {
            nu.MI(d, j) = (VT)pm[d * D + j];
            nu.CH(d, j) = (VT)pc[d * D + j];
          }
        }
      }
      sl.lnl_p = A.lnl[sl.pid];
      nu.sync();
      sl.done = 0;
      active = nu.advance(sl, false, nullptr, 0.0, nullptr);
    }
    if (tg == 0) {
      S.pending[my] = active ? 1 : 0;
      S.sstate[my] = sl;
    }
  }
  __syncthreads();
  const long max_ticks = A.tick_limit > 0 ? (long)A.tick_limit : (long)A.n_steps * ((1L << A.max_depth) + 1) + 4;
  for (long tick = 0;; ++tick) {
    // warp 0: any pending evaluation left?
    if (warp == cw) {
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
    // (A) prologues (GW models; lane = slot): the phase half on the control
    // warp, the sky half on its neighbour, on another sub-partition
    if (gw && (warp == cw || warp == (cw ^ 1)) && lane < SLOTS && S.pending[lane]) {
      double x[kMaxDim];
      for (int i = 0; i < D; ++i) x[i] = S.pos[P_N][lane][i];
      if (warp == cw)
        prologue_phase<DT, true, PREC == SHARPY_MIXED_SPLIT>(A.m, A.ev, x, sc[lane], ec[lane]);
      else
        prologue_sky<DT, true, PREC == SHARPY_MIXED_SPLIT>(A.m, A.ev, x, sc[lane], ec[lane]);
    }
    if (gw && warp == cw) {
      // order this tick's sweeps by decreasing k_ISCO (ties: slot order)
      const int key = (lane < SLOTS && S.pending[lane] && sc[lane].ok) ? sc[lane].kisco : -2;
      int rank = 0;
#pragma unroll
      for (int j = 0; j < SLOTS; ++j) {
        const int kj = __shfl_sync(0xffffffffu, key, j);
        rank += (kj > key || (kj == key && j < lane)) ? 1 : 0;
      }
      if (key >= -1) S.order[rank] = lane;
      const unsigned sweeps = __ballot_sync(0xffffffffu, key >= -1);
      if (lane == 0) {
        S.n_order = __popc(sweeps);
        S.next = 0;
      }
      if (A.stream_part) {
        // a sweep of more than one chunk becomes its kStreams streams, each a
        // work item, longest sweeps first
        __syncwarp();
        if (lane == 0) {
          int ni = 0;
          for (int r = 0; r < S.n_order; ++r) {
            const int slot = S.order[r];
            if (sc[slot].kisco >= kChunkBins)
              for (int st = 0; st < kStreams; ++st) S.items[ni++] = (short)(slot * 16 + st + 1);
            else
              S.items[ni++] = (short)(slot * 16);
          }
          S.n_items = ni;
        }
      }
    }
    if (warp == cw) {
      // this tick's state machines, one per warp before a second one on any
      // warp: pending slot of rank i goes to group (i mod 4) SPW + i / 4
      const bool pd = lane < SLOTS && S.pending[lane];
      const unsigned pm = __ballot_sync(0xffffffffu, pd);
      if (lane < SLOTS) S.cslot[lane] = -1;
      __syncwarp();
      if (pd) {
        const int r = __popc(pm & ((1u << lane) - 1u));
        S.cslot[(r % kNutsWarps) * SPW + r / kNutsWarps] = lane;
      }
    }
    __syncthreads();
    // (B) sweeps: each warp claims the next sweep of the longest-first order
    // (a sweep writes all its moments; the warp that runs it does not change
    // the result)
    if (gw && !A.stream_part) {
      for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&S.next, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= S.n_order) break;
        const int slot = S.order[k];
        sweep<PREC, true, NDET>(A.ev, sc[slot], mom[slot]);
      }
    } else if (gw) {
      // long signals: whole short sweeps, and the streams of the long ones
      // with their sums stored per stream (merged in stream order below)
      constexpr int NACC = MomCount<NDET, true>::value;
      using FS = FlushShape<NACC>;
      for (;;) {
        int k = 0;
        if (lane == 0) k = atomicAdd(&S.next, 1);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= S.n_items) break;
        const int item = S.items[k];
        const int slot = item >> 4, st = (item & 15) - 1;
        if (st < 0) {
          sweep<PREC, true, NDET>(A.ev, sc[slot], mom[slot]);
          continue;
        }
        double v[FS::KEEP];
        if constexpr (PREC == SHARPY_FP64) {
          fp64_stream<true, NDET>(A.ev, sc[slot], st, v);
        } else {
          float hi[FS::KEEP], lo[FS::KEEP];
          mixed_stream<true, NDET, PREC == SHARPY_MIXED_SPLIT>(A.ev, sc[slot], st, hi, lo);
#pragma unroll
          for (int t = 0; t < FS::KEEP; ++t) v[t] = (double)hi[t] + (double)lo[t];
        }
        double* part = A.stream_part + (((int64_t)blockIdx.x * SLOTS + slot) * kStreams + st) * 64;
#pragma unroll
        for (int t = 0; t < FS::KEEP; ++t) part[lane * FS::KEEP + t] = v[t];
      }
    }
    __syncthreads();
    // (C) epilogues (or direct evaluations: Gaussian mixture) and state
    // machines, each on the lane group assigned to it this tick (the scalar
    // parts run identically on every lane of the group); which group runs a
    // slot does not change what it computes
    const int cs = in_group ? S.cslot[warp * SPW + lane / G] : -1;
    if (cs >= 0) {
      if (gw && A.stream_part && sc[cs].ok && sc[cs].kisco >= kChunkBins) {
        // the slot's streams, in stream order (the sum sweep() forms on one warp)
        constexpr int NACC = MomCount<NDET, true>::value;
        const double* part = A.stream_part + ((int64_t)blockIdx.x * SLOTS + cs) * kStreams * 64;
        for (int idx = tg; idx < NACC; idx += G) {
          double tot = 0.0;
          for (int st = 0; st < kStreams; ++st) tot += part[st * 64 + idx];
          mom[cs][acc_to_mom<NDET, true>(idx)] = (MT)tot;
        }
        __syncwarp(gmask);
      }
      Slot<VT> sl = S.sstate[cs];
      NT nu(A, S, cs, tg, gmask);
      VT gl_new[DPL], glp_new[DPL];
      double x[DPL];
#pragma unroll
      for (int k = 0; k < DPL; ++k) x[k] = nu.has(k) ? nu.X(P_N, nu.dim(k)) : 0.0;
      if (gw) {
        DT gph[SHARPY_NPHYS];
        sl.lnl_new = NAN;
        if (sc[cs].ok) {
          epilogue<DT, true>(A.ev, sc[cs], ec[cs], mom[cs], &sl.lnl_new, gph);
          sl.st_bins += (long long)(sc[cs].kisco + 1) * A.ev.n_det;
        }
#pragma unroll
        for (int k = 0; k < DPL; ++k)
          gl_new[k] = !nu.has(k) ? VT(0) : sc[cs].ok ? (VT)gph[A.m.phys[nu.dim(k)]] : (VT)NAN;
      } else {
        double xa[kMaxDim], g[kMaxDim];
        for (int i = 0; i < D; ++i) xa[i] = nu.X(P_N, i);
        gaussmix(A.m, xa, &sl.lnl_new, g);
#pragma unroll
        for (int k = 0; k < DPL; ++k) gl_new[k] = nu.has(k) ? (VT)g[nu.dim(k)] : VT(0);
      }
      const double lp_new = nu.template prior<false>(x, glp_new);
      if (!isfinite(sl.lnl_new)) sl.lnl_new = -INFINITY;  // rejected leaf (U = +inf)
#pragma unroll
      for (int k = 0; k < DPL; ++k)
        if (!isfinite(gl_new[k])) gl_new[k] = VT(0);
      const bool more = nu.advance(sl, true, gl_new, lp_new, glp_new);
      nu.sync();
      if (tg == 0) {
        S.pending[cs] = more ? 1 : 0;
        S.sstate[cs] = sl;
      }
    }
    __syncthreads();  // the control warp reads every slot's pending flag next
  }
  // write back
  if (!in_group) return;
  const Slot<VT> sl = S.sstate[my];
  if (sl.pid < A.n) {
    NT nu(A, S, my, tg, gmask);
#pragma unroll
    for (int k = 0; k < DPL; ++k) {
      if (!nu.has(k)) continue;
      A.theta[sl.pid * D + nu.dim(k)] = nu.X(P_P, nu.dim(k));
      A.grad[sl.pid * D + nu.dim(k)] = (double)nu.V(F_PGL, nu.dim(k));
    }
  }
  if (tg == 0 && sl.pid < A.n) {
    A.lnl[sl.pid] = sl.lnl_p;
    if (A.stats) {
      sharpy_nuts_stats st;
      st.accept_sum = sl.st_acc;
      st.active_bins = (double)sl.st_bins;
      st.depth_sum = sl.st_depth;
      st.n_leapfrog = sl.st_leap;
      st.n_divergent = sl.st_div;
      st.pad = 0;
      A.stats[sl.pid] = st;
    }
  }
}

// Launch helper for one (precision, detector count); the slot count is picked
// by the caller; grid 0 means one CTA per SLOTS particles of A (a batched
// launch passes its CTA count). Defined in nuts_inst.cu, compiled once per
// combination.
int launch_nuts(int precision, int ndet, int slots, const NutsArgs& A, unsigned grid, cudaStream_t s);

template <int P, int ND>
int launch_nuts_impl(int slots, const NutsArgs& A, unsigned grid, cudaStream_t s) {
  auto go = [&](auto kernel, int sl, size_t bytes) -> int {
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
      return SHARPY_ECUDA;
    const unsigned g = grid ? grid : (unsigned)((A.n + sl - 1) / sl);
    kernel<<<g, kNutsWarps * 32, bytes, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? SHARPY_OK : SHARPY_ECUDA;
  };
  const bool local = A.local_metric != 0;
  if (slots == 4) return go(nuts_kernel<P, ND, 4>, 4, nuts_smem_bytes<P, ND, 4>(local));
  if (slots == 32) return go(nuts_kernel<P, ND, 32>, 32, nuts_smem_bytes<P, ND, 32>(local));
  if (slots == 16) return go(nuts_kernel<P, ND, 16>, 16, nuts_smem_bytes<P, ND, 16>(local));
  return go(nuts_kernel<P, ND, 8>, 8, nuts_smem_bytes<P, ND, 8>(local));
}

}  // namespace sharpy
