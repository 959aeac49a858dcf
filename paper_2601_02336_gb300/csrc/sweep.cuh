// The per-bin sweep: one warp accumulates the moments of one particle.
//
// Lane l visits bins k = l, l+32, ... <= k_ISCO (coalesced SoA table reads).
// Per bin the phase polynomial sum_j alpha_j B_j(f_k) + c0 is shared by all
// detectors; per detector it adds f_k tau_a, reduces mod 1 turn, forms the
// carrier e^{-i Psi}, multiplies the pre-whitened data E_ak and accumulates
// Z_a (and, for the gradient, Y_aj = sum z B_j).
//
//   SHARPY_FP64  : FP64 throughout; reduction Psi - rint(Psi); sincospi.
//   SHARPY_MIXED_SPLIT : as SHARPY_MIXED, but the phase polynomial is built
//                  from hi/lo FP32 splits of alpha_j, tau_a and B_j(f_k):
//                  each product's integer turns are removed exactly (FMA error
//                  term kept), the fraction stays in [-1/2, 1/2]; no FP64 in
//                  the bin loop (worst-case phase error ~3e-7 turns).
//   SHARPY_MIXED : the post-Newtonian terms that carry the large phase
//                  (x^5, x^3, x^2, ln f) accumulated in FP64 on top of the
//                  offset 1.5 * 2^20 turns, whose low mantissa word is their
//                  fractional turn in 2^-32 units; the four terms below ~8
//                  turns (x, y, y ln f, y^2) in FP32 pairs as in the split
//                  path, added in 32-bit fixed point; the delay term f tau_a
//                  of each detector in FP32 from hi/lo splits (exact FMA error
//                  term, fraction added in 32-bit fixed point); FP32 sincos,
//                  carrier and moments. Per-lane FP32 partial sums are flushed
//                  every kFlush iterations through a fixed-order warp tree
//                  into compensated FP32 outer accumulators (blocked pairwise
//                  summation).
#pragma once
#include "physics.cuh"

namespace sharpy {

constexpr int kFlush = 64;  // lane iterations per FP32 block
// Long sweeps are cut into chunks of kFlush lane iterations (2048 bins) dealt
// to kStreams streams (chunk c to stream c mod kStreams); a stream's result
// does not depend on which warp computes it, and streams are merged in a fixed
// order, so any number of warps per particle gives the same moments.
constexpr int kChunkBins = kFlush * 32;
constexpr int kStreams = 8;

template <int NDET, bool GRAD>
struct MomCount {
  static constexpr int value = GRAD ? NDET * kNMom * 2 : NDET * 2;
};

// Index of moment (a, j, ri) in the full layout.
__device__ __forceinline__ int mom_index(int a, int j, int ri) { return (a * kNMom + j) * 2 + ri; }

template <int NDET, bool GRAD>
__device__ __forceinline__ int acc_to_mom(int i) {
  if (GRAD) return i;
  return mom_index(i / 2, 9, i & 1);
}

// Warp reduce-scatter of NP per-lane values (NP a power of two): at each
// butterfly level a lane keeps one half of its values and sends the other
// half to its partner, so the 32-lane sums of all NP values take
// NP/2 + NP/4 + ... shuffles instead of 5 NP. Fixed pairing: deterministic.
// Afterwards, for NP >= 32, lane l holds the sums of values
// l (NP/32) ... l (NP/32) + NP/32 - 1 in v[0 .. NP/32); for NP < 32 the lanes
// of each group of 32/NP consecutive lanes all hold the sum of value
// l / (32/NP) in v[0].
template <int N, int OFF, class T = float>
struct ReduceScatter {
  static __device__ __forceinline__ void run(T* v, int lane) {
    constexpr int H = N / 2;
    const bool up = (lane & OFF) != 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
      const T send = up ? v[j] : v[j + H];
      const T keep = up ? v[j + H] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    ReduceScatter<H, OFF / 2, T>::run(v, lane);
  }
};
template <int OFF, class T>
struct ReduceScatter<1, OFF, T> {
  static __device__ __forceinline__ void run(T* v, int) {
#pragma unroll
    for (int o = OFF; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  }
};
template <int N, class T>
struct ReduceScatter<N, 0, T> {
  static __device__ __forceinline__ void run(T*, int) {}
};
template <class T>
struct ReduceScatter<1, 0, T> {
  static __device__ __forceinline__ void run(T*, int) {}
};

template <int NACC>
struct FlushShape {
  static constexpr int NP = NACC <= 2 ? 2 : NACC <= 4 ? 4 : NACC <= 8 ? 8 : NACC <= 16 ? 16 : NACC <= 32 ? 32 : 64;
  static constexpr int KEEP = NP >= 32 ? NP / 32 : 1;  // sums held per lane
  static __device__ __forceinline__ int index(int lane, int t) { return NP >= 32 ? lane * KEEP + t : lane / (32 / NP); }
  static __device__ __forceinline__ bool owner(int lane) { return NP >= 32 || lane % (32 / NP) == 0; }
};

// Flush per-lane FP32 partials into the lane-distributed outer accumulators:
// each block sum (reduce-scatter above) is added with an error-free two-sum,
// so the outer sums carry ~48 bits without FP64 arithmetic.
template <int NACC>
__device__ __forceinline__ void flush(float* acc, float* hi, float* lo, int lane) {
  using F = FlushShape<NACC>;
  static_assert(NACC <= 64, "at most 64 moments per lane");
  float v[F::NP];
#pragma unroll
  for (int i = 0; i < F::NP; ++i) v[i] = i < NACC ? acc[i] : 0.0f;
  ReduceScatter<F::NP, 16>::run(v, lane);
#pragma unroll
  for (int t = 0; t < F::KEEP; ++t) {
    const float s = hi[t] + v[t];
    const float bp = s - hi[t];
    lo[t] += (hi[t] - (s - bp)) + (v[t] - bp);
    hi[t] = s;
  }
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.0f;
}

// Magic constant for exact round-to-nearest of |x| < 2^22 in FP32.
constexpr float kRound32 = 12582912.0f;  // 1.5 * 2^23

// x - rint(x) for |x| < 2^22, exact (explicit roundings: no contraction).
__device__ __forceinline__ float frac_turn(float x) {
  return __fsub_rn(x, __fsub_rn(__fadd_rn(x, kRound32), kRound32));
}

// One stream of a mixed sweep: the chunks c = s, s + kStreams, ... of 2048
// bins (64 lane iterations: one FP32 block each) below k_ISCO, accumulated
// into this lane's compensated outer sums hi, lo (kept lane-distributed as
// the flush leaves them). Returns whether the stream had any bin.
// Table values of one bin for the mixed sweep, from the SoA tables in global
// memory (bin k).
struct GlobalBin {
  const DevEvent& ev;
  int64_t K;
  int k;
  __device__ __forceinline__ float b32(int j) const { return __ldg(ev.b32 + (int64_t)j * K + k); }
  __device__ __forceinline__ float b32lo(int j) const { return __ldg(ev.b32lo + (int64_t)j * K + k); }
  __device__ __forceinline__ double b64(int j) const { return __ldg(ev.b64 + (int64_t)j * K + k); }
  __device__ __forceinline__ float2 e32(int a) const { return __ldg(ev.e32 + (int64_t)a * K + k); }
};

// The same values from a staged record in shared memory (bin i of its block;
// the mixed sweep's tables only: the split sweep also reads the large terms'
// lo parts).
struct StagedBin {
  const unsigned char* rec;
  int i;
  __device__ __forceinline__ float b32(int j) const { return reinterpret_cast<const float*>(rec)[j * kStageBins + i]; }
  __device__ __forceinline__ float b32lo(int j) const {
    return reinterpret_cast<const float*>(rec + stage_off_lo())[stage_lo_row(j) * kStageBins + i];
  }
  __device__ __forceinline__ double b64(int j) const {
    return reinterpret_cast<const double*>(rec + stage_off_b64())[stage_b64_row(j) * kStageBins + i];
  }
  __device__ __forceinline__ float2 e32(int a) const {
    return reinterpret_cast<const float2*>(rec + stage_off_e32())[a * kStageBins + i];
  }
};

// Per-particle constants of the mixed sweep, held in registers.
template <int NDET>
struct MixedCoef {
  double al[kNPn];
  double s0;
  float ah[kNPn], alo[kNPn], th[NDET], tl[NDET];
};

template <int NDET>
__device__ __forceinline__ void mixed_coef(const SweepCoef& sc, MixedCoef<NDET>& P) {
#pragma unroll
  for (int j = 0; j < kNPn; ++j) P.al[j] = sc.alpha[j];
  P.s0 = sc.c0 + kTurnOffset;
#pragma unroll
  for (int j = 0; j < kNPn; ++j) {
    P.ah[j] = sc.ahi[j];
    P.alo[j] = sc.alo[j];
  }
#pragma unroll
  for (int a = 0; a < NDET; ++a) {
    P.th[a] = sc.thi[a];
    P.tl[a] = sc.tlo[a];
  }
}

// One bin of the mixed (or split) sweep: its phase, carrier and moment
// updates, with the bin's table values from the loader ld (global memory or a
// shared-memory stage: the same values, so the same sums).
template <bool GRAD, int NDET, bool SPLIT, class L>
__device__ __forceinline__ void mixed_bin(const SweepCoef& sc, const MixedCoef<NDET>& P, const L& ld, float* acc) {
  const double (&al)[kNPn] = P.al;
  const double s0 = P.s0;
  const float (&ah)[kNPn] = P.ah;
  const float (&alo)[kNPn] = P.alo;
  const float (&th)[NDET] = P.th;
  const float (&tl)[NDET] = P.tl;
  float bf[kNBasis];
  if (GRAD || SPLIT) {
#pragma unroll
    for (int j = 0; j < kNBasis; ++j) bf[j] = ld.b32(j);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) bf[small_pn(i)] = ld.b32(small_pn(i));
    bf[8] = ld.b32(8);
  }
  const float fl = ld.b32lo(8);
  // phase: FP64 accumulation on the turn offset, or split single precision
  double S = s0;
  int turn_s = 0;
  float F = 0.0f, Sm = 0.0f;
  if (!SPLIT) {
    // the four terms that carry the large phase (Newtonian, 1PN, 1.5PN and
    // the 2.5PN logarithm: up to ~2e3 turns on the long segment) accumulated
    // in FP64 on the offset
#pragma unroll
    for (int i = 0; i < 4; ++i) S = fma(al[large_pn(i)], ld.b64(large_pn(i)), S);
    turn_s = __double2loint(S);  // fractional turn of the large terms, 2^-32 units
    // the four terms below ~8 turns (2PN, 3PN, its logarithm, 3.5PN) in FP32
    // pairs: each product's integer turns removed exactly (FMA error term
    // kept), the fractions summed pairwise in [-1/2, 1/2], then added to the
    // FP64 part in 32-bit fixed point
    float fr[4], er[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = small_pn(i);
      const float bl = ld.b32lo(j);
      const float p = __fmul_rn(ah[j], bf[j]);
      fr[i] = frac_turn(p);
      er[i] = fmaf(ah[j], bl, fmaf(alo[j], bf[j], fmaf(ah[j], bf[j], -p)));
    }
    const float f = frac_turn(__fadd_rn(frac_turn(__fadd_rn(fr[0], fr[1])), frac_turn(__fadd_rn(fr[2], fr[3]))));
    const float q = frac_turn(__fadd_rn(f, __fadd_rn(__fadd_rn(er[0], er[1]), __fadd_rn(er[2], er[3]))));
    turn_s += __float2int_rn(q * 4294967296.0f);  // wraps mod 1 turn
  } else {
    // sum_j alpha_j B_j mod 1: p = ahi*bhi is exact up to e (FMA), its integer
    // part is removed exactly; the fractions are summed pairwise, reduced to
    // [-1/2, 1/2] at every level (three levels instead of an eight-step
    // chain), the error and cross terms likewise pairwise in Sm.
    static_assert(kNPn == 8, "the pairwise tree below is written for eight basis terms");
    float fr[kNPn], er[kNPn];
#pragma unroll
    for (int j = 0; j < kNPn; ++j) {
      const float bl = ld.b32lo(j);
      const float p = __fmul_rn(ah[j], bf[j]);
      fr[j] = frac_turn(p);
      er[j] = fmaf(ah[j], bl, fmaf(alo[j], bf[j], fmaf(ah[j], bf[j], -p)));
    }
    const float f01 = frac_turn(__fadd_rn(fr[0], fr[1])), f23 = frac_turn(__fadd_rn(fr[2], fr[3]));
    const float f45 = frac_turn(__fadd_rn(fr[4], fr[5])), f67 = frac_turn(__fadd_rn(fr[6], fr[7]));
    const float f03 = frac_turn(__fadd_rn(f01, f23)), f47 = frac_turn(__fadd_rn(f45, f67));
    F = frac_turn(__fadd_rn(__fadd_rn(f03, f47), sc.c0f));
    Sm = __fadd_rn(__fadd_rn(__fadd_rn(er[0], er[1]), __fadd_rn(er[2], er[3])),
                   __fadd_rn(__fadd_rn(er[4], er[5]), __fadd_rn(er[6], er[7])));
  }
#pragma unroll
  for (int a = 0; a < NDET; ++a) {
    float ang;
    if (!SPLIT) {
      // f tau_a mod 1 from (thi + tlo)(fhi + flo): p = thi fhi is exact up
      // to e (FMA), the other products are below 2^-20 turn
      const float p = __fmul_rn(th[a], bf[8]);
      const float e = fmaf(th[a], fl, fmaf(tl[a], bf[8], fmaf(th[a], bf[8], -p)));
      const float q = frac_turn(__fadd_rn(frac_turn(p), e));  // [-1/2, 1/2] turn
      const int turn = turn_s + __float2int_rn(q * 4294967296.0f);  // wraps mod 1 turn
      ang = (float)turn * 1.46291807926715968e-9f;  // 2 pi / 2^32
    } else {
      const float p = __fmul_rn(th[a], bf[8]);
      float Sa = Sm + fmaf(th[a], bf[8], -p);
      Sa = fmaf(th[a], fl, fmaf(tl[a], bf[8], Sa));
      const float Fa = frac_turn(__fadd_rn(F, frac_turn(p)));
      ang = (Fa + Sa) * 6.28318530717958648f;
    }
    float sn, cs;
    __sincosf(ang, &sn, &cs);
    const float2 E = ld.e32(a);
    const float zr = E.x * cs + E.y * sn;
    const float zi = E.y * cs - E.x * sn;
    if (GRAD) {
#pragma unroll
      for (int j = 0; j < kNBasis; ++j) {
        acc[(a * kNMom + j) * 2] += zr * bf[j];
        acc[(a * kNMom + j) * 2 + 1] += zi * bf[j];
      }
      acc[(a * kNMom + 9) * 2] += zr;
      acc[(a * kNMom + 9) * 2 + 1] += zi;
    } else {
      acc[a * 2] += zr;
      acc[a * 2 + 1] += zi;
    }
  }
}

template <bool GRAD, int NDET, bool SPLIT>
__device__ bool mixed_stream(const DevEvent& ev, const SweepCoef& sc, int s, float* hi, float* lo) {
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  constexpr int NOUT = FlushShape<NACC>::KEEP;
  const int lane = threadIdx.x & 31;
  const int64_t K = ev.n_bins;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < NOUT; ++i) hi[i] = lo[i] = 0.0f;
  MixedCoef<NDET> P;
  mixed_coef<NDET>(sc, P);
  const int kend = sc.kisco;
  bool any = false;
  // Warp-uniform trip counts: lanes past k_ISCO idle but still join the flushes.
  for (int c = s; c * kChunkBins <= kend; c += kStreams) {
    any = true;
    for (int it = 0; it < kFlush; ++it) {
      const int k0 = c * kChunkBins + it * 32;
      if (k0 > kend) break;
      const int k = k0 + lane;
      if (k <= kend) mixed_bin<GRAD, NDET, SPLIT>(sc, P, GlobalBin{ev, K, k}, acc);
    }
    flush<NACC>(acc, hi, lo, lane);
  }
  return any;
}

// Moments of one particle on one warp (the NUTS kernel's sweep). A sweep of
// one chunk (k_ISCO < 2048: every BBH workload here) is its single stream:
// the moments are hi + lo. Longer sweeps take the kStreams streams in order
// and add each stream's hi + lo in FP64: the result the likelihood kernel
// gets from the same streams spread over several warps, bit for bit.
template <bool GRAD, int NDET, bool SPLIT>
__device__ void sweep_mixed(const DevEvent& ev, const SweepCoef& sc, float* mom) {
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  constexpr int NOUT = FlushShape<NACC>::KEEP;
  const int lane = threadIdx.x & 31;
  float hi[NOUT], lo[NOUT];
  float out[NOUT];
  if (sc.kisco < kChunkBins) {
    mixed_stream<GRAD, NDET, SPLIT>(ev, sc, 0, hi, lo);
#pragma unroll
    for (int t = 0; t < NOUT; ++t) out[t] = hi[t] + lo[t];
  } else {
    double tot[NOUT];
#pragma unroll
    for (int t = 0; t < NOUT; ++t) tot[t] = 0.0;
    for (int st = 0; st < kStreams; ++st) {
      if (!mixed_stream<GRAD, NDET, SPLIT>(ev, sc, st, hi, lo)) break;
#pragma unroll
      for (int t = 0; t < NOUT; ++t) tot[t] += (double)hi[t] + (double)lo[t];
    }
#pragma unroll
    for (int t = 0; t < NOUT; ++t) out[t] = (float)tot[t];
  }
  if (FlushShape<NACC>::owner(lane)) {
#pragma unroll
    for (int t = 0; t < NOUT; ++t) {
      const int idx = FlushShape<NACC>::index(lane, t);
      if (idx < NACC) mom[acc_to_mom<NDET, GRAD>(idx)] = out[t];
    }
  }
}

// One stream of the FP64 sweep (chunks c = s, s + kStreams, ... of 2048 bins
// below k_ISCO): per-lane FP64 sums, then the warp reduce-scatter (the same
// pairing as a butterfly sum per moment, with NP/2 + NP/4 + ... FP64 adds per
// lane instead of 5 NP); lane l holds its sums in v. Returns whether the
// stream had any bin.
template <bool GRAD, int NDET>
__device__ bool fp64_stream(const DevEvent& ev, const SweepCoef& sc, int s, double* v_out) {
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  const int lane = threadIdx.x & 31;
  const int64_t K = ev.n_bins;
  double acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.0;
  double al[kNPn];
#pragma unroll
  for (int j = 0; j < kNPn; ++j) al[j] = sc.alpha[j];
  const int kend = sc.kisco;
  bool any = false;
  for (int c = s; c * kChunkBins <= kend; c += kStreams) {
    any = true;
    const int kstop = min(kend, c * kChunkBins + kChunkBins - 1);
    for (int k = c * kChunkBins + lane; k <= kstop; k += 32) {
      double S = sc.c0;
#pragma unroll
      for (int j = 0; j < kNPn; ++j) S = fma(al[j], ev.b64[(int64_t)j * K + k], S);
      const double f = ev.b64[(int64_t)8 * K + k];
      double bf[kNBasis];
      if (GRAD) {
#pragma unroll
        for (int j = 0; j < kNBasis; ++j) bf[j] = ev.b64[(int64_t)j * K + k];
      }
#pragma unroll
      for (int a = 0; a < NDET; ++a) {
        const double P = fma(f, sc.tau[a], S);
        const double r = P - rint(P);
        double sn, cs;
        sincospi(2.0 * r, &sn, &cs);
        const double2 E = ev.e64[(int64_t)a * K + k];
        const double zr = E.x * cs + E.y * sn;
        const double zi = E.y * cs - E.x * sn;
        if (GRAD) {
#pragma unroll
          for (int j = 0; j < kNBasis; ++j) {
            acc[(a * kNMom + j) * 2] += zr * bf[j];
            acc[(a * kNMom + j) * 2 + 1] += zi * bf[j];
          }
          acc[(a * kNMom + 9) * 2] += zr;
          acc[(a * kNMom + 9) * 2 + 1] += zi;
        } else {
          acc[a * 2] += zr;
          acc[a * 2 + 1] += zi;
        }
      }
    }
  }
  using F = FlushShape<NACC>;
  double v[F::NP];
#pragma unroll
  for (int i = 0; i < F::NP; ++i) v[i] = i < NACC ? acc[i] : 0.0;
  ReduceScatter<F::NP, 16, double>::run(v, lane);
#pragma unroll
  for (int t = 0; t < F::KEEP; ++t) v_out[t] = v[t];
  return any;
}

// FP64 moments of one particle on one warp; streams as in sweep_mixed (a
// sweep below 2048 bins is its single stream).
template <bool GRAD, int NDET>
__device__ void sweep_fp64(const DevEvent& ev, const SweepCoef& sc, double* mom) {
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  using F = FlushShape<NACC>;
  const int lane = threadIdx.x & 31;
  double v[F::KEEP], tot[F::KEEP];
  if (sc.kisco < kChunkBins) {
    fp64_stream<GRAD, NDET>(ev, sc, 0, tot);
  } else {
#pragma unroll
    for (int t = 0; t < F::KEEP; ++t) tot[t] = 0.0;
    for (int st = 0; st < kStreams; ++st) {
      if (!fp64_stream<GRAD, NDET>(ev, sc, st, v)) break;
#pragma unroll
      for (int t = 0; t < F::KEEP; ++t) tot[t] += v[t];
    }
  }
  if (F::owner(lane)) {
#pragma unroll
    for (int t = 0; t < F::KEEP; ++t) {
      const int idx = F::index(lane, t);
      if (idx < NACC) mom[acc_to_mom<NDET, GRAD>(idx)] = tot[t];
    }
  }
}

// Moment storage type of each path.
template <int PREC>
struct MomType {
  using type = float;
};
template <>
struct MomType<SHARPY_FP64> {
  using type = double;
};

template <int PREC, bool GRAD, int NDET>
__device__ __forceinline__ void sweep(const DevEvent& ev, const SweepCoef& sc, typename MomType<PREC>::type* mom) {
  if constexpr (PREC == SHARPY_FP64)
    sweep_fp64<GRAD, NDET>(ev, sc, mom);
  else
    sweep_mixed<GRAD, NDET, PREC == SHARPY_MIXED_SPLIT>(ev, sc, mom);
}

}  // namespace sharpy
