// The standalone likelihood kernel (sharpy_loglike_grad): one CTA of kWarps
// warps; warp 0 computes the per-particle prologue lane-parallel (lane s =
// particle s of the CTA), the warps sweep the particles' bins, and warp 0
// finishes with the lane-parallel epilogue. The instantiations of each
// precision are compiled in their own unit (loglike_inst.cu).
#pragma once
#include "context.cuh"
#include "sweep.cuh"

namespace sharpy {

constexpr int kWarps = 8;

// SPLIT warps share each particle's sweep (kWarps / SPLIT particles per CTA):
// warp r of a particle computes the streams r, r + SPLIT, ... of the fixed
// stream decomposition (sweep.cuh), stores each stream's sums in shared
// memory, and the particle's first warp merges them in stream order. The
// moments, hence ln L and the gradient, do not depend on SPLIT, which the
// call's autotuner picks per (bins, detectors, particles, precision).
template <int PREC, bool GRAD, int NDET, int SPLIT>
__global__ void __launch_bounds__(kWarps * 32)
loglike_kernel(DevModel m, DevEvent ev, int64_t n, const double* __restrict__ theta, double* __restrict__ lnl,
               double* __restrict__ grad, int* status) {
  using DT = typename std::conditional<PREC == SHARPY_FP64, double, float>::type;
  constexpr int PPC = kWarps / SPLIT;  // particles per CTA
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  using FS = FlushShape<NACC>;
  __shared__ SweepCoef sc[PPC];
  __shared__ EpiCoef<DT> ec[PPC];
  using MT = typename MomType<PREC>::type;
  __shared__ MT mom[PPC][NDET * kNMom * 2];
  // per-stream sums (SPLIT > 1): [particle][stream][32 lanes x KEEP]
  __shared__ double part[SPLIT > 1 ? PPC : 1][SPLIT > 1 ? kStreams : 1][SPLIT > 1 ? 32 * FS::KEEP : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * PPC;
  const int D = m.n_dim;
  if (warp == 0 && lane < PPC) {
    int64_t p = base + lane;
    if (p < n) {
      double th[kMaxDim];
      for (int i = 0; i < D; ++i) th[i] = theta[p * D + i];
      prologue<DT, GRAD, PREC == SHARPY_MIXED_SPLIT>(m, ev, th, sc[lane], ec[lane]);
    } else {
      sc[lane].ok = 0;
      sc[lane].kisco = -1;
    }
  }
  __syncthreads();
  const int pl = warp / SPLIT, r = warp % SPLIT;
  const int64_t p = base + pl;
  if (SPLIT == 1) {
    MT* mw = mom[pl];
    for (int i = lane; i < NDET * kNMom * 2; i += 32) mw[i] = MT(0);
    __syncwarp();
    if (p < n && sc[pl].ok) sweep<PREC, GRAD, NDET>(ev, sc[pl], mw);
  } else {
    if (r == 0)
      for (int i = lane; i < NDET * kNMom * 2; i += 32) mom[pl][i] = MT(0);
    const bool live = p < n && sc[pl].ok;
    for (int st = r; st < kStreams; st += SPLIT) {
      double v[FS::KEEP];
      if (PREC == SHARPY_FP64) {
        if (live) {
          fp64_stream<GRAD, NDET>(ev, sc[pl], st, v);
        } else {
#pragma unroll
          for (int t = 0; t < FS::KEEP; ++t) v[t] = 0.0;
        }
      } else {
        float hi[FS::KEEP], lo[FS::KEEP];
#pragma unroll
        for (int t = 0; t < FS::KEEP; ++t) hi[t] = lo[t] = 0.0f;
        if (live) mixed_stream<GRAD, NDET, PREC == SHARPY_MIXED_SPLIT>(ev, sc[pl], st, hi, lo);
#pragma unroll
        for (int t = 0; t < FS::KEEP; ++t) v[t] = (double)hi[t] + (double)lo[t];
      }
#pragma unroll
      for (int t = 0; t < FS::KEEP; ++t) part[pl][st][lane * FS::KEEP + t] = v[t];
    }
    __syncthreads();
    if (r == 0 && FS::owner(lane)) {
#pragma unroll
      for (int t = 0; t < FS::KEEP; ++t) {
        double tot = 0.0;
        for (int st = 0; st < kStreams; ++st) tot += part[pl][st][lane * FS::KEEP + t];
        const int idx = FS::index(lane, t);
        if (idx < NACC) mom[pl][acc_to_mom<NDET, GRAD>(idx)] = (MT)tot;
      }
    }
  }
  __syncthreads();
  if (warp == 0 && lane < PPC) {
    int64_t q = base + lane;
    if (q < n) {
      double l = NAN, gph[SHARPY_NPHYS];
      if (sc[lane].ok) epilogue<DT, GRAD>(ev, sc[lane], ec[lane], mom[lane], &l, gph);
      lnl[q] = l;
      bool fin = isfinite(l);
      if (GRAD) {
        for (int i = 0; i < D; ++i) {
          double g = sc[lane].ok ? gph[m.phys[i]] : NAN;
          grad[q * D + i] = g;
          fin = fin && isfinite(g);
        }
      }
      if (!fin) set_status(status, SHARPY_ENONFINITE);
    }
  }
}

template <int PREC, bool GRAD, int NDET, int SPLIT>
inline void launch_ll_one(sharpy_ctx* c, int64_t n, const double* th, double* lnl, double* grad, cudaStream_t s) {
  constexpr int PPC = kWarps / SPLIT;
  dim3 grid((unsigned)((n + PPC - 1) / PPC));
  loglike_kernel<PREC, GRAD, NDET, SPLIT><<<grid, kWarps * 32, 0, s>>>(c->model, c->ev, n, th, lnl, grad, c->d_status);
}

template <int PREC, bool GRAD, int NDET>
inline cudaError_t launch_ll_split(sharpy_ctx* c, int split, int64_t n, const double* th, double* lnl, double* grad,
                                   cudaStream_t s) {
  switch (split) {
    case 2: launch_ll_one<PREC, GRAD, NDET, 2>(c, n, th, lnl, grad, s); break;
    case 4: launch_ll_one<PREC, GRAD, NDET, 4>(c, n, th, lnl, grad, s); break;
    case 8: launch_ll_one<PREC, GRAD, NDET, 8>(c, n, th, lnl, grad, s); break;
    default: launch_ll_one<PREC, GRAD, NDET, 1>(c, n, th, lnl, grad, s); break;
  }
  return cudaGetLastError();
}

template <int PREC, bool GRAD>
inline cudaError_t launch_ll_det(sharpy_ctx* c, int split, int64_t n, const double* th, double* lnl, double* grad,
                                 cudaStream_t s) {
  switch (c->ev.n_det) {
    case 1: return launch_ll_split<PREC, GRAD, 1>(c, split, n, th, lnl, grad, s);
    case 2: return launch_ll_split<PREC, GRAD, 2>(c, split, n, th, lnl, grad, s);
    default: return launch_ll_split<PREC, GRAD, 3>(c, split, n, th, lnl, grad, s);
  }
}

// Defined by the three compilations of loglike_inst.cu (one per precision).
cudaError_t launch_ll_p0(sharpy_ctx* c, bool grad, int split, int64_t n, const double* th, double* lnl, double* g,
                         cudaStream_t s);
cudaError_t launch_ll_p1(sharpy_ctx* c, bool grad, int split, int64_t n, const double* th, double* lnl, double* g,
                         cudaStream_t s);
cudaError_t launch_ll_p2(sharpy_ctx* c, bool grad, int split, int64_t n, const double* th, double* lnl, double* g,
                         cudaStream_t s);

}  // namespace sharpy
