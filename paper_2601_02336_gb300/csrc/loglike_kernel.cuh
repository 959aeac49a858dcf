// The standalone likelihood kernel (sharpy_loglike_grad): one CTA of kWarps
// warps; warp 0 computes the per-particle prologue lane-parallel (lane s =
// particle s of the CTA), the warps sweep the particles' bins, and warp 0
// finishes with the lane-parallel epilogue. The instantiations of each
// precision are compiled in their own unit (loglike_inst.cu).
#pragma once
#include "bulk.cuh"
#include "context.cuh"
#include "split_stage.cuh"
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

// Staged variant for long segments on the mixed and split paths
// (warps-per-vector choice kSplitStaged): one vector per warp, kWarps vectors per CTA walking
// the same bins in step. Each block of kStageBins bins of the tables comes
// into shared memory by one bulk copy (two buffers, each completed on an
// mbarrier) and is read there by all the CTA's vectors, instead of by each
// vector from L2. The blocks are visited in the order of mixed_stream (stream
// s: chunks s, s + kStreams, ...; the 8 blocks of a chunk in order), each
// vector runs mixed_bin on the same bins in the same order and flushes at the
// same chunk ends, and the streams are added in order in FP64: the moments
// equal those of the other choices bit for bit. The split path (SPLIT) reads
// its own records (split_stage.cuh), which carry the lo parts of every basis
// function instead of the FP64 tables.
constexpr int kSplitStaged = 16;

// The walk over the blocks for a CTA whose vectors' last active bin is kmax.
struct StageWalk {
  int kmax, st, c, b;
  __device__ explicit StageWalk(int km) : kmax(km), st(0), c(0), b(0) {}
  __device__ bool valid() const { return st < kStreams && c * kChunkBins + b * kStageBins <= kmax; }
  __device__ int block() const { return c * (kChunkBins / kStageBins) + b; }
  __device__ void next() {
    if (++b < kChunkBins / kStageBins && c * kChunkBins + b * kStageBins <= kmax) return;
    b = 0;
    c += kStreams;
    if (c * kChunkBins <= kmax) return;
    c = ++st;
  }
};

template <bool GRAD, int NDET, bool SPLIT>
__global__ void __launch_bounds__(kWarps * 32, 2)
loglike_staged_kernel(DevModel m, DevEvent ev, int64_t n, const double* __restrict__ theta, double* __restrict__ lnl,
                      double* __restrict__ grad, int* status, int skip_block, int wait_polls) {
  constexpr int NACC = MomCount<NDET, GRAD>::value;
  using FS = FlushShape<NACC>;
  constexpr int NOUT = FS::KEEP;
  constexpr int REC = SPLIT ? split_rec_bytes(NDET) : stage_rec_bytes(NDET);
  using Ld = typename std::conditional<SPLIT, StagedSplitBin, StagedBin>::type;
  const unsigned char* recs = ev.stage + (SPLIT ? split_set_offset(ev.stage_blocks, NDET) : 0);
  extern __shared__ __align__(128) unsigned char stage_buf[];  // two records
  __shared__ __align__(8) uint64_t full[2];
  __shared__ SweepCoef sc[kWarps];
  __shared__ EpiCoef<float> ec[kWarps];
  __shared__ float mom[kWarps][NDET * kNMom * 2];
  __shared__ int kmax_s, abort_s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * kWarps;
  const int D = m.n_dim;
  if (warp == 0 && lane < kWarps) {
    const int64_t p = base + lane;
    if (p < n) {
      double th[kMaxDim];
      for (int i = 0; i < D; ++i) th[i] = theta[p * D + i];
      prologue<float, GRAD, SPLIT>(m, ev, th, sc[lane], ec[lane]);
    } else {
      sc[lane].ok = 0;
      sc[lane].kisco = -1;
    }
  }
  for (int i = lane; i < NDET * kNMom * 2; i += 32) mom[warp][i] = 0.0f;
  if (threadIdx.x == 0) {
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    mbar_fence_init();
    abort_s = 0;
  }
  __syncthreads();
  if (warp == 0) {
    int km = (lane < kWarps && sc[lane].ok) ? sc[lane].kisco : -1;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) km = max(km, __shfl_xor_sync(0xffffffffu, km, o));
    if (lane == 0) kmax_s = km;
  }
  __syncthreads();
  const int kmax = kmax_s;
  const bool live = sc[warp].ok != 0;
  const int kend = live ? sc[warp].kisco : -1;
  MixedCoef<NDET> P;
  if (live) mixed_coef<NDET>(sc[warp], P);
  // the first two blocks; then block i + 2 into the buffer that block i leaves
  StageWalk issue(kmax);
  int issued[2] = {0, 0};  // phases armed per buffer (thread 0)
  // skip_block (failure-detection tests only): that block's copy is left out,
  // so the waits for it run out
  if (threadIdx.x == 0)
    for (int q = 0; q < 2 && issue.valid(); ++q, issue.next()) {
      if (issue.block() == skip_block) continue;
      mbar_arrive_expect_tx(&full[q], REC);
      bulk_copy_g2s(stage_buf + q * REC, recs + (size_t)issue.block() * REC, REC, &full[q]);
      ++issued[q];
    }
  bool timed_out = false;
  float acc[NACC], hi[NOUT], lo[NOUT];
  double tot[NOUT];
#pragma unroll
  for (int t = 0; t < NOUT; ++t) tot[t] = 0.0;
  int i = 0;  // blocks consumed
  for (int st = 0; st < kStreams && st * kChunkBins <= kmax; ++st) {
#pragma unroll
    for (int t = 0; t < NOUT; ++t) hi[t] = lo[t] = 0.0f;
    for (int c = st; c * kChunkBins <= kmax; c += kStreams) {
      const bool mine = c * kChunkBins <= kend;  // a chunk of this vector's sweep
#pragma unroll
      for (int a = 0; a < NACC; ++a) acc[a] = 0.0f;
      for (int b = 0; b < kChunkBins / kStageBins && c * kChunkBins + b * kStageBins <= kmax; ++b, ++i) {
        const int buf = i & 1;
        if (!timed_out && !mbar_wait(&full[buf], (uint32_t)(i >> 1) & 1u, wait_polls)) {
          timed_out = true;
          abort_s = 1;
        }
        const unsigned char* rec = stage_buf + buf * REC;
        if (mine && !timed_out) {
          for (int u = 0; u < kStageBins / 32; ++u) {
            const int k0 = c * kChunkBins + b * kStageBins + u * 32;
            if (k0 > kend) break;
            const int k = k0 + lane;
            if (k <= kend) mixed_bin<GRAD, NDET, SPLIT>(sc[warp], P, Ld{rec, u * 32 + lane}, acc);
          }
        }
        __syncthreads();  // every warp is done with this buffer
        if (threadIdx.x == 0 && issue.valid() && !abort_s) {
          if (issue.block() != skip_block) {
            mbar_arrive_expect_tx(&full[buf], REC);
            bulk_copy_g2s(stage_buf + buf * REC, recs + (size_t)issue.block() * REC, REC, &full[buf]);
            ++issued[buf];
          }
          issue.next();
        }
      }
      if (mine) flush<NACC>(acc, hi, lo, lane);
    }
    if (st * kChunkBins <= kend)
#pragma unroll
      for (int t = 0; t < NOUT; ++t) tot[t] += (double)hi[t] + (double)lo[t];
  }
  if (timed_out) set_status(status, SHARPY_ETIMEOUT);
  // after a timeout, wait (bounded, with the full bound whatever wait_polls
  // says) for the copies still in flight before the CTA's shared memory goes
  // away: they were all issued, in bounds, so they land
  __syncthreads();
  if (threadIdx.x == 0 && abort_s)
    for (int q = 0; q < 2; ++q)
      if (issued[q] > 0) mbar_wait(&full[q], (uint32_t)(issued[q] - 1) & 1u, kMbarWaitPolls);
  if (live && FS::owner(lane)) {
#pragma unroll
    for (int t = 0; t < NOUT; ++t) {
      const int idx = FS::index(lane, t);
      if (idx < NACC) mom[warp][acc_to_mom<NDET, GRAD>(idx)] = (float)tot[t];
    }
  }
  __syncthreads();
  if (warp == 0 && lane < kWarps) {
    const int64_t q = base + lane;
    if (q < n) {
      double l = NAN, gph[SHARPY_NPHYS];
      if (sc[lane].ok) epilogue<float, GRAD>(ev, sc[lane], ec[lane], mom[lane], &l, gph);
      lnl[q] = l;
      bool fin = isfinite(l);
      if (GRAD) {
        for (int d = 0; d < D; ++d) {
          const double g = sc[lane].ok ? gph[m.phys[d]] : NAN;
          grad[q * D + d] = g;
          fin = fin && isfinite(g);
        }
      }
      if (!fin) set_status(status, SHARPY_ENONFINITE);
    }
  }
}

template <bool GRAD, int NDET, bool SPLIT>
inline cudaError_t launch_ll_staged(sharpy_ctx* c, int64_t n, const double* th, double* lnl, double* grad,
                                    cudaStream_t s) {
  constexpr int bytes = 2 * (SPLIT ? split_rec_bytes(NDET) : stage_rec_bytes(NDET));
  const cudaError_t e = cudaFuncSetAttribute(loglike_staged_kernel<GRAD, NDET, SPLIT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  loglike_staged_kernel<GRAD, NDET, SPLIT><<<(unsigned)((n + kWarps - 1) / kWarps), kWarps * 32, bytes, s>>>(
      c->model, c->ev, n, th, lnl, grad, c->d_status, c->stage_skip_block,
      c->stage_wait_polls > 0 ? c->stage_wait_polls : kMbarWaitPolls);
  return cudaGetLastError();
}

// Defined in loglike_staged.cu and loglike_staged_split.cu (units of their own).
cudaError_t launch_ll_staged_unit(sharpy_ctx* c, bool grad, int ndet, int64_t n, const double* th, double* lnl,
                                  double* g, cudaStream_t s);
cudaError_t launch_ll_staged_split_unit(sharpy_ctx* c, bool grad, int ndet, int64_t n, const double* th, double* lnl,
                                        double* g, cudaStream_t s);

template <int PREC, bool GRAD, int NDET, int SPLIT>
inline void launch_ll_one(sharpy_ctx* c, int64_t n, const double* th, double* lnl, double* grad, cudaStream_t s) {
  constexpr int PPC = kWarps / SPLIT;
  dim3 grid((unsigned)((n + PPC - 1) / PPC));
  loglike_kernel<PREC, GRAD, NDET, SPLIT><<<grid, kWarps * 32, 0, s>>>(c->model, c->ev, n, th, lnl, grad, c->d_status);
}

template <int PREC, bool GRAD, int NDET>
inline cudaError_t launch_ll_split(sharpy_ctx* c, int split, int64_t n, const double* th, double* lnl, double* grad,
                                   cudaStream_t s) {
  if (split == kSplitStaged) {
    if constexpr (PREC == SHARPY_MIXED) {
      if (c->ev.stage) return launch_ll_staged_unit(c, GRAD, NDET, n, th, lnl, grad, s);
    }
    if constexpr (PREC == SHARPY_MIXED_SPLIT) {
      if (c->ev.stage) return launch_ll_staged_split_unit(c, GRAD, NDET, n, th, lnl, grad, s);
    }
    split = 8;  // no staged tables, or the FP64 path: the 8-warp split
  }
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
