/*
 * sharpy — GPU hot path of a Sequential Monte Carlo sampler with a No-U-Turn
 * transition kernel for gravitational-wave inference (arXiv:2601.02336,
 * "The Sequential Monte Carlo goes NUTS").
 *
 * C ABI. Plain pointers and sizes; no C++ or torch types. Every call returns
 * an int status (SHARPY_OK = 0, negative on error), never aborts, never
 * throws, and never synchronises the device except where stated
 * (sharpy_set_data, sharpy_log_evidence, sharpy_get_status, sharpy_smc_run).
 *
 * Memory: arrays are FP64, row-major and contiguous unless stated. Device
 * pointers are owned by the caller and must stay valid until the work queued
 * on `stream` has finished. Tables, scratch and the status word are owned by
 * the context. A context is bound to one device and may be used from one
 * host thread at a time. Calls on one context are stream-ordered; running
 * calls of one context concurrently on different streams is not supported
 * (they share the context's scratch).
 *
 * Parameters theta are the free dimensions of the model ([N][D], D =
 * cfg->n_dim); the physical meaning of dimension i is cfg->phys[i]. Units:
 * chirp mass [Msun], distance [Mpc], times [s], angles [rad].
 */
#ifndef SHARPY_H
#define SHARPY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sharpy_ctx sharpy_ctx;
/* A cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st* sharpy_stream;

enum {
  SHARPY_OK = 0,
  SHARPY_EINVAL = -1,     /* bad argument (null pointer, size, range)          */
  SHARPY_ECUDA = -2,      /* a CUDA runtime call failed                        */
  SHARPY_ENOMEM = -3,     /* device or host allocation failed                  */
  SHARPY_ENONFINITE = -4, /* NaN/Inf in data or PSD, or a non-finite ln L       */
  SHARPY_ETIMEOUT = -5,   /* a device loop hit its iteration bound             */
  SHARPY_EBOUNDS = -6,    /* a device index check failed                       */
  SHARPY_ESTATE = -7      /* call out of order (e.g. no data set yet)          */
};

/* Arithmetic of the likelihood sweep. */
enum {
  SHARPY_FP64 = 0,  /* every per-bin operation in FP64                                     */
  SHARPY_MIXED = 1, /* FP64 PN phase polynomial, FP32 delay term, carrier, inner products  */
  SHARPY_MIXED_SPLIT = 2 /* phase in split single precision (no FP64 in the bin loop), FP32 rest */
};

/* Models. */
enum {
  SHARPY_MODEL_TAYLORF2 = 0, /* Whittle likelihood of a TaylorF2 signal (Sec. 2, Eq. 2) */
  SHARPY_MODEL_GAUSSMIX = 1  /* diagonal Gaussian mixture ln L (test targets, App. A)     */
};

/* Physical parameters of the aligned-spin TaylorF2 model. */
enum {
  SHARPY_MC = 0, SHARPY_Q = 1, SHARPY_CHI1 = 2, SHARPY_CHI2 = 3, SHARPY_DL = 4, SHARPY_COSI = 5,
  SHARPY_PHIC = 6, SHARPY_PSI = 7, SHARPY_RA = 8, SHARPY_SINDEC = 9, SHARPY_TC = 10,
  SHARPY_NPHYS = 11
};

enum { SHARPY_PRIOR_UNIFORM = 0, SHARPY_PRIOR_POWER2 = 1 }; /* density ~ const or ~ x^2 on [lo,hi] */
enum { SHARPY_BOUND_REFLECT = 0, SHARPY_BOUND_PERIODIC = 1 }; /* Sec. 5, "Boundary conditions" */

#define SHARPY_MAX_DIM 11
#define SHARPY_MAX_COMP 4
#define SHARPY_MAX_DET 4
#define SHARPY_MAX_DEPTH 10

/* Model and prior (Sec. 2 Eq. 1; Sec. 5). */
typedef struct {
  int model;                        /* SHARPY_MODEL_*                                   */
  int n_dim;                        /* D, 1..11                                          */
  int phys[SHARPY_MAX_DIM];         /* TaylorF2: physical parameter of free dimension i  */
  double lo[SHARPY_MAX_DIM];        /* prior box [lo, hi]                                */
  double hi[SHARPY_MAX_DIM];
  int prior[SHARPY_MAX_DIM];        /* SHARPY_PRIOR_*                                    */
  int boundary[SHARPY_MAX_DIM];     /* SHARPY_BOUND_*                                    */
  double fixed[SHARPY_NPHYS];       /* TaylorF2: values of the parameters that are not free */
  int n_comp;                       /* GAUSSMIX: ln L = log sum_c exp(logw_c) N(x; mu_c, diag sigma_c^2) */
  double mix_logw[SHARPY_MAX_COMP];
  double mix_mu[SHARPY_MAX_COMP][SHARPY_MAX_DIM];
  double mix_sigma[SHARPY_MAX_COMP][SHARPY_MAX_DIM];
} sharpy_config;

/* Detector on a spherical Earth (GMST = 0). Arms at `azimuth` (clockwise from
   local north) and azimuth + pi/2. fixed_response = 1 uses fplus, fcross and
   delay as given, independent of the sky position and polarisation. */
typedef struct {
  double lat, lon, azimuth;
  int fixed_response;
  double fplus, fcross, delay;
} sharpy_detector;

/* Per-particle NUTS statistics, accumulated over the n_steps transitions of
   one sharpy_nuts_mutate call. */
typedef struct {
  double accept_sum;  /* sum of per-transition mean min(1, exp(-dH))              */
  double active_bins; /* sum over gradient evaluations of the bins below f_ISCO x detectors */
  int depth_sum;      /* sum of tree depths                                         */
  int n_leapfrog;     /* leapfrog steps = likelihood+gradient evaluations           */
  int n_divergent;    /* transitions that stopped on a divergence (dH > 1000)       */
  int pad;
} sharpy_nuts_stats;

/* Full-run options (Sec. 3 and Sec. 6 run settings). */
typedef struct {
  int64_t n_particles;
  double alpha;        /* target ESS fraction, Eq. (6)                               */
  int n_mut;           /* NUTS transitions per stage                                 */
  int max_depth;       /* NUTS tree depth limit (<= SHARPY_MAX_DEPTH)                */
  int metric;          /* 0: identity, step = eps_scale * min_j sigma_j; 1: weighted covariance, step = eps_scale;
                          2: per-particle local metric (sharpy_local_metric at the stage's beta), step = eps_scale */
  double eps_scale;
  int precision;       /* SHARPY_FP64 / SHARPY_MIXED / SHARPY_MIXED_SPLIT            */
  int max_stages;
  int timing;          /* 1: time each stage's NUTS launch with CUDA events (sharpy_stage.nuts_ms) */
  int pad;
  /* Sample-recycling pool (sharpy_smc_run only; NULL: none): after the
     mutation of stage t the N particles are copied to rows (t-1) N .. t N - 1
     of pool_theta [pool_cap][D] and pool_lnl [pool_cap] (device), while they
     fit (stages beyond pool_cap / N are not kept). */
  double* pool_theta;
  double* pool_lnl;
  int64_t pool_cap;
} sharpy_smc_options;

typedef struct {
  double beta, dbeta, ess, dlnz, eps, accept_mean, depth_mean;
  int64_t n_leapfrog;
  int n_divergent;
  int pad;
  double active_bins;  /* sum over the stage's gradient evaluations of (bins below f_ISCO) x detectors */
  double nuts_ms;      /* duration of the stage's NUTS launch (opt->timing = 1), else 0 */
  double reweight_ms;  /* duration of the stage's reweight/resample/gather (opt->timing = 1), else 0 */
  double lnz;          /* ln Z after this stage: the running sum of the increments (Sec. 3.1, Eq. 8),
                          accumulated on the device */
} sharpy_stage;

/* Context. Owns the staged data tables, scratch, the evidence accumulator and
   the sticky status word. cfg is copied. Returns SHARPY_EINVAL for an invalid
   configuration, SHARPY_ECUDA / SHARPY_ENOMEM on device errors. */
int sharpy_create(sharpy_ctx** out, const sharpy_config* cfg, int device);
void sharpy_destroy(sharpy_ctx* ctx);

/* Stage one event (Sec. 2, Eq. 2): frequency grid f_k = f_min + k df,
   k < n_bins; data d[n_det][n_bins][2] (re, im) and one-sided PSD
   psd[n_det][n_bins], both HOST arrays, copied (the caller keeps ownership).
   Builds the noise weights w = 4 df / S, the pre-whitened data, the basis and
   prefix tables and <d|d>. Synchronous. SHARPY_ENONFINITE if d or the PSD has
   a NaN/Inf or the PSD is not positive. A call for a new event on the same
   grid and detector count keeps the grid tables and device buffers (it waits
   for the device, then rebuilds and copies only the data-dependent tables);
   the local-metric tables are kept while the PSD is unchanged. */
int sharpy_set_data(sharpy_ctx* ctx, int n_det, int64_t n_bins, double f_min, double df,
                    const double* d_re_im, const double* psd, const sharpy_detector* det);

/* Prior draws (Philox4x32-10, purpose 1, counter (particle, ctr, 1, dim)). theta: [N][D] device. */
int sharpy_prior_sample(sharpy_ctx* ctx, int64_t n, double* theta, uint64_t key, uint64_t ctr,
                        sharpy_stream stream);
/* ln pi(theta) [N] and grad ln pi [N][D] (glp may be NULL); device arrays.
   Outside the box ln pi = -inf. */
int sharpy_prior_logpdf_grad(sharpy_ctx* ctx, int64_t n, const double* theta, double* lp, double* glp,
                             sharpy_stream stream);

/* Whittle log-likelihood ln L = -1/2 <d-h|d-h> (Sec. 2, Eq. 2) and its
   gradient (Sec. 4: exact derivative, here a hand-written adjoint over
   per-bin moments) at N parameter vectors. theta [N][D], lnl [N],
   grad [N][D] or NULL (forward-only sweep): device arrays. precision:
   SHARPY_FP64 / SHARPY_MIXED / SHARPY_MIXED_SPLIT. The bins of one vector
   are cut into chunks of 2048 dealt to 8 streams that are merged in a fixed
   order, and 1, 2, 4 or 8 warps share a vector's streams. On segments of
   65536 bins or more, SHARPY_MIXED has a fifth choice (16): one vector per
   warp, eight vectors per CTA reading each block of 256 bins' tables from
   shared memory, where one bulk copy brings it (sharpy_set_data lays the
   tables out in such blocks, 28 KB each for three detectors). The first call
   for a (bins, detectors, N, precision, gradient) shape times the choices on
   its own arguments (synchronising `stream`; the outputs do not depend on
   the choice) and the context keeps the fastest; later calls are
   asynchronous. A bulk copy that does not complete within its wait bound
   sets SHARPY_ETIMEOUT in the status word. */
int sharpy_loglike_grad(sharpy_ctx* ctx, int64_t n, const double* theta, double* lnl, double* grad,
                        int precision, sharpy_stream stream);
/* The warps per vector the context picked for sharpy_loglike_grad calls of
   N vectors at `precision` (with_grad: with or without the gradient) on its
   current event's grid; 0 before the first such call. */
int sharpy_loglike_split(sharpy_ctx* ctx, int64_t n, int precision, int with_grad);
/* Use `split` (1, 2, 4 or 8 warps per vector, or 16: the staged kernel of
   segments of at least 65536 bins on the mixed and split paths, which falls
   back to 8 where it does not apply) in every later
   sharpy_loglike_grad call of the context instead of the tuned choice; 0
   returns to tuning. SHARPY_EINVAL for other values. */
int sharpy_set_loglike_split(sharpy_ctx* ctx, int split);
/* Failure-detection tests of the staged kernel (choice 16): its bulk copy of
   table block `skip_block` is left out (-1: none), so the mbarrier waits for
   that block run out, and each wait polls at most `wait_polls` times (0: the
   default bound). A wait that runs out records SHARPY_ETIMEOUT in the status
   word; the kernel issues no further copies, waits (bounded) for the copies in
   flight and returns, and the context stays usable. SHARPY_EINVAL for
   skip_block < -1 or wait_polls < 0. */
int sharpy_set_stage_test_hooks(sharpy_ctx* ctx, int skip_block, int wait_polls);

/* Detector-frame strain h_a(f_k) [N][n_det][n_bins][2] (device) of N
   parameter vectors (used to build injections). FP64. TaylorF2 only. */
int sharpy_waveform(sharpy_ctx* ctx, int64_t n, const double* theta, double* h, sharpy_stream stream);

/* n_steps multinomial NUTS transitions per particle (Sec. 4; Hoffman &
   Gelman 2014) targeting L^beta * pi (Sec. 3, Eq. 3), leapfrog per Sec. 4
   Eqs. (11)-(13), boundary maps per Sec. 5. theta, lnl, grad (grad ln L)
   are updated in place (device). inv_mass: [D][D] device metric, or NULL
   for the identity. step: leapfrog step. max_depth <= SHARPY_MAX_DEPTH.
   Random numbers: Philox4x32-10 keyed by `key`, transition t of particle i
   uses step counter ctr + t. stats: [N] device or NULL. One persistent
   launch; uneven trees are handled on the device. */
int sharpy_nuts_mutate(sharpy_ctx* ctx, int64_t n, double beta, double* theta, double* lnl,
                       double* grad, const double* inv_mass, double step, int max_depth, int n_steps,
                       uint64_t key, uint64_t ctr, int precision, sharpy_nuts_stats* stats,
                       sharpy_stream stream);

/* sharpy_nuts_mutate with the identity metric and the step size of the
   identity-metric runs (Sec. 6 gives step 0.5 for its Hessian metric; with
   an identity mass matrix the step is scaled by the stage's particle spread):
   step = eps_scale * min_j sqrt(cov[j][j]), computed on the device from the
   weighted covariance cov [D][D] (device, e.g. the one
   sharpy_smc_reweight_resample writes), so a host-side stage loop needs no
   readback. SHARPY_EINVAL as sharpy_nuts_mutate, or if cov is NULL or
   eps_scale is not positive and finite. */
int sharpy_nuts_mutate_cov_step(sharpy_ctx* ctx, int64_t n, double beta, double* theta, double* lnl,
                                double* grad, const double* cov, double eps_scale, int max_depth, int n_steps,
                                uint64_t key, uint64_t ctr, int precision, sharpy_nuts_stats* stats,
                                sharpy_stream stream);

/* Failure detection: the persistent NUTS kernel bounds its tick loop (one
   tick = one leapfrog of every slot with a pending evaluation) by
   n_steps (2^max_depth + 1) + 4, which no valid trajectory reaches; on
   reaching the bound it records SHARPY_ETIMEOUT in the status word and writes
   back each particle's current proposal (a point of its trajectory with its
   own ln L and gradient). max_ticks > 0 lowers that bound for the context's
   later NUTS launches (single-event calls and sharpy_smc_run), so that tests
   can drive the bound without a fault; 0 restores the default. SHARPY_EINVAL
   for max_ticks < 0. */
int sharpy_set_nuts_tick_limit(sharpy_ctx* ctx, int64_t max_ticks);

/* NUTS particle slots per CTA (4, 8, 16 or 32) for the context's later
   single-event launches (sharpy_nuts_mutate*, sharpy_smc_run, which then
   skips its slot tuning) instead of the tuned or default choice; 0 returns to
   those. A NUTS result does not depend on the slot count. SHARPY_EINVAL for
   other values. */
int sharpy_set_nuts_slots(sharpy_ctx* ctx, int slots);

/* Particle sharding of one event over several GPUs (one context per GPU,
   Sec. 7 names splitting the particles across devices as the way to scale
   out): the particle arrays given to this context's later prior draws and
   NUTS calls (sharpy_prior_sample, sharpy_nuts_mutate*, and those inside
   sharpy_smc_run) are rows first_id .. first_id + N - 1 of a larger ensemble.
   Row i draws the random numbers of ensemble index first_id + i (the Philox
   counter's particle word), so a shard computes exactly what a single call
   over the whole ensemble computes for those rows. 0 (the default) is an
   unsharded ensemble. SHARPY_EINVAL for first_id outside [0, 2^31). */
int sharpy_set_shard(sharpy_ctx* ctx, int64_t first_id);

/* sharpy_nuts_mutate with one metric per particle (the local metric of
   Sec. 5, e.g. from sharpy_local_metric): inv_mass [N][D][D] = M_i^-1 and
   chol [N][D][D] = L_i lower triangular with L_i L_i^T = M_i^-1 (device,
   FP64), fixed through the call. */
int sharpy_nuts_mutate_local(sharpy_ctx* ctx, int64_t n, double beta, double* theta, double* lnl,
                             double* grad, const double* inv_mass, const double* chol, double step,
                             int max_depth, int n_steps, uint64_t key, uint64_t ctr, int precision,
                             sharpy_nuts_stats* stats, sharpy_stream stream);

/* One tempering step (Sec. 3, Eqs. 4-8): the increment dbeta solving
   ESS = alpha N (the largest FP64-verified dbeta with ESS >= alpha N, within
   1e-12 relative of the root; or dbeta = 1 - beta_prev if that already keeps
   ESS >= alpha N), weights W_i = exp(dbeta (lnL_i - max)),
   dlnz = logsumexp(dbeta lnL) - ln N (also added to the context's ln Z),
   the weighted covariance of theta under W (cov [D][D], or NULL), then
   systematic resampling with uniform u in [0,1) (see
   sharpy_systematic_resample) and the gather of theta, lnl, grad in place.
   beta_next, dlnz, ess: device scalars; ancestors [N] int32 device or NULL.
   N <= 1<<20. */
int sharpy_smc_reweight_resample(sharpy_ctx* ctx, int64_t n, double* theta, double* lnl, double* grad,
                                 double beta_prev, double alpha, double u, double* beta_next,
                                 double* dlnz, double* ess, int32_t* ancestors, double* cov,
                                 sharpy_stream stream);

/* Systematic resampling on integer-quantised weights (bit-exact): W [N] in
   [0,1] (device), q_i = floor(W_i 2^32), C = inclusive prefix sum,
   U = floor(u 2^32), p_m = floor((m 2^32 + U) C_{N-1} / (N 2^32)),
   ancestor(m) = min{ j : C_j > p_m }. anc [N] int32 device. Needs no context.
   SHARPY_EINVAL if u is outside [0,1) or N is outside [1, 1<<20]; also if
   some W_i is outside [0,1] or not finite, in which case the ancestors are
   still written, with that weight taken as 0. An all-zero W is reported
   through ancestors = -1. Synchronises `stream`. */
int sharpy_systematic_resample(int64_t n, const double* w, double u, int32_t* anc, sharpy_stream stream);

/* Allocation-free variant of sharpy_systematic_resample, with the same
   inputs, outputs and results. The paper has no counterpart: this is for
   callers that cannot call cudaMalloc once they are running, for example a
   sampler service that reserves its device memory up front and keeps its
   budget fixed afterwards, or a caller that cannot accept the device-wide
   synchronisation that allocating and freeing can cause. Its scratch (the
   integer prefix sums and an invalid-weight flag) is a fixed device array
   inside the library, sized for N <= 262144 (2 MiB), which every GPU that
   loads the library keeps until the process exits. N above that returns
   SHARPY_EINVAL, as does a weight outside [0,1] (ancestors still written, that
   weight taken as 0); it allocates nothing (no cudaMalloc/cudaFree, no
   allocating library call). Every call looks up the array's device address on
   the current device (a lookup, not an allocation). All calls share the one
   array, which keeps the last call's
   contents (the flag is cleared by each call): calls that overlap on the GPU
   (other streams, other threads) race and must be serialised by the caller.
   Synchronises `stream` (like sharpy_systematic_resample). */
int sharpy_systematic_resample_static(int64_t n, const double* w, double u, int32_t* anc,
                                      sharpy_stream stream);

/* Reset the context's evidence accumulator (ln Z = 0, zero stages). */
int sharpy_reset_evidence(sharpy_ctx* ctx, sharpy_stream stream);
/* Set the context's evidence accumulator to ln Z = lnz after n_stages stages
   (resuming a run from a stage-boundary checkpoint). Synchronises `stream`.
   SHARPY_EINVAL for a non-finite lnz or n_stages < 0. */
int sharpy_set_evidence(sharpy_ctx* ctx, double lnz, int n_stages, sharpy_stream stream);
/* Sum of the evidence increments since the last reset (Sec. 3.1, Eq. 8) and
   the number of stages. Synchronises the context's last stream. */
int sharpy_log_evidence(sharpy_ctx* ctx, double* lnz, int* n_stages);

/* Full SMC run (Sec. 3): prior draw, ln L, then stages of reweight/resample,
   metric and step size, n_mut NUTS transitions, until beta = 1. The stage
   loop runs on the device except for one 8-byte read of beta per stage.
   theta_out [N][D], lnl_out [N]: device or NULL; stages: HOST array of
   opt->max_stages entries or NULL. Returns SHARPY_ETIMEOUT if beta = 1 was
   not reached within max_stages. Synchronous. */
int sharpy_smc_run(sharpy_ctx* ctx, const sharpy_smc_options* opt, uint64_t key, double* lnz,
                   int* n_stages, double* theta_out, double* lnl_out, sharpy_stage* stages,
                   sharpy_stream stream);

/* Batched SMC over many events (Sec. 3 applied to each event independently;
   the paper runs one event at a time). Every event keeps its own tempering
   ladder, particles, metric and evidence; each stage "round" advances all
   events that have not reached beta = 1 with one reweight launch (one
   thread-block cluster per event), one resampling pass and ONE persistent
   NUTS launch over every particle of every event, its CTAs ordered by event
   cost. The round is captured once as a CUDA graph and replayed; the host
   reads the events' active flags every few rounds only.
   events: n_events contexts with data staged (sharpy_set_data), all with the
   same model kind and detector count; n_particles[e]: particles of event e
   (HOST array); opt: alpha, n_mut, max_depth, metric, eps_scale, precision,
   max_stages as in sharpy_smc_run (opt->n_particles and opt->timing are
   ignored). The contexts must outlive the batch and be unsharded
   (sharpy_set_shard 0). Allocates the batch's device
   memory (particles of all events, stage scratch, records). Synchronous. */
typedef struct sharpy_batch sharpy_batch;
typedef struct {
  double lnz;          /* ln Z of the event (Sec. 3.1, Eq. 8)                    */
  double beta;         /* final beta (1 unless max_stages was reached)           */
  double n_leapfrog;   /* leapfrogs (likelihood+gradient evaluations), all stages */
  double active_bins;  /* sum over those evaluations of (bins below f_ISCO) x detectors */
  int n_stages;
  int pad;
} sharpy_batch_result;
int sharpy_batch_create(sharpy_batch** out, sharpy_ctx* const* events, int n_events, const int64_t* n_particles,
                        const sharpy_smc_options* opt);
void sharpy_batch_destroy(sharpy_batch* b);
/* Run every event from its prior draw to beta = 1: event e uses keys[e]
   exactly as sharpy_smc_run(events[e], opt, keys[e]) does, and gives the same
   particles and ln Z bit for bit. results: HOST array [n_events]; rounds:
   HOST, optional (stage rounds replayed). Returns SHARPY_ETIMEOUT if some
   event did not reach beta = 1 within max_stages. Synchronous. */
int sharpy_batch_run(sharpy_batch* b, const uint64_t* keys, sharpy_batch_result* results, int* rounds,
                     sharpy_stream stream);
/* Particles of event e after the last run: theta [N_e][D], lnl [N_e]
   (device, either may be NULL). Stream-ordered. */
int sharpy_batch_particles(sharpy_batch* b, int e, double* theta, double* lnl, sharpy_stream stream);
/* Stage records of event e from the last run (HOST array of `cap` entries;
   *n = stages written). nuts_ms and reweight_ms are 0. Synchronous. */
int sharpy_batch_stages(sharpy_batch* b, int e, sharpy_stage* stages, int cap, int* n);
/* Slot count (particles per NUTS CTA: 4, 8, 16 or 32) the batch's launches
   use, picked by timing each candidate on full mutations of copies of the
   particles at the third stage round of the first run (0 until then; the
   launches use a count derived from the CTA count meanwhile). The results do
   not depend on it. */
int sharpy_batch_slots(sharpy_batch* b);
/* Set the slot count (4, 8, 16 or 32) instead of tuning it; 0 tunes it again on
   the next run. SHARPY_EINVAL for other values. */
int sharpy_batch_set_slots(sharpy_batch* b, int slots);
/* Kernels the last sharpy_batch_run launched: eager launches counted as they
   are enqueued, every graph replay counted by the kernel nodes of the
   captured round. -1 if b is NULL. */
int64_t sharpy_batch_launches(sharpy_batch* b);

/* Per-particle mass matrices (Sec. 5, "Exploitation of local geometry": at the
   start of each SMC iteration every particle gets the Hessian of the tempered
   posterior as its metric, fixed through the mutation). Reading: the
   likelihood part is its Gauss-Newton part beta F(theta), F_jk = <d_j h|d_k h>
   the Fisher information of Eq. (2) (positive semi-definite; the residual
   term of the exact Hessian is dropped), plus the exact prior Hessian
   (2 / d^2 for a prior proportional to d^2) and 12 / width^2 on the diagonal
   (the precision of each uniform box) so that the matrix stays positive
   definite where F is degenerate. Gaussian-mixture models: F = the
   components' precisions weighted by their responsibilities. theta [N][D]
   device; outputs (device, [N][D][D], each may be NULL but not all):
   mass = M, inv_mass = M^-1, chol = L lower triangular with L L^T = M^-1.
   The first call on a TaylorF2 context builds the prefix tables of
   w f^-7/3 B_m B_n it needs (synchronous then; 54 x n_det x n_bins doubles). */
int sharpy_local_metric(sharpy_ctx* ctx, int64_t n, const double* theta, double beta, double* mass,
                        double* inv_mass, double* chol, sharpy_stream stream);

/* Sample recycling (Sec. 5, "Samples recycling"): a pool of m particles
   collected after the mutation of every stage t = 1..T (particle of stage t
   distributed as p_t = L^beta_t pi / Z_t), taken together as draws from the
   mixture (1/T) sum_t p_t. Each gets its importance weight for the final
   target p_T = L pi / Z_T:
     ln w_i = ln L_i - ln Z_T - ln[(1/T) sum_t exp(beta_t ln L_i - ln Z_t)],
   and a rejection step keeps particle i when u_i < w_i / max_j w_j, u_i the
   first 53-bit uniform of Philox4x32-10 (key, counter (i mod 2^32,
   i div 2^32, 7, 0)). theta [m][d], lnl [m]: device; beta [T], lnz_t [T]
   (ln Z at each stage, i.e. the running sum of the stage increments): HOST;
   log_w [m] device or NULL; out_theta [m][d] device or NULL: the kept
   particles in pool order; *n_out (HOST) = number kept. Synchronous.
   SHARPY_EINVAL on sizes out of range or non-finite beta / ln Z_t. */
int sharpy_recycle(int64_t m, int d, int t, const double* theta, const double* lnl, const double* beta,
                   const double* lnz_t, uint64_t key, double* log_w, double* out_theta, int64_t* n_out,
                   sharpy_stream stream);

/* The kernels' random numbers on the host: the two 53-bit uniforms u[2] of
   Philox4x32-10 (Salmon et al. 2011) under `key` at counter (c0, c1, c2, c3).
   The run uses (particle, step, purpose, index) counters with purposes 1
   prior, 2 momentum, 3 direction, 4 leaf, 5 top-level acceptance, 6
   resampling (particle 0, step = stage), 7 recycling. Lets a host-side stage
   loop reproduce sharpy_smc_run (e.g. to checkpoint between stages). */
void sharpy_uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double* u);

/* Measurement helper: FP32 FMA TFLOP/s, FP64 FMA TFLOP/s and SFU sin+cos
   Gop/s of `device` from register-only kernels (out[3], host). Used as the
   roofline denominators of the ALU-bound likelihood sweep. Synchronous. */
int sharpy_probe_peaks(int device, double* out);

/* Sticky device status (synchronises): SHARPY_OK or the first error a kernel
   recorded. sharpy_clear_status resets it. */
int sharpy_get_status(sharpy_ctx* ctx);
int sharpy_clear_status(sharpy_ctx* ctx);
const char* sharpy_error_string(int code);

#ifdef __cplusplus
}
#endif
#endif
