/*
 * Oracle for the SMC-with-NUTS Whittle-likelihood sampler — TEST
 * INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of what the GPU library computes,
 * written from the paper's definitions. Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark load it. It shares no code,
 * header, table or constant with the CUDA library, and the library never
 * loads it.
 *
 * What it follows:
 *   - Whittle log-likelihood, Sec. 2 Eq. (2): ln L = -1/2 <d-h|d-h>,
 *     <a|b> = 4 Re sum_k a_k^* b_k / S_k * df  (the literal sum, all bins).
 *   - Bayes / evidence definitions, Sec. 2 Eq. (1); tempered targets
 *     L^beta * pi, Sec. 3 Eq. (3); reweighting Eq. (4); ESS Eq. (5);
 *     adaptive beta Eq. (6); resampling (Sec. 3 item 2); evidence ratios
 *     Sec. 3.1 Eqs. (7)-(8).
 *   - Hamiltonian, leapfrog, NUTS: Sec. 4 Eqs. (9)-(13) and the NUTS
 *     reference cited there (Hoffman & Gelman 2014), multinomial variant.
 *   - Reflective / periodic boundaries: Sec. 5, "Boundary conditions".
 *   - Waveform: TaylorF2 (3.5PN non-spinning phase, aligned-spin terms to
 *     2.5PN, Newtonian amplitude, cut at f_ISCO), the workload's stand-in
 *     for the paper's IMRPhenomD (Sec. 6).
 *
 * Gradients come from forward-mode dual numbers through the literal
 * per-bin sum (dual.h): exact up to rounding, independent of the GPU
 * library's moment-based adjoint.
 *
 * Parity pins live in tests/ (closed forms, finite differences, analytic
 * evidences, brute force; the PN phase coefficients, sigma included, through
 * the chirp time against the published TaylorT2 series and an energy-balance
 * derivation; the constant phase terms, i.e. the "1" of 1 + 3 ln(v / v_lso)
 * and v_lso, through Psi itself against the stationary-phase transform of the
 * energy-balance orbit with its 2.5PN logarithm referenced at v_lso = 6^-1/2).
 */
#ifndef SHARPY_ORACLE_H
#define SHARPY_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Physical parameters of the aligned-spin model. */
enum {
  REF_MC = 0,     /* chirp mass [Msun] */
  REF_Q = 1,      /* mass ratio m2/m1 in (0, 1] */
  REF_CHI1 = 2,   /* aligned spin of the heavier body */
  REF_CHI2 = 3,   /* aligned spin of the lighter body */
  REF_DL = 4,     /* luminosity distance [Mpc] */
  REF_COSI = 5,   /* cosine of the inclination */
  REF_PHIC = 6,   /* coalescence phase [rad] */
  REF_PSI = 7,    /* polarisation angle [rad] */
  REF_RA = 8,     /* right ascension [rad] (GMST = 0) */
  REF_SINDEC = 9, /* sine of the declination */
  REF_TC = 10,    /* coalescence time [s] */
  REF_NPHYS = 11
};

enum { REF_KIND_GW = 0, REF_KIND_GAUSSMIX = 1 };
enum { REF_PRIOR_UNIFORM = 0, REF_PRIOR_POWER2 = 1 };
enum { REF_BOUND_REFLECT = 0, REF_BOUND_PERIODIC = 1 };

#define REF_MAX_DIM 11
#define REF_MAX_COMP 4
#define REF_MAX_DET 4

typedef struct {
  int kind;                     /* REF_KIND_* */
  int n_dim;                    /* D, free dimensions */
  int phys[REF_MAX_DIM];        /* GW: physical parameter of free dim i */
  double lo[REF_MAX_DIM];       /* prior box */
  double hi[REF_MAX_DIM];
  int prior[REF_MAX_DIM];       /* REF_PRIOR_* */
  int boundary[REF_MAX_DIM];    /* REF_BOUND_* */
  double fixed[REF_NPHYS];      /* GW: value of each non-free parameter */
  /* Gaussian mixture (test targets): ln L = log sum_c w_c N(x; mu_c, diag sigma_c^2) */
  int n_comp;
  double mix_logw[REF_MAX_COMP];
  double mix_mu[REF_MAX_COMP][REF_MAX_DIM];
  double mix_sigma[REF_MAX_COMP][REF_MAX_DIM];
} ref_model;

typedef struct {
  double lat, lon, azimuth;     /* radians; arms at azimuth and azimuth + pi/2 */
  int fixed_response;           /* 1: use fplus, fcross, delay as given */
  double fplus, fcross, delay;
} ref_detector;

typedef struct {
  int n_det;
  int64_t n_bins;
  double f_min, df;             /* f_k = f_min + k * df */
  const double* data;           /* [n_det][n_bins][2] (re, im) */
  const double* psd;            /* [n_det][n_bins] one-sided PSD */
  ref_detector det[REF_MAX_DET];
} ref_event;

typedef struct {
  double accept_sum;            /* sum over transitions of the mean min(1, e^{-dH}) */
  int depth_sum;                /* sum over transitions of the tree depth reached */
  int n_leapfrog;               /* total leapfrog steps (= likelihood+gradient evaluations) */
  int n_divergent;              /* transitions that ended on a divergence */
} ref_nuts_stats;

typedef struct {
  int64_t n_particles;
  double alpha;                 /* target ESS fraction */
  int n_mut;                    /* NUTS transitions per stage */
  int max_depth;
  int metric;                   /* 0: identity, eps = eps_scale * min_j sigma_j; 1: dense weighted covariance, eps = eps_scale;
                                   2: per-particle local metric (ref_local_metric), eps = eps_scale */
  double eps_scale;
  int max_stages;
} ref_smc_opts;

typedef struct {
  double beta, dbeta, ess, dlnz, eps, accept_mean, depth_mean;
  int64_t n_leapfrog;
  int n_divergent;
} ref_stage;

/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers
   0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 / 0xBB67AE85. */
void ref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Two uniforms in (0, 1) with 53-bit resolution from one Philox block. */
void ref_uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[2]);
/* Two standard normals (Box-Muller) from one Philox block. */
void ref_normal2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[2]);

/* Antenna pattern and geocentric delay of one detector for a source at
   (ra, sin_dec) with polarisation psi, GMST = 0. */
void ref_antenna(const ref_detector* det, double ra, double sin_dec, double psi,
                 double* fplus, double* fcross, double* delay);

/* TaylorF2 pieces, exposed for the closed-form pins. */
double ref_pn_phase(double mc, double q, double chi1, double chi2, double f);   /* (3/128 eta v^5) sum phi_k v^k */
double ref_pn_phase_dmc(double mc, double q, double chi1, double chi2, double f); /* d ref_pn_phase / d mc (exact, dual numbers) */
double ref_pn_beta(double q, double chi1, double chi2);                          /* 1.5PN spin-orbit beta */
double ref_amplitude(double mc, double dl, double f);                            /* Newtonian |h~| for an optimal source */
double ref_f_isco(double mc, double q);

/* Detector-frame strain h_a(f_k) of one parameter vector theta (free dims). */
int ref_waveform(const ref_model* m, const ref_event* ev, const double* theta, double* h);

/* Fisher information of the Whittle likelihood (Sec. 2, Eq. 2) at N parameter
   vectors: F_jk = <d_j h | d_k h> = sum_a sum_bins (4 df / S) Re(conj(d_j h) d_k h),
   the derivatives of the strain taken exactly (dual numbers), h = 0 above
   f_ISCO. F: [N][D][D]. (The Gauss-Newton part of -d^2 ln L: the part that
   stays positive semi-definite.) TaylorF2 models only. */
int ref_fisher(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double* fisher);

/* Per-particle mass matrix of Sec. 5 ("Exploitation of local geometry"): the
   Hessian of -ln[L^beta pi] at the particle, with the likelihood part replaced
   by its Gauss-Newton part beta F (positive semi-definite), the prior part
   exact (2 / d^2 for a prior proportional to d^2, 0 for uniform), plus the
   precision 12 / width^2 of each uniform box so that the matrix stays positive
   definite where F is degenerate (beta -> 0). For a Gaussian-mixture model F
   is the components' precisions weighted by their responsibilities at the
   point (the exact Hessian of -ln L for a single component). M: [N][D][D]. */
int ref_local_metric(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double beta,
                     double* mass);

/* Number of OpenMP threads the particle loops use (timing only: every result
   is independent of it). Returns the previous setting. */
int ref_set_threads(int n);

/* ln L (and its gradient if grad != NULL) of N parameter vectors [N][D]. */
int ref_loglike(const ref_model* m, const ref_event* ev, int64_t n, const double* theta,
                double* lnl, double* grad);

/* Prior: draws (Philox purpose 1), log-density and gradient. */
int ref_prior_sample(const ref_model* m, int64_t n, double* theta, uint64_t key, uint32_t ctr);
int ref_prior_logpdf_grad(const ref_model* m, int64_t n, const double* theta, double* lp, double* glp);

/* n_steps NUTS transitions per particle at target L^beta * pi, in place.
   inv_mass: [D][D] or NULL (identity). stats: [N] or NULL. */
int ref_nuts_mutate(const ref_model* m, const ref_event* ev, int64_t n, double beta,
                    double* theta, double* lnl, double* grad, const double* inv_mass,
                    double step, int max_depth, int n_steps, uint64_t key, uint32_t ctr,
                    ref_nuts_stats* stats);

/* As ref_nuts_mutate on n rows of an ensemble: row i is the particle whose
   index in the ensemble is ids[i] (0 <= ids[i] < 2^32), which names its
   random numbers. */
int ref_nuts_mutate_ids(const ref_model* m, const ref_event* ev, int64_t n, const int64_t* ids, double beta,
                        double* theta, double* lnl, double* grad, const double* inv_mass,
                        double step, int max_depth, int n_steps, uint64_t key, uint32_t ctr,
                        ref_nuts_stats* stats);

/* As ref_nuts_mutate with one inverse mass matrix per particle
   (inv_mass [N][D][D]: the local metric of Sec. 5). */
int ref_nuts_mutate_local(const ref_model* m, const ref_event* ev, int64_t n, double beta,
                          double* theta, double* lnl, double* grad, const double* inv_mass,
                          double step, int max_depth, int n_steps, uint64_t key, uint32_t ctr,
                          ref_nuts_stats* stats);
/* The same on n rows of an ensemble, row i being particle ids[i] (as in
   ref_nuts_mutate_ids). */
int ref_nuts_mutate_local_ids(const ref_model* m, const ref_event* ev, int64_t n, const int64_t* ids,
                              double beta, double* theta, double* lnl, double* grad, const double* inv_mass,
                              double step, int max_depth, int n_steps, uint64_t key, uint32_t ctr,
                              ref_nuts_stats* stats);
/* The inverse mass matrices [N][D][D] of ref_smc_run's metric 2 at beta: each
   particle's ref_local_metric, inverted through its Cholesky factor. */
int ref_local_inv_mass(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double beta,
                       double* inv_mass);

/* Adaptive tempering step: beta_next, the incremental weights W (max 1),
   their ESS and the evidence increment dlnz = logsumexp(dbeta lnL) - ln N. */
int ref_smc_reweight(int64_t n, const double* lnl, double beta_prev, double alpha,
                     double* beta_next, double* dlnz, double* ess, double* w);
/* Systematic resampling on integer-quantised weights (bit-exact). */
int ref_systematic_resample(int64_t n, const double* w, double u, int32_t* anc);
/* Weighted mean-centred covariance [D][D]. */
int ref_weighted_cov(int d, int64_t n, const double* theta, const double* w, double* cov);

/* Sample recycling (Sec. 5, "Samples recycling"): a pool of m particles of
   the stages t = 1..T, particle i drawn from p_t(i) = L^beta_t pi / Z_t, stands
   for the mixture p~ = (1/T) sum_t p_t. Its importance weight for the target
   p_T = L pi / Z_T (beta_T = 1) is
     ln w_i = ln L_i - ln Z_T - ln[(1/T) sum_t exp(beta_t ln L_i - ln Z_t)].
   beta[T], lnz_t[T] (ln Z_t = ln Z at beta_t). */
int ref_recycle_weights(int64_t m, int t, const double* lnl, const double* beta, const double* lnz_t,
                        double* log_w);
/* Rejection step of the recycling: particle i is kept when
   u_i < w_i / max_j w_j, u_i the first uniform of Philox4x32-10 (key,
   counter (i mod 2^32, i div 2^32, 7, 0)). keep[m] = 0/1. */
int ref_rejection_sample(int64_t m, const double* log_w, uint64_t key, int32_t* keep);

/* Full SMC run from the prior to beta = 1. */
int ref_smc_run(const ref_model* m, const ref_event* ev, const ref_smc_opts* o, uint64_t key,
                double* lnz, int* n_stages, double* theta_out, double* lnl_out,
                ref_stage* stages);

#ifdef __cplusplus
}
#endif
#endif
