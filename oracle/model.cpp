// Oracle model: Philox, antenna patterns, TaylorF2 waveform, the literal
// Whittle log-likelihood and its gradient, the prior, and the Gaussian
// mixture test targets. TEST INFRASTRUCTURE ONLY (see oracle.h).
#include <cmath>
#include <cstdint>
#include <cstring>

#include "dual.h"
#include "oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace oracle {

// Physical constants (CODATA / IAU nominal values).
const double kPi = 3.14159265358979323846;
const double kTsun = 4.925491025543576e-6;           // G Msun / c^3 [s]
const double kMpcSec = 3.085677581491367e22 / 299792458.0;  // 1 Mpc / c [s]
const double kEarthRadius = 6.371e6;                 // spherical Earth [m]
const double kC = 299792458.0;                       // [m/s]
const double kEulerGamma = 0.57721566490153286061;

// Compensated (Neumaier) running sum; works for double and Dual.
template <class T>
struct NeumaierSum {
  T sum{0.0};
  T comp{0.0};
  void add(const T& x) {
    T t = sum + x;
    if (std::fabs(val(sum)) >= std::fabs(val(x)))
      comp = comp + ((sum - t) + x);
    else
      comp = comp + ((x - t) + sum);
    sum = t;
  }
  T result() const { return sum + comp; }
};

// ---------------------------------------------------------------- Philox
static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c[0], &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c[2], &hi1, &lo1);
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

static inline double u53(uint32_t a, uint32_t b) {
  uint64_t m = ((uint64_t)a << 21) | (uint64_t)(b >> 11);
  return ((double)m + 0.5) * 0x1.0p-53;
}

void uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[2]) {
  uint32_t ctr[4] = {c0, c1, c2, c3};
  uint32_t k[2] = {(uint32_t)key, (uint32_t)(key >> 32)};
  uint32_t x[4];
  philox(ctr, k, x);
  u[0] = u53(x[0], x[1]);
  u[1] = u53(x[2], x[3]);
}

void normal2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[2]) {
  double u[2];
  uniform2(key, c0, c1, c2, c3, u);
  double r = std::sqrt(-2.0 * std::log(u[0]));
  z[0] = r * std::cos(2.0 * kPi * u[1]);
  z[1] = r * std::sin(2.0 * kPi * u[1]);
}

// ------------------------------------------------------- antenna patterns
// Detector tensor D = (x x^T - y y^T)/2 with unit arm vectors in Earth-fixed
// coordinates; polarisation tensors from the wave frame (m, l) rotated by psi;
// F+ = D:e+, Fx = D:ex; delay = -r.n/c.
template <class T>
void antenna_t(const ref_detector* det, const T& ra, const T& sin_dec, const T& psi,
               T* fplus, T* fcross, T* delay) {
  if (det->fixed_response) {
    *fplus = T(det->fplus);
    *fcross = T(det->fcross);
    *delay = T(det->delay);
    return;
  }
  double lat = det->lat, lon = det->lon, az = det->azimuth;
  double east[3] = {-std::sin(lon), std::cos(lon), 0.0};
  double north[3] = {-std::sin(lat) * std::cos(lon), -std::sin(lat) * std::sin(lon), std::cos(lat)};
  double xa[3], ya[3], r[3];
  for (int i = 0; i < 3; ++i) {
    xa[i] = std::cos(az) * north[i] + std::sin(az) * east[i];
    ya[i] = -std::sin(az) * north[i] + std::cos(az) * east[i];
  }
  r[0] = kEarthRadius * std::cos(lat) * std::cos(lon);
  r[1] = kEarthRadius * std::cos(lat) * std::sin(lon);
  r[2] = kEarthRadius * std::sin(lat);
  double D[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = 0.5 * (xa[i] * xa[j] - ya[i] * ya[j]);

  T cos_dec = sqrt(1.0 - sin_dec * sin_dec);
  T n[3] = {cos_dec * cos(ra), cos_dec * sin(ra), sin_dec};
  T p[3] = {sin(ra), -cos(ra), T(0.0)};
  T qv[3] = {n[1] * p[2] - n[2] * p[1], n[2] * p[0] - n[0] * p[2], n[0] * p[1] - n[1] * p[0]};
  T cp = cos(psi), sp = sin(psi);
  T mv[3], lv[3];
  for (int i = 0; i < 3; ++i) {
    mv[i] = p[i] * cp + qv[i] * sp;
    lv[i] = -(p[i] * sp) + qv[i] * cp;
  }
  T fp(0.0), fc(0.0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T ep = mv[i] * mv[j] - lv[i] * lv[j];
      T ec = mv[i] * lv[j] + lv[i] * mv[j];
      fp = fp + ep * D[i][j];
      fc = fc + ec * D[i][j];
    }
  *fplus = fp;
  *fcross = fc;
  *delay = -(n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) / kC;
}

// ---------------------------------------------------------------- TaylorF2
// Stationary-phase TaylorF2 (non-spinning to 3.5PN, aligned-spin spin-orbit
// at 1.5PN and 2.5PN, spin-spin at 2PN), Psi_PN = 3/(128 eta v^5) sum phi_k v^k.
template <class T>
T pn_phase_t(const T& mc, const T& q, const T& chi1, const T& chi2, double f) {
  T eta = q / ((1.0 + q) * (1.0 + q));
  T mtot = mc * pow(eta, -0.6);
  T m1m = 1.0 / (1.0 + q);
  T m2m = q / (1.0 + q);
  T delta = m1m - m2m;
  T chis = 0.5 * (chi1 + chi2);
  T chia = 0.5 * (chi1 - chi2);
  T v = pow(kPi * kTsun * f * mtot, 1.0 / 3.0);
  double vlso = 1.0 / std::sqrt(6.0);

  T beta = (113.0 / 12.0 - 19.0 / 3.0 * eta) * chis + 113.0 / 12.0 * delta * chia;
  T gamma = (732985.0 / 2268.0 - 24260.0 / 81.0 * eta - 340.0 / 9.0 * eta * eta) * chis +
            (732985.0 / 2268.0 + 140.0 / 9.0 * eta) * delta * chia;
  T sigma = 79.0 / 8.0 * eta * chi1 * chi2 + 81.0 / 16.0 * (m1m * m1m * chi1 * chi1 + m2m * m2m * chi2 * chi2);

  T phi0(1.0);
  T phi2 = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
  T phi3 = -16.0 * kPi + 4.0 * beta;
  T phi4 = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * sigma;
  T phi5 = (kPi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) - gamma) * (1.0 + 3.0 * log(v / vlso));
  T phi6 = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi - 6848.0 / 21.0 * kEulerGamma -
           6848.0 / 21.0 * log(4.0 * v) +
           (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) * eta +
           76055.0 / 1728.0 * eta * eta - 127825.0 / 1296.0 * eta * eta * eta;
  T phi7 = kPi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);

  T v2 = v * v;
  T v3 = v2 * v;
  T v4 = v3 * v;
  T v5 = v4 * v;
  T v6 = v5 * v;
  T v7 = v6 * v;
  T series = phi0 + phi2 * v2 + phi3 * v3 + phi4 * v4 + phi5 * v5 + phi6 * v6 + phi7 * v7;
  return 3.0 / (128.0 * eta * v5) * series;
}

template <class T>
T total_mass_t(const T& mc, const T& q) {
  T eta = q / ((1.0 + q) * (1.0 + q));
  return mc * pow(eta, -0.6);
}

template <class T>
T f_isco_t(const T& mc, const T& q) {
  return 1.0 / (std::pow(6.0, 1.5) * kPi * kTsun * total_mass_t(mc, q));
}

// Newtonian amplitude of one polarisation for an optimally oriented source.
template <class T>
T amplitude_t(const T& mc, const T& dl, double f) {
  return std::sqrt(5.0 / 24.0) * std::pow(kPi, -2.0 / 3.0) * pow(kTsun * mc, 5.0 / 6.0) *
         std::pow(f, -7.0 / 6.0) / (dl * kMpcSec);
}

// Map free parameters (as T) to the eleven physical parameters.
template <class T>
void physical(const ref_model* m, const T* free, T* phys) {
  for (int i = 0; i < REF_NPHYS; ++i) phys[i] = T(m->fixed[i]);
  for (int i = 0; i < m->n_dim; ++i) phys[m->phys[i]] = free[i];
}

// h_a(f_k) for one detector and bin; returns false above f_ISCO (h = 0).
template <class T>
struct Projection {
  T fp, fc, dt;
};

template <class T>
bool strain_bin(const T* ph, const Projection<T>& pr, const T& fisco, double f, T* hre, T* him) {
  if (!(f <= val(fisco))) return false;
  T A = amplitude_t(ph[REF_MC], ph[REF_DL], f);
  T psi = 2.0 * kPi * f * ph[REF_TC] - ph[REF_PHIC] - kPi / 4.0 +
          pn_phase_t(ph[REF_MC], ph[REF_Q], ph[REF_CHI1], ph[REF_CHI2], f);
  T phase = psi + 2.0 * kPi * f * pr.dt;
  T ci = ph[REF_COSI];
  // h_+ = A (1 + cos^2 i)/2 e^{-i Psi},  h_x = -i A cos i e^{-i Psi}
  T cre = pr.fp * (1.0 + ci * ci) * 0.5;   // Re(F+ (1+c^2)/2 - i Fx c)
  T cim = -(pr.fc * ci);                    // Im(...)
  T c = cos(phase), s = sin(phase);
  // A (cre + i cim)(cos - i sin)
  *hre = A * (cre * c + cim * s);
  *him = A * (cim * c - cre * s);
  return true;
}

template <class T>
T loglike_gw_t(const ref_model* m, const ref_event* ev, const T* free) {
  T ph[REF_NPHYS];
  physical(m, free, ph);
  T fisco = f_isco_t(ph[REF_MC], ph[REF_Q]);
  NeumaierSum<T> acc;
  for (int a = 0; a < ev->n_det; ++a) {
    Projection<T> pr;
    antenna_t(&ev->det[a], ph[REF_RA], ph[REF_SINDEC], ph[REF_PSI], &pr.fp, &pr.fc, &pr.dt);
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = ev->f_min + (double)k * ev->df;
      double w = 4.0 * ev->df / ev->psd[a * ev->n_bins + k];
      const double* d = ev->data + 2 * (a * ev->n_bins + k);
      T hre(0.0), him(0.0);
      strain_bin(ph, pr, fisco, f, &hre, &him);
      T rre = d[0] - hre;
      T rim = d[1] - him;
      acc.add(w * (rre * rre + rim * rim));
    }
  }
  return -0.5 * acc.result();
}

// Gaussian mixture with diagonal covariances (test targets).
template <class T>
T loglike_mix_t(const ref_model* m, const T* x) {
  T terms[REF_MAX_COMP];
  double best = -INFINITY;
  for (int c = 0; c < m->n_comp; ++c) {
    T s(m->mix_logw[c]);
    for (int i = 0; i < m->n_dim; ++i) {
      double sg = m->mix_sigma[c][i];
      T z = (x[i] - m->mix_mu[c][i]) / sg;
      s = s - 0.5 * z * z - std::log(sg) - 0.5 * std::log(2.0 * kPi);
    }
    terms[c] = s;
    if (val(s) > best) best = val(s);
  }
  T tot(0.0);
  for (int c = 0; c < m->n_comp; ++c) tot = tot + exp(terms[c] - best);
  return log(tot) + best;
}

template <class T>
T loglike_t(const ref_model* m, const ref_event* ev, const T* free) {
  if (m->kind == REF_KIND_GAUSSMIX) return loglike_mix_t(m, free);
  return loglike_gw_t(m, ev, free);
}

template <int N>
void loglike_dual(const ref_model* m, const ref_event* ev, const double* theta, double* lnl, double* grad) {
  DualN<N> x[REF_MAX_DIM];
  for (int i = 0; i < m->n_dim; ++i) x[i] = DualN<N>::variable(theta[i], i);
  DualN<N> r = loglike_t<DualN<N>>(m, ev, x);
  *lnl = r.v;
  for (int i = 0; i < m->n_dim; ++i) grad[i] = r.d[i];
}

// One parameter vector: ln L and optionally its gradient.
void loglike_one(const ref_model* m, const ref_event* ev, const double* theta, double* lnl, double* grad) {
  if (grad == nullptr) {
    double x[REF_MAX_DIM];
    for (int i = 0; i < m->n_dim; ++i) x[i] = theta[i];
    *lnl = loglike_t<double>(m, ev, x);
    return;
  }
  if (m->n_dim <= 2)
    loglike_dual<2>(m, ev, theta, lnl, grad);
  else if (m->n_dim <= 4)
    loglike_dual<4>(m, ev, theta, lnl, grad);
  else
    loglike_dual<REF_MAX_DIM>(m, ev, theta, lnl, grad);
}

// ------------------------------------------------------------------ prior
double prior_logpdf_one(const ref_model* m, const double* x, double* g) {
  double lp = 0.0;
  for (int i = 0; i < m->n_dim; ++i) {
    double lo = m->lo[i], hi = m->hi[i];
    if (g) g[i] = 0.0;
    if (!(x[i] >= lo && x[i] <= hi)) return -INFINITY;
    if (m->prior[i] == REF_PRIOR_POWER2) {
      lp += std::log(3.0 * x[i] * x[i] / (hi * hi * hi - lo * lo * lo));
      if (g) g[i] = 2.0 / x[i];
    } else {
      lp += -std::log(hi - lo);
    }
  }
  return lp;
}

}  // namespace oracle

using namespace oracle;

extern "C" {

void ref_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox(ctr, key, out); }
void ref_uniform2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double u[2]) {
  uniform2(key, c0, c1, c2, c3, u);
}
void ref_normal2(uint64_t key, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, double z[2]) {
  normal2(key, c0, c1, c2, c3, z);
}

void ref_antenna(const ref_detector* det, double ra, double sin_dec, double psi, double* fplus,
                 double* fcross, double* delay) {
  antenna_t<double>(det, ra, sin_dec, psi, fplus, fcross, delay);
}

double ref_pn_phase(double mc, double q, double chi1, double chi2, double f) {
  return pn_phase_t<double>(mc, q, chi1, chi2, f);
}
double ref_pn_phase_dmc(double mc, double q, double chi1, double chi2, double f) {
  DualN<1> m = DualN<1>::variable(mc, 0);
  return pn_phase_t<DualN<1>>(m, DualN<1>(q), DualN<1>(chi1), DualN<1>(chi2), f).d[0];
}
double ref_pn_beta(double q, double chi1, double chi2) {
  double eta = q / ((1 + q) * (1 + q));
  double delta = (1 - q) / (1 + q);
  return (113.0 / 12.0 - 19.0 / 3.0 * eta) * 0.5 * (chi1 + chi2) + 113.0 / 12.0 * delta * 0.5 * (chi1 - chi2);
}
double ref_amplitude(double mc, double dl, double f) { return amplitude_t<double>(mc, dl, f); }
double ref_f_isco(double mc, double q) { return f_isco_t<double>(mc, q); }

int ref_waveform(const ref_model* m, const ref_event* ev, const double* theta, double* h) {
  if (m->kind != REF_KIND_GW) return -1;
  double ph[REF_NPHYS];
  physical(m, theta, ph);
  double fisco = f_isco_t(ph[REF_MC], ph[REF_Q]);
  for (int a = 0; a < ev->n_det; ++a) {
    Projection<double> pr;
    antenna_t(&ev->det[a], ph[REF_RA], ph[REF_SINDEC], ph[REF_PSI], &pr.fp, &pr.fc, &pr.dt);
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = ev->f_min + (double)k * ev->df;
      double hre = 0.0, him = 0.0;
      strain_bin(ph, pr, fisco, f, &hre, &him);
      h[2 * (a * ev->n_bins + k)] = hre;
      h[2 * (a * ev->n_bins + k) + 1] = him;
    }
  }
  return 0;
}

// Fisher information: F_jk = sum_a sum_k w_k Re(conj(dh_j) dh_k), w = 4 df / S,
// with dh the exact derivatives of the strain (dual numbers in every free
// dimension).
static void fisher_one(const ref_model* m, const ref_event* ev, const double* theta, double* F) {
  using T = DualN<REF_MAX_DIM>;
  const int D = m->n_dim;
  T x[REF_MAX_DIM];
  for (int i = 0; i < D; ++i) x[i] = T::variable(theta[i], i);
  T ph[REF_NPHYS];
  physical(m, x, ph);
  T fisco = f_isco_t(ph[REF_MC], ph[REF_Q]);
  for (int i = 0; i < D * D; ++i) F[i] = 0.0;
  for (int a = 0; a < ev->n_det; ++a) {
    Projection<T> pr;
    antenna_t(&ev->det[a], ph[REF_RA], ph[REF_SINDEC], ph[REF_PSI], &pr.fp, &pr.fc, &pr.dt);
    for (int64_t k = 0; k < ev->n_bins; ++k) {
      double f = ev->f_min + (double)k * ev->df;
      double w = 4.0 * ev->df / ev->psd[a * ev->n_bins + k];
      T hre(0.0), him(0.0);
      if (!strain_bin(ph, pr, fisco, f, &hre, &him)) continue;
      for (int j = 0; j < D; ++j)
        for (int l = 0; l < D; ++l) F[j * D + l] += w * (hre.d[j] * hre.d[l] + him.d[j] * him.d[l]);
    }
  }
}

int ref_fisher(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double* fisher) {
  if (m->kind != REF_KIND_GW || !ev) return -1;
  const int D = m->n_dim;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) fisher_one(m, ev, theta + i * D, fisher + i * D * D);
  return 0;
}

int ref_local_metric(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double beta,
                     double* mass) {
  const int D = m->n_dim;
  if (m->kind == REF_KIND_GW) {
    int rc = ref_fisher(m, ev, n, theta, mass);
    if (rc) return rc;
  } else {
    // Gaussian mixture: the components' precisions weighted by their
    // responsibilities at the point (the exact Hessian for one component)
    for (int64_t i = 0; i < n; ++i) {
      const double* x = theta + i * D;
      double* M = mass + i * D * D;
      for (int j = 0; j < D * D; ++j) M[j] = 0.0;
      double lc[REF_MAX_COMP], best = -INFINITY;
      for (int c = 0; c < m->n_comp; ++c) {
        double t = m->mix_logw[c];
        for (int j = 0; j < D; ++j) {
          const double z = (x[j] - m->mix_mu[c][j]) / m->mix_sigma[c][j];
          t += -0.5 * z * z - std::log(m->mix_sigma[c][j]);
        }
        lc[c] = t;
        best = std::fmax(best, t);
      }
      double tot = 0.0;
      for (int c = 0; c < m->n_comp; ++c) tot += std::exp(lc[c] - best);
      for (int c = 0; c < m->n_comp; ++c) {
        const double r = std::exp(lc[c] - best) / tot;
        for (int j = 0; j < D; ++j) M[j * D + j] += r / (m->mix_sigma[c][j] * m->mix_sigma[c][j]);
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) {
    double* M = mass + i * D * D;
    for (int j = 0; j < D * D; ++j) M[j] *= beta;
    for (int j = 0; j < D; ++j) {
      const double w = m->hi[j] - m->lo[j];
      M[j * D + j] += 12.0 / (w * w);
      if (m->prior[j] == REF_PRIOR_POWER2) {
        const double xj = theta[i * D + j];
        M[j * D + j] += 2.0 / (xj * xj);
      }
    }
  }
  return 0;
}

int ref_set_threads(int n) {
#ifdef _OPENMP
  const int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}

int ref_loglike(const ref_model* m, const ref_event* ev, int64_t n, const double* theta, double* lnl,
                double* grad) {
  int D = m->n_dim;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i)
    loglike_one(m, ev, theta + i * D, lnl + i, grad ? grad + i * D : nullptr);
  return 0;
}

int ref_prior_sample(const ref_model* m, int64_t n, double* theta, uint64_t key, uint32_t ctr) {
  int D = m->n_dim;
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < D; ++j) {
      double u[2];
      uniform2(key, (uint32_t)i, ctr, 1u, (uint32_t)j, u);
      double lo = m->lo[j], hi = m->hi[j];
      double x;
      if (m->prior[j] == REF_PRIOR_POWER2)
        x = std::cbrt(lo * lo * lo + u[0] * (hi * hi * hi - lo * lo * lo));
      else
        x = lo + u[0] * (hi - lo);
      theta[i * D + j] = x;
    }
  return 0;
}

int ref_prior_logpdf_grad(const ref_model* m, int64_t n, const double* theta, double* lp, double* glp) {
  int D = m->n_dim;
  for (int64_t i = 0; i < n; ++i) lp[i] = prior_logpdf_one(m, theta + i * D, glp ? glp + i * D : nullptr);
  return 0;
}

}  // extern "C"
