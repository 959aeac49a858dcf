// Per-particle prologue and epilogue of the likelihood sweep.
//
// The TaylorF2 phase in turns is written over a fixed basis of frequency
// functions, Psi_a(f)/(2 pi) = sum_j alpha_j B_j(f) + f tau_a + c0, with
// B = {x^5, x^3, x^2, x, ln f, y, y ln f, y^2}, x = f^-1/3, y = f^1/3,
// tau_a = t_c + delay_a. The prologue turns theta into (alpha, tau, c0,
// amplitude A0, complex response C_a, k_ISCO) and their Jacobians; the sweep
// accumulates the moments Z_a = sum_k E_ak e^{-i Psi_ak} and
// Y_aj = sum_k E_ak e^{-i Psi_ak} B_j(f_k) below f_ISCO; the epilogue assembles
//   ln L = sum_a [Re(G_a Z_a) - |G_a|^2 P_a(k_ISCO)/2] - <d|d>/2,  G_a = A0 C_a,
// (Sec. 2, Eq. 2 with the Newtonian amplitude: <h|h> comes from the prefix
// table P_a of w f^-7/3) and the exact gradient by the chain rule through the
// moments (the adjoint of the sweep; the paper gets it by autodiff, Sec. 4).
#pragma once
#include "common.cuh"

namespace sharpy {

// Value (FP64) with derivatives along four directions (type DT).
template <class DT>
struct I4 {
  double v;
  DT d[4];
  __device__ __forceinline__ I4() {}
  __device__ __forceinline__ I4(double x) : v(x) {
#pragma unroll
    for (int i = 0; i < 4; ++i) d[i] = DT(0);
  }
  __device__ __forceinline__ static I4 var(double x, int i) {
    I4 r(x);
    r.d[i] = DT(1);
    return r;
  }
};
template <class DT>
__device__ __forceinline__ I4<DT> chain(const I4<DT>& x, double fv, double fp) {
  I4<DT> r;
  r.v = fv;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = DT(fp) * x.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator+(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator-(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator*(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] * DT(b.v) + DT(a.v) * b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator*(double s, const I4<DT>& a) {
  I4<DT> r;
  r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = DT(s) * a.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator+(double s, const I4<DT>& a) {
  I4<DT> r = a;
  r.v = s + a.v;
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> recip(const I4<DT>& a) {
  double iv = 1.0 / a.v;
  return chain(a, iv, -iv * iv);
}
template <class DT>
__device__ __forceinline__ I4<DT> ipow(const I4<DT>& a, double p) {  // a^p, a > 0
  double y = pow(a.v, p);
  return chain(a, y, p * y / a.v);
}
template <class DT>
__device__ __forceinline__ I4<DT> ilog(const I4<DT>& a) {
  return chain(a, log(a.v), 1.0 / a.v);
}

// Everything the sweep needs for one particle (kept in shared memory).
struct SweepCoef {
  double alpha[kNPn];   // phase basis coefficients [turns]
  double c0;            // constant phase [turns]
  double tau[kMaxDet];  // t_c + delay_a [s]
  int kisco;            // last bin with f_k <= f_ISCO (-1: none)
  int ok;               // 0 if the parameters are outside the model's domain
};

// Everything the epilogue needs beyond the moments.
template <class DT>
struct EpiCoef {
  double A0;
  double cre[kMaxDet], cim[kMaxDet];
  DT dalpha[kNPn][4];           // d alpha_j / d(Mc, q, chi1, chi2)
  DT dc0[4];
  DT dA0_mc, dA0_dl;
  DT dcre[kMaxDet][4], dcim[kMaxDet][4];  // d C_a / d(cos i, psi, ra, sin dec)
  DT dtau[kMaxDet][2];                     // d tau_a / d(ra, sin dec)
};

// Map the free parameters of one particle onto the eleven physical ones.
__device__ __forceinline__ void to_physical(const DevModel& m, const double* th, double* ph) {
#pragma unroll
  for (int i = 0; i < SHARPY_NPHYS; ++i) ph[i] = m.fixed[i];
  for (int i = 0; i < m.n_dim; ++i) ph[m.phys[i]] = th[i];
}

// TaylorF2 phase coefficients in turns and their Jacobian w.r.t. (Mc, q, chi1, chi2).
template <class DT>
__device__ void pn_coefficients(const double* ph, I4<DT>* alpha, I4<DT>& cpn, I4<DT>& mtot) {
  I4<DT> mc = I4<DT>::var(ph[SHARPY_MC], 0);
  I4<DT> q = I4<DT>::var(ph[SHARPY_Q], 1);
  I4<DT> c1 = I4<DT>::var(ph[SHARPY_CHI1], 2);
  I4<DT> c2 = I4<DT>::var(ph[SHARPY_CHI2], 3);
  I4<DT> onepq = 1.0 + q;
  I4<DT> m1 = recip(onepq);        // m1 / M
  I4<DT> m2 = q * m1;              // m2 / M
  I4<DT> eta = m1 * m2;
  I4<DT> delta = m1 - m2;
  mtot = mc * ipow(eta, -0.6);
  I4<DT> u = ipow((kPi * kTsun) * mtot, 1.0 / 3.0);   // v = u f^(1/3)
  I4<DT> lnu = ilog(u);
  I4<DT> chis = 0.5 * (c1 + c2);
  I4<DT> chia = 0.5 * (c1 - c2);
  I4<DT> eta2 = eta * eta;
  // spin-orbit (1.5PN, 2.5PN) and spin-spin (2PN) combinations
  I4<DT> beta = ((113.0 / 12.0) + (-19.0 / 3.0) * eta) * chis + (113.0 / 12.0) * (delta * chia);
  I4<DT> gam = ((732985.0 / 2268.0) + (-24260.0 / 81.0) * eta + (-340.0 / 9.0) * eta2) * chis +
               ((732985.0 / 2268.0) + (140.0 / 9.0) * eta) * (delta * chia);
  I4<DT> sig = (79.0 / 8.0) * (eta * (c1 * c2)) + (81.0 / 16.0) * (m1 * m1 * c1 * c1 + m2 * m2 * c2 * c2);
  I4<DT> p2 = (3715.0 / 756.0) + (55.0 / 9.0) * eta;
  I4<DT> p3 = (-16.0 * kPi) + 4.0 * beta;
  I4<DT> p4 = (15293365.0 / 508032.0) + (27145.0 / 504.0) * eta + (3085.0 / 72.0) * eta2 + (-10.0) * sig;
  I4<DT> p5 = (kPi * 38645.0 / 756.0) + (-kPi * 65.0 / 9.0) * eta - gam;
  I4<DT> p6 = (11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi - 6848.0 / 21.0 * kEulerGamma) +
              (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) * eta + (76055.0 / 1728.0) * eta2 +
              (-127825.0 / 1296.0) * (eta2 * eta);
  I4<DT> p7 = kPi * ((77096675.0 / 254016.0) + (378515.0 / 1512.0) * eta + (-74045.0 / 756.0) * eta2);
  I4<DT> nt = (3.0 / (128.0 * kTwoPi)) * recip(eta);   // 3 / (128 eta) in turns
  I4<DT> ui = recip(u);
  I4<DT> ui2 = ui * ui;
  I4<DT> ui3 = ui2 * ui;
  alpha[0] = nt * (ui3 * ui2);                        // x^5
  alpha[1] = nt * (p2 * ui3);                         // x^3
  alpha[2] = nt * (p3 * ui2);                         // x^2
  alpha[3] = nt * (p4 * ui);                          // x
  alpha[4] = nt * p5;                                 // ln f
  I4<DT> l4u = ilog(4.0 * u);
  alpha[5] = nt * (u * (p6 + (-6848.0 / 21.0) * l4u));  // y
  alpha[6] = (-6848.0 / 63.0) * (nt * u);               // y ln f
  alpha[7] = nt * (p7 * (u * u));                       // y^2
  // constant: p5 (1 + 3 ln(u / v_lso)), v_lso = 6^(-1/2)
  cpn = nt * (p5 * ((1.0 + 1.5 * 1.791759469228055) + 3.0 * lnu));
}

// Antenna pattern, delay and their derivatives w.r.t. (psi, ra, sin dec).
struct Antenna {
  double fp, fc, dt;
  double dfp[3], dfc[3];  // d/d(psi, ra, sin dec)
  double ddt[2];          // d/d(ra, sin dec)
};

__device__ __forceinline__ double quad(const double D[3][3], const double* a, const double* b) {
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s += a[i] * D[i][j] * b[j];
  return s;
}

static __device__ void antenna(const DevDetector& det, double ra, double sdec, double psi, Antenna& out) {
  if (det.fixed_response) {
    out.fp = det.fplus;
    out.fc = det.fcross;
    out.dt = det.delay;
    for (int i = 0; i < 3; ++i) out.dfp[i] = out.dfc[i] = 0.0;
    out.ddt[0] = out.ddt[1] = 0.0;
    return;
  }
  double sa, ca, s2, c2;
  sincos(ra, &sa, &ca);
  sincos(2.0 * psi, &s2, &c2);
  double cd = sqrt(fmax(1.0 - sdec * sdec, 0.0));
  double n[3] = {cd * ca, cd * sa, sdec};
  double p[3] = {sa, -ca, 0.0};
  double q[3] = {sdec * ca, sdec * sa, -cd};
  double dp_ra[3] = {ca, sa, 0.0};
  double dq_ra[3] = {-sdec * sa, sdec * ca, 0.0};
  double dq_sd[3] = {ca, sa, sdec / cd};
  double dn_ra[3] = {-cd * sa, cd * ca, 0.0};
  double dn_sd[3] = {-sdec * ca / cd, -sdec * sa / cd, 1.0};
  double fp0 = quad(det.D, p, p) - quad(det.D, q, q);
  double fc0 = 2.0 * quad(det.D, p, q);
  double dfp0_ra = 2.0 * quad(det.D, p, dp_ra) - 2.0 * quad(det.D, q, dq_ra);
  double dfc0_ra = 2.0 * (quad(det.D, dp_ra, q) + quad(det.D, p, dq_ra));
  double dfp0_sd = -2.0 * quad(det.D, q, dq_sd);
  double dfc0_sd = 2.0 * quad(det.D, p, dq_sd);
  out.fp = c2 * fp0 + s2 * fc0;
  out.fc = -s2 * fp0 + c2 * fc0;
  out.dfp[0] = 2.0 * out.fc;
  out.dfc[0] = -2.0 * out.fp;
  out.dfp[1] = c2 * dfp0_ra + s2 * dfc0_ra;
  out.dfc[1] = -s2 * dfp0_ra + c2 * dfc0_ra;
  out.dfp[2] = c2 * dfp0_sd + s2 * dfc0_sd;
  out.dfc[2] = -s2 * dfp0_sd + c2 * dfc0_sd;
  const double* r = det.r;
  out.dt = -(r[0] * n[0] + r[1] * n[1] + r[2] * n[2]) / kClight;
  out.ddt[0] = -(r[0] * dn_ra[0] + r[1] * dn_ra[1] + r[2] * dn_ra[2]) / kClight;
  out.ddt[1] = -(r[0] * dn_sd[0] + r[1] * dn_sd[1] + r[2] * dn_sd[2]) / kClight;
}

// Last bin with f_k <= f_isco, using the staged frequency table.
__device__ __forceinline__ int isco_bin(const DevEvent& ev, double fisco) {
  int64_t K = ev.n_bins;
  double t = floor((fisco - ev.f_min) / ev.df);
  int64_t k = t < -1.0 ? -1 : (t > (double)(K - 1) ? K - 1 : (int64_t)t);
  while (k + 1 < K && ev.f[k + 1] <= fisco) ++k;
  while (k >= 0 && ev.f[k] > fisco) --k;
  return (int)k;
}

// theta (free dims) -> sweep and epilogue coefficients.
template <class DT, bool GRAD>
__device__ void prologue(const DevModel& m, const DevEvent& ev, const double* th, SweepCoef& sc,
                         EpiCoef<DT>& ec) {
  double ph[SHARPY_NPHYS];
  to_physical(m, th, ph);
  sc.ok = (ph[SHARPY_MC] > 0.0 && ph[SHARPY_Q] > 0.0 && ph[SHARPY_DL] > 0.0 && fabs(ph[SHARPY_SINDEC]) <= 1.0 &&
           fabs(ph[SHARPY_COSI]) <= 1.0) ? 1 : 0;
  if (!sc.ok) {
    sc.kisco = -1;
    return;
  }
  I4<DT> alpha[kNPn], cpn, mtot;
  pn_coefficients<DT>(ph, alpha, cpn, mtot);
#pragma unroll
  for (int j = 0; j < kNPn; ++j) {
    sc.alpha[j] = alpha[j].v;
    if (GRAD)
#pragma unroll
      for (int i = 0; i < 4; ++i) ec.dalpha[j][i] = alpha[j].d[i];
  }
  sc.c0 = cpn.v - ph[SHARPY_PHIC] / kTwoPi - 0.125;
  if (GRAD)
#pragma unroll
    for (int i = 0; i < 4; ++i) ec.dc0[i] = cpn.d[i];
  double fisco = 1.0 / (14.696938456699069 * kPi * kTsun * mtot.v);  // 6^(3/2) pi M
  sc.kisco = isco_bin(ev, fisco);

  // Newtonian amplitude of an optimally oriented source: sqrt(5/24) pi^(-2/3) (T Mc)^(5/6) / D
  double mc = ph[SHARPY_MC], dl = ph[SHARPY_DL];
  ec.A0 = 0.45643546458763845 * 0.46619407703541166 * pow(kTsun * mc, 5.0 / 6.0) / (dl * kMpcSec);
  if (GRAD) {
    ec.dA0_mc = DT(5.0 / 6.0 * ec.A0 / mc);
    ec.dA0_dl = DT(-ec.A0 / dl);
  }
  double ci = ph[SHARPY_COSI];
  for (int a = 0; a < ev.n_det; ++a) {
    Antenna an;
    antenna(ev.det[a], ph[SHARPY_RA], ph[SHARPY_SINDEC], ph[SHARPY_PSI], an);
    sc.tau[a] = ph[SHARPY_TC] + an.dt;
    double hp = 0.5 * (1.0 + ci * ci);
    ec.cre[a] = an.fp * hp;
    ec.cim[a] = -an.fc * ci;
    if (GRAD) {
      ec.dcre[a][0] = DT(an.fp * ci);
      ec.dcim[a][0] = DT(-an.fc);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ec.dcre[a][k + 1] = DT(an.dfp[k] * hp);
        ec.dcim[a][k + 1] = DT(-an.dfc[k] * ci);
      }
      ec.dtau[a][0] = DT(an.ddt[0]);
      ec.dtau[a][1] = DT(an.ddt[1]);
    }
  }
}

// Moments layout: mom[a][j][re/im], j = 0..8 basis (8 = f), j = 9 plain sum Z.
constexpr int kNMom = kNBasis + 1;

// ln L and d lnL / d(physical parameters) from the moments. The arithmetic is
// FP64 throughout (the moments and prefix sums span ~1e-22..1e43, beyond FP32
// range); DT only sets the storage precision of the Jacobian.
template <class DT, bool GRAD>
__device__ void epilogue(const DevEvent& ev, const SweepCoef& sc, const EpiCoef<DT>& ec, const double* mom,
                         double* lnl, double* gph) {
  double acc = -0.5 * ev.dd;
  double g[SHARPY_NPHYS];
#pragma unroll
  for (int i = 0; i < SHARPY_NPHYS; ++i) g[i] = 0.0;
  for (int a = 0; a < ev.n_det; ++a) {
    const double* M = mom + a * kNMom * 2;
    const double P = sc.kisco >= 0 ? ev.pref[(int64_t)a * ev.n_bins + sc.kisco] : 0.0;
    const double Gr = ec.A0 * ec.cre[a], Gi = ec.A0 * ec.cim[a];
    const double Zr = M[2 * 9], Zi = M[2 * 9 + 1];
    acc += (Gr * Zr - Gi * Zi) - 0.5 * (Gr * Gr + Gi * Gi) * P;
    if (!GRAD) continue;
    const double tp = kTwoPi;
    // Im(G X) for a phase-derivative moment X
    auto imgx = [&](double xr, double xi) { return Gr * xi + Gi * xr; };
    // Re(dG Z) - Re(conj(G) dG) P for an amplitude/response derivative dG
    auto amp = [&](double dr, double di) { return (dr * Zr - di * Zi) - (Gr * dr + Gi * di) * P; };
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      double xr = (double)ec.dc0[p] * Zr, xi = (double)ec.dc0[p] * Zi;
#pragma unroll
      for (int j = 0; j < kNPn; ++j) {
        xr += (double)ec.dalpha[j][p] * M[2 * j];
        xi += (double)ec.dalpha[j][p] * M[2 * j + 1];
      }
      g[p] += tp * imgx(xr, xi);
    }
    const double cr = ec.cre[a], ci = ec.cim[a], A0 = ec.A0;
    g[SHARPY_MC] += amp((double)ec.dA0_mc * cr, (double)ec.dA0_mc * ci);
    g[SHARPY_DL] += amp((double)ec.dA0_dl * cr, (double)ec.dA0_dl * ci);
    g[SHARPY_COSI] += amp(A0 * (double)ec.dcre[a][0], A0 * (double)ec.dcim[a][0]);
    g[SHARPY_PSI] += amp(A0 * (double)ec.dcre[a][1], A0 * (double)ec.dcim[a][1]);
    const double yfr = M[2 * 8], yfi = M[2 * 8 + 1];
    const double dt0 = ec.dtau[a][0], dt1 = ec.dtau[a][1];
    g[SHARPY_RA] += amp(A0 * (double)ec.dcre[a][2], A0 * (double)ec.dcim[a][2]) + tp * imgx(dt0 * yfr, dt0 * yfi);
    g[SHARPY_SINDEC] += amp(A0 * (double)ec.dcre[a][3], A0 * (double)ec.dcim[a][3]) + tp * imgx(dt1 * yfr, dt1 * yfi);
    g[SHARPY_TC] += tp * imgx(yfr, yfi);
    g[SHARPY_PHIC] += -imgx(Zr, Zi);
  }
  *lnl = acc;
  if (GRAD)
#pragma unroll
    for (int i = 0; i < SHARPY_NPHYS; ++i) gph[i] = g[i];
}

// Diagonal Gaussian mixture (test targets): ln L and its gradient.
static __device__ void gaussmix(const DevModel& m, const double* x, double* lnl, double* g) {
  double lc[SHARPY_MAX_COMP];
  double best = -INFINITY;
  for (int c = 0; c < m.n_comp; ++c) {
    double s = m.mix_logw[c];
    for (int i = 0; i < m.n_dim; ++i) {
      double z = (x[i] - m.mix_mu[c][i]) / m.mix_sigma[c][i];
      s += -0.5 * z * z - log(m.mix_sigma[c][i]) - 0.91893853320467274178;  // ln sqrt(2 pi)
    }
    lc[c] = s;
    best = fmax(best, s);
  }
  double tot = 0.0;
  for (int c = 0; c < m.n_comp; ++c) tot += exp(lc[c] - best);
  *lnl = best + log(tot);
  if (g) {
    for (int i = 0; i < m.n_dim; ++i) g[i] = 0.0;
    for (int c = 0; c < m.n_comp; ++c) {
      double r = exp(lc[c] - best) / tot;
      for (int i = 0; i < m.n_dim; ++i) {
        double s = m.mix_sigma[c][i];
        g[i] += -r * (x[i] - m.mix_mu[c][i]) / (s * s);
      }
    }
  }
}

// ln pi and grad ln pi of the box prior (uniform, or density ~ x^2).
static __device__ double prior_logpdf(const DevModel& m, const double* x, double* g) {
  double lp = 0.0;
  bool inside = true;
  for (int i = 0; i < m.n_dim; ++i) {
    double lo = m.lo[i], hi = m.hi[i];
    if (g) g[i] = 0.0;
    if (!(x[i] >= lo && x[i] <= hi)) inside = false;
    if (m.prior[i] == SHARPY_PRIOR_POWER2) {
      lp += log(3.0 * x[i] * x[i] / (hi * hi * hi - lo * lo * lo));
      if (g) g[i] = 2.0 / x[i];
    } else {
      lp += -log(hi - lo);
    }
  }
  return inside ? lp : -INFINITY;
}

}  // namespace sharpy
