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
//
// Precision (template DT): DT = double is the FP64 path. DT = float is the
// mixed path: what the phase needs to ~1e-12 (the values of alpha and c0) is
// computed in double-float arithmetic (FP32 pairs, ~48 bits, no FP64
// instruction but the conversions) and handed to the sweep as FP64, the delays, k_ISCO and the ln L
// assembly stay FP64; the antenna patterns, the amplitude, every Jacobian
// entry and the gradient contraction are FP32 (relative error ~1e-7, far
// inside the 1e-4 gradient tolerance).
#pragma once
#include <type_traits>

#include "common.cuh"
#include "dfloat.cuh"

namespace sharpy {

// Value with derivatives along four directions. The value is FP64 (DT =
// double) or double-float (DT = float); for DT = float an FP32 shadow of the
// value feeds the derivative arithmetic, so derivatives need neither FP64
// operations nor conversions.
template <class DT>
struct I4;

template <>
struct I4<double> {
  double v;
  double d[4];
  __device__ __forceinline__ double f() const { return v; }
  __device__ __forceinline__ void setf(double) {}
};

template <>
struct I4<float> {
  DF v;
  float vf;
  float d[4];
  __device__ __forceinline__ float f() const { return vf; }
  __device__ __forceinline__ void setf(float x) { vf = x; }
};

// value type of I4<DT>, its FP64 value and its low-precision shadow
__device__ __forceinline__ double vdbl(double x) { return x; }
__device__ __forceinline__ double vdbl(DF x) { return df_to_double(x); }
template <class DT>
__device__ __forceinline__ DT vlow(double x) { return (DT)x; }
template <class DT>
__device__ __forceinline__ DT vlow(DF x) { return x.hi; }
__device__ __forceinline__ double vrecip(double x) { return 1.0 / x; }
__device__ __forceinline__ DF vrecip(DF x) { return df_recip(x); }
template <class DT>
__device__ __forceinline__ auto vval(double x) {
  if constexpr (std::is_same<DT, double>::value)
    return x;
  else
    return df_from(x);
}

template <class DT>
__device__ __forceinline__ I4<DT> iconst(double x) {
  I4<DT> r;
  r.v = vval<DT>(x);
  r.setf((DT)x);
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = DT(0);
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> ivar(double x, int k) {
  I4<DT> r = iconst<DT>(x);
  r.d[k] = DT(1);
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator+(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v + b.v;
  r.setf(a.f() + b.f());
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator-(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v - b.v;
  r.setf(a.f() - b.f());
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator*(const I4<DT>& a, const I4<DT>& b) {
  I4<DT> r;
  r.v = a.v * b.v;
  r.setf(a.f() * b.f());
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = a.d[i] * b.f() + a.f() * b.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator*(double s, const I4<DT>& a) {
  I4<DT> r;
  r.v = s * a.v;
  r.setf((DT)s * a.f());
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = (DT)s * a.d[i];
  return r;
}
template <class DT>
__device__ __forceinline__ I4<DT> operator+(double s, const I4<DT>& a) {
  I4<DT> r = a;
  r.v = s + a.v;
  r.setf((DT)s + a.f());
  return r;
}
// 1 / a
template <class DT>
__device__ __forceinline__ I4<DT> recip(const I4<DT>& a) {
  I4<DT> r;
  r.v = vrecip(a.v);
  r.setf(vlow<DT>(r.v));
  const DT g = -r.f() * r.f();
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = g * a.d[i];
  return r;
}
// ln a
template <class DT>
__device__ __forceinline__ I4<DT> ilog(const I4<DT>& a) {
  I4<DT> r;
  r.v = log(a.v);
  r.setf((DT)r.v);
  const DT g = DT(1) / a.f();
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = g * a.d[i];
  return r;
}
// e^a
template <class DT>
__device__ __forceinline__ I4<DT> iexp(const I4<DT>& a) {
  I4<DT> r;
  r.v = exp(a.v);
  r.setf((DT)r.v);
#pragma unroll
  for (int i = 0; i < 4; ++i) r.d[i] = r.f() * a.d[i];
  return r;
}

// Everything the sweep needs for one particle (kept in shared memory).
struct SweepCoef {
  double alpha[kNPn];   // phase basis coefficients [turns]
  double c0;            // constant phase [turns]
  double tau[kMaxDet];  // t_c + delay_a [s]
  // split single-precision copies (SHARPY_MIXED_SPLIT): x = hi + lo to ~48 bits
  float ahi[kNPn], alo[kNPn];
  float thi[kMaxDet], tlo[kMaxDet];  // (also the mixed path's delays)
  float c0f;            // c0 reduced to [-1/2, 1/2] turns
  int kisco;            // last bin with f_k <= f_ISCO (-1: none)
  int ok;               // 0 if the parameters are outside the model's domain
};

__device__ __forceinline__ void split2(double x, float* hi, float* lo) {
  *hi = (float)x;
  *lo = (float)(x - (double)*hi);
}

// Everything the epilogue needs beyond the moments.
template <class DT>
struct EpiCoef {
  double A0;
  double A0sq;                            // A0 * A0
  DT a0;                                  // A0 in the epilogue's type
  DT cre[kMaxDet], cim[kMaxDet];          // C_a
  DT dalpha[kNPn][4];                     // d alpha_j / d(Mc, q, chi1, chi2)
  DT dc0[4];
  DT rel_mc, rel_dl;                      // d ln A0 / d Mc, d ln A0 / d d_L
  DT dcre[kMaxDet][4], dcim[kMaxDet][4];  // d C_a / d(cos i, psi, ra, sin dec)
  DT dtau[kMaxDet][2];                    // d tau_a / d(ra, sin dec)
};

// Map the free parameters of one particle onto the eleven physical ones.
__device__ __forceinline__ void to_physical(const DevModel& m, const double* th, double* ph) {
#pragma unroll
  for (int i = 0; i < SHARPY_NPHYS; ++i) ph[i] = m.fixed[i];
  for (int i = 0; i < m.n_dim; ++i) ph[m.phys[i]] = th[i];
}

// u = (pi Tsun M)^(1/3) = (pi Tsun Mc)^(1/3) eta^(-1/5), 1/u and ln u for the
// mixed path in double-float: u = c^(1/15) with c = (pi Tsun Mc)^5 / eta^3.
// v = 1/u = c^(-1/15) from an FP32 start and two division-free Newton steps
// v <- v + v (1 - c v^15) / 15 (quadratic: 1e-7 -> 1e-14 -> rounding),
// u = c v^14, ln u by the double-float logarithm (it sets the constant and
// 3PN phase terms, which need ~1e-10). Derivatives from
// d ln u = (d Mc / Mc - 3/5 d eta / eta) / 3.
__device__ __forceinline__ void u_mixed(const I4<float>& mcv, const I4<float>& eta, const I4<float>& ieta,
                                        I4<float>& u, I4<float>& ui, I4<float>& lnu) {
  const DF p = (kPi * kTsun) * mcv.v;
  const DF p2 = p * p;
  const DF ie = ieta.v;
  const DF c = (p2 * p2 * p) * (ie * ie * ie);
  DF v = {powf(c.hi, -1.0f / 15.0f), 0.0f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const DF v2 = v * v, v4 = v2 * v2, v8 = v4 * v4;
    const DF v15 = v8 * v4 * v2 * v;
    v = v + ((1.0 / 15.0) * v) * (df_from(1.0) - c * v15);
  }
  const DF v2 = v * v, v4 = v2 * v2, v8 = v4 * v4;
  const DF uu = c * (v8 * v4 * v2);
  const DF l = df_log(uu);
  lnu.v = l;
  lnu.vf = l.hi;
  u.v = uu;
  u.vf = uu.hi;
  ui.v = v;
  ui.vf = v.hi;
  const float imc = 1.0f / mcv.vf, ieta_f = 1.0f / eta.vf;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    lnu.d[i] = (1.0f / 3.0f) * (mcv.d[i] * imc - 0.6f * eta.d[i] * ieta_f);
    u.d[i] = u.vf * lnu.d[i];
    ui.d[i] = -ui.vf * lnu.d[i];
  }
}

// TaylorF2 phase coefficients in turns and their Jacobian w.r.t. (Mc, q, chi1, chi2).
// FP64 path: ln eta, ln Mc and one exponential (u) in FP64; mixed path: u_mixed.
template <class DT>
__device__ void pn_coefficients(const double* ph, I4<DT>* alpha, I4<DT>& cpn, double& mtot, double& fisco) {
  const I4<DT> mc = ivar<DT>(ph[SHARPY_MC], 0);
  const I4<DT> q = ivar<DT>(ph[SHARPY_Q], 1);
  const I4<DT> c1 = ivar<DT>(ph[SHARPY_CHI1], 2);
  const I4<DT> c2 = ivar<DT>(ph[SHARPY_CHI2], 3);
  const I4<DT> onepq = 1.0 + q;
  const I4<DT> m1 = recip(onepq);  // m1 / M
  const I4<DT> m2 = q * m1;        // m2 / M
  const I4<DT> eta = m1 * m2;
  const I4<DT> delta = m1 - m2;
  const I4<DT> iq = recip(q);
  const I4<DT> ieta = onepq * onepq * iq;  // 1 / eta = (1+q)^2 / q
  // ln u = (ln(pi Tsun) + ln Mc - 3/5 ln eta) / 3, v = u f^(1/3), M = u^3 / (pi Tsun)
  I4<DT> lnu, u, ui;
  if constexpr (std::is_same<DT, double>::value) {
    lnu = (1.0 / 3.0) * ((-11.076356701842613) + (ilog(mc) + (-0.6) * ilog(eta)));
    u = iexp(lnu);
    ui = recip(u);
    mtot = u.v * u.v * u.v / (kPi * kTsun);
    fisco = 1.0 / (14.696938456699069 * kPi * kTsun * mtot);  // 6^(3/2) pi M
  } else {
    u_mixed(mc, eta, ieta, u, ui, lnu);
    mtot = 0.0;  // not needed: f_ISCO from 1/u directly
    fisco = df_to_double((1.0 / 14.696938456699069) * (ui.v * ui.v * ui.v));  // 1 / (6^(3/2) u^3)
  }
  const I4<DT> chis = 0.5 * (c1 + c2);
  const I4<DT> chia = 0.5 * (c1 - c2);
  const I4<DT> eta2 = eta * eta;
  // spin-orbit (1.5PN, 2.5PN) and spin-spin (2PN) combinations
  const I4<DT> beta = ((113.0 / 12.0) + (-19.0 / 3.0) * eta) * chis + (113.0 / 12.0) * (delta * chia);
  const I4<DT> gam = ((732985.0 / 2268.0) + ((-24260.0 / 81.0) * eta + (-340.0 / 9.0) * eta2)) * chis +
                     ((732985.0 / 2268.0) + (140.0 / 9.0) * eta) * (delta * chia);
  const I4<DT> sig =
      (79.0 / 8.0) * (eta * (c1 * c2)) + (81.0 / 16.0) * (m1 * m1 * c1 * c1 + m2 * m2 * c2 * c2);
  const I4<DT> p2 = (3715.0 / 756.0) + (55.0 / 9.0) * eta;
  const I4<DT> p3 = (-16.0 * kPi) + 4.0 * beta;
  const I4<DT> p4 =
      (15293365.0 / 508032.0) + ((27145.0 / 504.0) * eta + (3085.0 / 72.0) * eta2 + (-10.0) * sig);
  const I4<DT> p5 = (kPi * 38645.0 / 756.0) + ((-kPi * 65.0 / 9.0) * eta - gam);
  const I4<DT> p6 =
      (11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * kPi * kPi - 6848.0 / 21.0 * kEulerGamma) +
      ((-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * kPi * kPi) * eta + (76055.0 / 1728.0) * eta2 +
       (-127825.0 / 1296.0) * (eta2 * eta));
  const I4<DT> p7 = kPi * ((77096675.0 / 254016.0) + ((378515.0 / 1512.0) * eta + (-74045.0 / 756.0) * eta2));
  // 3 / (128 eta) in turns
  const I4<DT> nt = (3.0 / (128.0 * kTwoPi)) * ieta;
  const I4<DT> ui2 = ui * ui;
  const I4<DT> ui3 = ui2 * ui;
  alpha[0] = nt * (ui3 * ui2);  // x^5
  alpha[1] = nt * (p2 * ui3);   // x^3
  alpha[2] = nt * (p3 * ui2);   // x^2
  alpha[3] = nt * (p4 * ui);    // x
  alpha[4] = nt * p5;           // ln f
  // ln(4u) = ln 4 + ln u
  alpha[5] = nt * (u * (p6 + (-6848.0 / 21.0) * (1.3862943611198906 + lnu)));  // y
  alpha[6] = (-6848.0 / 63.0) * (nt * u);                                       // y ln f
  alpha[7] = nt * (p7 * (u * u));                                               // y^2
  // constant: p5 (1 + 3 ln(u / v_lso)), v_lso = 6^(-1/2)
  cpn = nt * (p5 * ((1.0 + 1.5 * 1.791759469228055) + 3.0 * lnu));
}

// Antenna pattern (type AT), delay (FP64) and their derivatives w.r.t. (psi, ra, sin dec).
template <class AT>
struct Antenna {
  AT fp, fc;
  double dt;
  AT dfp[3], dfc[3];  // d/d(psi, ra, sin dec)
  AT ddt[2];          // d delay / d(ra, sin dec)
};

template <class AT>
__device__ __forceinline__ AT quad(const AT (*D)[3], const AT* a, const AT* b) {
  AT s = AT(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) s += a[i] * D[i][j] * b[j];
  return s;
}

__device__ __forceinline__ void sincos2psi(double psi, double* s2, double* c2) { sincos(2.0 * psi, s2, c2); }
__device__ __forceinline__ const double* det_rc(const DevDetector& det, double*) { return det.rcd; }
__device__ __forceinline__ const float* det_rc(const DevDetector& det, float*) { return det.rcf; }
__device__ __forceinline__ void sincos2psi(double psi, float* s2, float* c2) { sincosf(2.0f * (float)psi, s2, c2); }
__device__ __forceinline__ const double (*det_tensor(const DevDetector& det, double))[3] { return det.D; }
__device__ __forceinline__ const float (*det_tensor(const DevDetector& det, float))[3] { return det.Df; }

// Geocentric delay in FP64 (it multiplies frequencies up to kHz in the
// phase); patterns and all derivatives in type AT.
template <class AT>
static __device__ void antenna(const DevDetector& det, double sa, double ca, double cd, double sdec, AT s2, AT c2,
                               Antenna<AT>& out) {
  if (det.fixed_response) {
    out.fp = (AT)det.fplus;
    out.fc = (AT)det.fcross;
    out.dt = det.delay;
    for (int i = 0; i < 3; ++i) out.dfp[i] = out.dfc[i] = AT(0);
    out.ddt[0] = out.ddt[1] = AT(0);
    return;
  }
  const double* rd = det.rcd;  // position / c
  out.dt = -(rd[0] * (cd * ca) + rd[1] * (cd * sa) + rd[2] * sdec);
  const AT* rc = det_rc(det, (AT*)nullptr);
  const AT a_s = (AT)sa, a_c = (AT)ca, a_d = (AT)cd, a_z = (AT)sdec;
  const AT p[3] = {a_s, -a_c, AT(0)};
  const AT q[3] = {a_z * a_c, a_z * a_s, -a_d};
  const AT dp_ra[3] = {a_c, a_s, AT(0)};
  const AT dq_ra[3] = {-a_z * a_s, a_z * a_c, AT(0)};
  const AT dq_sd[3] = {a_c, a_s, a_z / a_d};
  const AT (*D)[3] = det_tensor(det, AT(0));
  const AT fp0 = quad<AT>(D, p, p) - quad<AT>(D, q, q);
  const AT fc0 = AT(2) * quad<AT>(D, p, q);
  const AT dfp0_ra = AT(2) * (quad<AT>(D, p, dp_ra) - quad<AT>(D, q, dq_ra));
  const AT dfc0_ra = AT(2) * (quad<AT>(D, dp_ra, q) + quad<AT>(D, p, dq_ra));
  const AT dfp0_sd = AT(-2) * quad<AT>(D, q, dq_sd);
  const AT dfc0_sd = AT(2) * quad<AT>(D, p, dq_sd);
  out.fp = c2 * fp0 + s2 * fc0;
  out.fc = -s2 * fp0 + c2 * fc0;
  out.dfp[0] = AT(2) * out.fc;
  out.dfc[0] = AT(-2) * out.fp;
  out.dfp[1] = c2 * dfp0_ra + s2 * dfc0_ra;
  out.dfc[1] = -s2 * dfp0_ra + c2 * dfc0_ra;
  out.dfp[2] = c2 * dfp0_sd + s2 * dfc0_sd;
  out.dfc[2] = -s2 * dfp0_sd + c2 * dfc0_sd;
  // d n / d ra = (-cd sa, cd ca, 0); d n / d sin dec = (-sdec ca / cd, -sdec sa / cd, 1)
  out.ddt[0] = -(rc[0] * (-a_d * a_s) + rc[1] * (a_d * a_c));
  out.ddt[1] = -(rc[0] * (-a_z * a_c / a_d) + rc[1] * (-a_z * a_s / a_d) + rc[2]);
}

// Last bin with f_k <= f_isco, using the staged frequency table.
__device__ __forceinline__ int isco_bin(const DevEvent& ev, double fisco) {
  int64_t K = ev.n_bins;
  double t = floor((fisco - ev.f_min) * ev.inv_df);
  int64_t k = t < -1.0 ? -1 : (t > (double)(K - 1) ? K - 1 : (int64_t)t);
  while (k + 1 < K && ev.f[k + 1] <= fisco) ++k;
  while (k >= 0 && ev.f[k] > fisco) --k;
  return (int)k;
}

// Whether theta lies in the model's domain (both halves of the prologue test it).
// x > 0 and |x| <= 1 decided on the bits of x (integer pipes, not the FP64
// one), with the comparisons' own results for every input: NaN fails both,
// +inf passes the first.
__device__ __forceinline__ bool bits_positive(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool bits_abs_le1(double x) {
  return (__double_as_longlong(x) & 0x7fffffffffffffffLL) <= 0x3ff0000000000000LL;
}
__device__ __forceinline__ bool phys_ok(const double* ph) {
  return bits_positive(ph[SHARPY_MC]) && bits_positive(ph[SHARPY_Q]) && bits_positive(ph[SHARPY_DL]) &&
         bits_abs_le1(ph[SHARPY_SINDEC]) && bits_abs_le1(ph[SHARPY_COSI]);
}

// The prologue in two independent halves, so that two warps can run them at
// once (the persistent NUTS kernel does): the phase half writes alpha, c0,
// k_ISCO, ok (and their Jacobians); the sky half writes the amplitude, the
// responses C_a, the delays tau_a (and theirs). Neither reads what the other
// writes.
template <class DT, bool GRAD, bool SPLIT = false>
__device__ void prologue_phase(const DevModel& m, const DevEvent& ev, const double* th, SweepCoef& sc,
                               EpiCoef<DT>& ec) {
  double ph[SHARPY_NPHYS];
  to_physical(m, th, ph);
  sc.ok = phys_ok(ph) ? 1 : 0;
  if (!sc.ok) {
    sc.kisco = -1;
    return;
  }
  I4<DT> alpha[kNPn], cpn;
  double mtot, fisco;
  pn_coefficients<DT>(ph, alpha, cpn, mtot, fisco);
  // the mixed sweep reads the four large terms' coefficients in FP64 and the
  // others as FP32 pairs: only the four get an FP64 copy there
  constexpr bool kAllF64 = SPLIT || std::is_same<DT, double>::value;
#pragma unroll
  for (int j = 0; j < kNPn; ++j) {
    if (kAllF64 || is_large_pn(j)) sc.alpha[j] = vdbl(alpha[j].v);
    if (GRAD)
#pragma unroll
      for (int i = 0; i < 4; ++i) ec.dalpha[j][i] = alpha[j].d[i];
  }
  sc.c0 = vdbl(cpn.v) - ph[SHARPY_PHIC] * (1.0 / kTwoPi) - 0.125;
  if (GRAD)
#pragma unroll
    for (int i = 0; i < 4; ++i) ec.dc0[i] = cpn.d[i];
  sc.kisco = isco_bin(ev, fisco);
  if (SPLIT) {
#pragma unroll
    for (int j = 0; j < kNPn; ++j) split2(sc.alpha[j], &sc.ahi[j], &sc.alo[j]);
    sc.c0f = (float)(sc.c0 - rint(sc.c0));
  } else if constexpr (!std::is_same<DT, double>::value) {
    // the mixed sweep's FP32-pair terms take the double-float values as they are
#pragma unroll
    for (int j = 0; j < kNPn; ++j) {
      sc.ahi[j] = alpha[j].v.hi;
      sc.alo[j] = alpha[j].v.lo;
    }
  }
}

template <class DT, bool GRAD, bool SPLIT = false>
__device__ void prologue_sky(const DevModel& m, const DevEvent& ev, const double* th, SweepCoef& sc,
                             EpiCoef<DT>& ec) {
  double ph[SHARPY_NPHYS];
  to_physical(m, th, ph);
  if (!phys_ok(ph)) return;
  // Newtonian amplitude of an optimally oriented source: sqrt(5/24) pi^(-2/3) (T Mc)^(5/6) / D.
  // Its square multiplies <h|h>, so for loud templates its precision sets that
  // of ln L: the mixed path takes (T Mc)^(5/6) from an FP32 power and one
  // Newton step on y^6 = x^5 in double-float (1e-7 -> 1e-14).
  const DT mc = (DT)ph[SHARPY_MC], dl = (DT)ph[SHARPY_DL];
  constexpr double kAmp = 0.45643546458763845 * 0.46619407703541166;
  if constexpr (std::is_same<DT, double>::value) {
    ec.A0 = kAmp * pow(kTsun * mc, 5.0 / 6.0) / (dl * kMpcSec);
  } else {
    const double x = kTsun * ph[SHARPY_MC];
    const DF X = df_from(x);
    const DF X2 = X * X, X5 = (X2 * X2) * X;
    const DF Y = {powf((float)x, 5.0f / 6.0f), 0.0f};
    const DF Y3 = (Y * Y) * Y, Y6 = Y3 * Y3;
    const DF t = X5 * df_recip(Y6) - df_from(1.0);
    const DF Y1 = Y + Y * ((1.0 / 6.0) * t);
    ec.A0 = df_to_double((kAmp * Y1) * df_recip(df_from(ph[SHARPY_DL] * kMpcSec)));
  }
  ec.A0sq = ec.A0 * ec.A0;
  ec.a0 = (DT)ec.A0;
  if (GRAD) {
    ec.rel_mc = DT(5.0 / 6.0) / mc;
    ec.rel_dl = DT(-1) / dl;
  }
  const DT ci = (DT)ph[SHARPY_COSI];
  // sky position in FP64: the delays multiply frequencies up to kHz
  double sa = 0.0, ca = 1.0, cd = 1.0;
  DT s2 = DT(0), c2 = DT(1);
  const double sdec = ph[SHARPY_SINDEC];
  bool any_sky = false;
  for (int a = 0; a < ev.n_det; ++a) any_sky = any_sky || !ev.det[a].fixed_response;
  if (any_sky) {
    sincos(ph[SHARPY_RA], &sa, &ca);
    cd = sqrt(fmax(1.0 - sdec * sdec, 0.0));
    sincos2psi(ph[SHARPY_PSI], &s2, &c2);
  }
  for (int a = 0; a < ev.n_det; ++a) {
    Antenna<DT> an;
    antenna<DT>(ev.det[a], sa, ca, cd, sdec, s2, c2, an);
    sc.tau[a] = ph[SHARPY_TC] + an.dt;
    const DT hp = DT(0.5) * (DT(1) + ci * ci);
    ec.cre[a] = an.fp * hp;
    ec.cim[a] = -an.fc * ci;
    if (GRAD) {
      ec.dcre[a][0] = an.fp * ci;
      ec.dcim[a][0] = -an.fc;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ec.dcre[a][k + 1] = an.dfp[k] * hp;
        ec.dcim[a][k + 1] = -an.dfc[k] * ci;
      }
      ec.dtau[a][0] = an.ddt[0];
      ec.dtau[a][1] = an.ddt[1];
    }
  }
  // hi/lo of the delays: the split and the mixed sweeps form f tau_a in FP32
  if (SPLIT || std::is_same<DT, float>::value)
    for (int a = 0; a < ev.n_det; ++a) split2(sc.tau[a], &sc.thi[a], &sc.tlo[a]);
}

// theta (free dims) -> sweep and epilogue coefficients.
template <class DT, bool GRAD, bool SPLIT = false>
__device__ void prologue(const DevModel& m, const DevEvent& ev, const double* th, SweepCoef& sc,
                         EpiCoef<DT>& ec) {
  prologue_phase<DT, GRAD, SPLIT>(m, ev, th, sc, ec);
  prologue_sky<DT, GRAD, SPLIT>(m, ev, th, sc, ec);
}

// Moments layout: mom[a][j][re/im], j = 0..8 basis (8 = f), j = 9 plain sum Z.
constexpr int kNMom = kNBasis + 1;

// ln L (FP64 total) and d lnL / d(physical parameters) from the moments.
// The gradient is contracted on the amplitude-scaled moments A0 Z, A0 Y_j and
// the scaled prefix sum A0^2 P, which are O(SNR^2) and fit FP32 (the raw moments
// and prefix sums span ~1e-22..1e43). FP64 path: ln L assembled in FP64 from
// the raw moments. Mixed paths: from the same scaled FP32 quantities with exact
// products and double-float sums (the moments are FP32 anyway), so only the
// scaling A0^2 P and the conversions remain FP64.
template <class DT, bool GRAD, class MT, class GT>
__device__ void epilogue(const DevEvent& ev, const SweepCoef& sc, const EpiCoef<DT>& ec, const MT* mom, double* lnl,
                         GT* gph) {
  constexpr bool kDF = std::is_same<DT, float>::value;
  double acc = -0.5 * ev.dd;
  DF accf = kDF ? DF{ev.ddh_hi, ev.ddh_lo} : DF{0.0f, 0.0f};  // = df_from(acc), formed when the data were set
  DT g[SHARPY_NPHYS];
#pragma unroll
  for (int i = 0; i < SHARPY_NPHYS; ++i) g[i] = DT(0);
  const DT a0 = ec.a0;
  for (int a = 0; a < ev.n_det; ++a) {
    const MT* M = mom + a * kNMom * 2;
    const double P = sc.kisco >= 0 ? ev.pref[(int64_t)a * ev.n_bins + sc.kisco] : 0.0;
    const DT cr = ec.cre[a], ci = ec.cim[a];
    const DT ps = (DT)(ec.A0sq * P);                   // A0^2 P
    const DT zr = a0 * (DT)M[18], zi = a0 * (DT)M[19];  // A0 Z
    if constexpr (kDF) {
      // Re(C A0 Z) - |C|^2 A0^2 P / 2
      const DF re = df_two_prod(cr, zr) - df_two_prod(ci, zi);
      const DF c2 = df_two_prod(cr, cr) + df_two_prod(ci, ci);
      const DF c2p = df_two_prod(c2.hi, 0.5f * ps) + DF{__fmul_rn(c2.lo, 0.5f * ps), 0.0f};
      accf = accf + (re - c2p);
    } else {
      const double Gr = ec.A0 * (double)ec.cre[a], Gi = ec.A0 * (double)ec.cim[a];
      acc += (Gr * (double)M[18] - Gi * (double)M[19]) - 0.5 * (Gr * Gr + Gi * Gi) * P;
    }
    if (!GRAD) continue;
    const DT tp = DT(kTwoPi);
    // Im(C X) for a scaled phase-derivative moment X
    auto imcx = [&](DT xr, DT xi) { return cr * xi + ci * xr; };
    // Re(dC A0 Z) - Re(conj(C) dC) A0^2 P for a response derivative dC
    auto resp = [&](DT dr, DT di) { return (dr * zr - di * zi) - (cr * dr + ci * di) * ps; };
    DT yr[kNPn], yi[kNPn];
#pragma unroll
    for (int j = 0; j < kNPn; ++j) {
      yr[j] = a0 * (DT)M[2 * j];
      yi[j] = a0 * (DT)M[2 * j + 1];
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      DT xr = ec.dc0[p] * zr, xi = ec.dc0[p] * zi;
#pragma unroll
      for (int j = 0; j < kNPn; ++j) {
        xr += ec.dalpha[j][p] * yr[j];
        xi += ec.dalpha[j][p] * yi[j];
      }
      g[p] += tp * imcx(xr, xi);
    }
    const DT amp = (cr * zr - ci * zi) - (cr * cr + ci * ci) * ps;  // d/d ln A0
    g[SHARPY_MC] += ec.rel_mc * amp;
    g[SHARPY_DL] += ec.rel_dl * amp;
    g[SHARPY_COSI] += resp(ec.dcre[a][0], ec.dcim[a][0]);
    g[SHARPY_PSI] += resp(ec.dcre[a][1], ec.dcim[a][1]);
    const DT yfr = a0 * (DT)M[16], yfi = a0 * (DT)M[17];
    g[SHARPY_RA] += resp(ec.dcre[a][2], ec.dcim[a][2]) + tp * imcx(ec.dtau[a][0] * yfr, ec.dtau[a][0] * yfi);
    g[SHARPY_SINDEC] += resp(ec.dcre[a][3], ec.dcim[a][3]) + tp * imcx(ec.dtau[a][1] * yfr, ec.dtau[a][1] * yfi);
    g[SHARPY_TC] += tp * imcx(yfr, yfi);
    g[SHARPY_PHIC] += -imcx(zr, zi);
  }
  *lnl = kDF ? df_to_double(accf) : acc;
  if (GRAD)
#pragma unroll
    for (int i = 0; i < SHARPY_NPHYS; ++i) gph[i] = (GT)g[i];
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
