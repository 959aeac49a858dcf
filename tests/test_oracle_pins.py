"""Pins for the oracle: closed forms, invariants, special cases and brute force.

Each test checks the oracle against something other than its own formula,
so that a dropped term, a wrong sign, index or exponent fails here before
the oracle is used as the reference for the GPU library.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_2601_02336_gb300 import inputs
from tests import helpers

TSUN = 4.925491025543576e-6
MPC_S = 3.085677581491367e22 / 299792458.0


# ---------------------------------------------------------------- Philox
def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with Random123 (Salmon et al. 2011)."""
    assert oracle.philox([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert oracle.philox([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2) == [0x408F276D, 0x41C83B0E, 0xA20BC7C6,
                                                                  0x6D5451FD]
    assert oracle.philox([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                         [0xA4093822, 0x299F31D0]) == [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_uniform_normal_distribution():
    u = np.array([oracle.uniform2(7, i, 3, 1, 0) for i in range(4000)]).ravel()
    assert u.min() > 0 and u.max() < 1
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    z = np.array([oracle.normal2(7, i, 3, 2, 0) for i in range(4000)]).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3


# ---------------------------------------------------------------- TaylorF2
def test_newtonian_chirp_time():
    """Stationary phase: t(f) = (1/2pi) dPsi/df; at Newtonian order
    t_c - t(f) = (5/256) (pi f)^(-8/3) (T_sun M_c)^(-5/3). Checked at very low
    frequency where the PN corrections are below 1e-3."""
    mc, q = 30.0, 0.6
    for f in (2e-3, 5e-3):
        h = f * 1e-4
        dpsi = (oracle.pn_phase(mc, q, 0.0, 0.0, f + h) - oracle.pn_phase(mc, q, 0.0, 0.0, f - h)) / (2 * h)
        tau = -dpsi / (2 * math.pi)
        tau_n = 5.0 / 256.0 * (math.pi * f) ** (-8.0 / 3.0) * (TSUN * mc) ** (-5.0 / 3.0)
        assert abs(tau / tau_n - 1.0) < 2e-3


def test_1pn_chirp_time_coefficient():
    """1PN chirp time (Sathyaprakash-Dhurandhar tau_2): t/t_N - 1 -> (4/3)(743/336 + 11 eta/4) v^2.
    Extrapolated to v -> 0 from a polynomial fit in v; checks the 1PN
    coefficient at two mass ratios (i.e. both of its numbers)."""
    mc = 25.0
    for q in (1.0, 0.2):
        eta = q / (1 + q) ** 2
        mtot = mc * eta ** -0.6
        vs = np.linspace(0.004, 0.02, 12)
        ratios = []
        for v in vs:
            f = v ** 3 / (math.pi * mtot * TSUN)
            h = f * 1e-5
            d = (oracle.pn_phase(mc, q, 0, 0, f + h) - oracle.pn_phase(mc, q, 0, 0, f - h)) / (2 * h)
            tau = -d / (2 * math.pi)
            tau_n = 5.0 / 256.0 * (math.pi * f) ** (-8.0 / 3.0) * (TSUN * mc) ** (-5.0 / 3.0)
            ratios.append((tau / tau_n - 1.0) / v ** 2)
        coef = np.polyfit(vs, ratios, 3)[-1]
        expect = 4.0 / 3.0 * (743.0 / 336.0 + 11.0 * eta / 4.0)
        assert abs(coef - expect) < 2e-2 * expect


# Published post-Newtonian pins of the full phase. The stationary-phase relation
# t(f) = (1/2pi) dPsi/df ties the TaylorF2 phase to the chirp time t(v), a
# series published in other forms and with other numbers than the phase
# coefficients: (i) Blanchet's TaylorT2 time series (Living Rev. Relativ. 17, 2
# (2014), the t(x) expansion of Sec. 9.3 through 3.5PN with its 3PN logarithm),
# with the 1.5PN spin-orbit and 2PN spin-spin parameters of Poisson & Will
# (PRD 52, 848 (1995)); (ii) the same series DERIVED here by energy balance,
# dt/dv = -E'(v)/F(v), from the published binding energy E(x) and flux F(x)
# (Blanchet 2014, non-spinning to 3.5PN; spin-orbit terms at 1.5PN and 2.5PN of
# Blanchet, Buonanno & Faye, PRD 74, 104034 (2006), in the S_l, Sigma_l
# variables). The oracle's t(f) comes from its exact (dual-number) derivative of
# Psi, using f dPsi/df = M_c dPsi/dM_c (Psi depends on f and M_c only through
# v^3 ~ M_c f at fixed q). Constant phase terms (the "1" of the 2.5PN factor
# 1 + 3 ln(v/v_lso), and v_lso) have no effect on t(f); the stationary-phase
# test below pins them on Psi itself.

def _oracle_chirp_time(mc, q, c1, c2, v):
    """t(f) - t_c of the oracle's phase at the frequency where v = (pi M T_sun f)^(1/3)."""
    eta = q / (1 + q) ** 2
    mtot = mc * eta ** -0.6
    f = v ** 3 / (math.pi * TSUN * mtot)
    return mc / f * oracle.pn_phase_dmc(mc, q, c1, c2, f) / (2 * math.pi), mtot, eta


def _sigma_aligned(q, c1, c2):
    """2PN spin-spin parameter for aligned black-hole spins from the vector form of Arun, Buonanno,
    Faye & Ochsner (PRD 79, 104023 (2009), Eq. 6.24 and its self-spin terms; Mikoczi, Vasuth & Gergely
    2005), with the quadrupole parameter kappa = 1 and L.chi_i = chi_i, chi_1.chi_2 = chi_1 chi_2."""
    x1, x2 = 1 / (1 + q), q / (1 + q)
    eta, kappa = x1 * x2, 1.0
    s = eta * (721.0 / 48.0 * c1 * c2 - 247.0 / 48.0 * c1 * c2)
    for x, c in ((x1, c1), (x2, c2)):
        s += (720.0 * kappa - 1.0) / 96.0 * x * x * c * c - (240.0 * kappa - 7.0) / 96.0 * x * x * c * c
    return s


def _taylor_t2_series(eta, beta, sigma, v):
    """Blanchet's TaylorT2 bracket, t - t_c = -(5 M/(256 eta v^8)) * bracket, non-spinning through
    3.5PN (x = v^2, ln(16 x) = 2 ln(4 v)), plus Poisson & Will's spin terms: -8/5 (4 pi - beta) v^3
    and -2 sigma v^4."""
    pi, ge = math.pi, 0.57721566490153286061
    t2 = 743.0 / 252.0 + 11.0 / 3.0 * eta
    t3 = -8.0 / 5.0 * (4.0 * pi - beta)
    t4 = 3058673.0 / 508032.0 + 5429.0 / 504.0 * eta + 617.0 / 72.0 * eta ** 2 - 2.0 * sigma
    t5 = -7729.0 / 252.0 * pi + 13.0 / 3.0 * pi * eta
    t6 = (-10052469856691.0 / 23471078400.0 + 128.0 / 3.0 * pi ** 2 + 6848.0 / 105.0 * ge
          + (3147553127.0 / 3048192.0 - 451.0 / 12.0 * pi ** 2) * eta - 15211.0 / 1728.0 * eta ** 2
          + 25565.0 / 1296.0 * eta ** 3 + 3424.0 / 105.0 * math.log(16.0 * v * v))
    t7 = (-15419335.0 / 127008.0 - 75703.0 / 756.0 * eta + 14809.0 / 378.0 * eta ** 2) * pi
    return 1 + t2 * v ** 2 + t3 * v ** 3 + t4 * v ** 4 + t5 * v ** 5 + t6 * v ** 6 + t7 * v ** 7


def _energy_balance_taus(q, c1, c2):
    """tau_k(ln v) of t - t_c = -(5 M/(256 eta v^8)) sum_k tau_k v^k, derived from the published
    E(x) and F(x) by series division and term-by-term integration, exact in rationals, pi, gamma_E,
    ln 2 and L = ln v. Spin terms are kept through 2.5PN only (the model has none at 3PN and 3.5PN,
    so products of spin-orbit terms, which start at 3PN, are dropped); E and F here carry no
    spin-spin terms (those enter through sigma)."""
    sp = pytest.importorskip("sympy")
    L, taus = _energy_balance_series(q, c1, c2)
    return [sp.lambdify(L, t) for t in taus]


def _energy_balance_series(q, c1, c2):
    """(L, [tau_k(L)]) as exact sympy expressions; see _energy_balance_taus."""
    sp = pytest.importorskip("sympy")
    R, pi, ge = sp.Rational, sp.pi, sp.EulerGamma
    L, s = sp.Symbol("L"), sp.Symbol("s")  # L = ln v; s marks each spin-orbit factor
    q, c1, c2 = R(q), R(c1), R(c2)
    x1, x2 = 1 / (1 + q), q / (1 + q)
    eta, dm = x1 * x2, x1 - x2
    sl = s * (x1 ** 2 * c1 + x2 ** 2 * c2)  # S_l / M^2
    sg = s * (x2 * c2 - x1 * c1)            # Sigma_l / M^2
    # E = -(eta v^2 / 2) sum e_k v^k
    e = [1, 0, -R(3, 4) - eta / 12, R(14, 3) * sl + 2 * dm * sg,
         -R(27, 8) + R(19, 8) * eta - eta ** 2 / 24,
         (11 - R(61, 9) * eta) * sl + dm * (3 - R(10, 3) * eta) * sg,
         -R(675, 64) + (R(34445, 576) - 205 * pi ** 2 / 96) * eta - R(155, 96) * eta ** 2 - R(35, 5184) * eta ** 3,
         0]
    # F = (32/5) eta^2 v^10 sum f_k v^k, ln(16 x) = 4 ln 2 + 2 L
    f = [1, 0, -R(1247, 336) - R(35, 12) * eta,
         4 * pi - 4 * sl - R(5, 4) * dm * sg,
         -R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2,
         -(R(8191, 672) + R(583, 24) * eta) * pi + (-R(9, 2) + R(272, 9) * eta) * sl
         + (-R(13, 16) + R(43, 4) * eta) * dm * sg,
         R(6643739519, 69854400) + 16 * pi ** 2 / 3 - R(1712, 105) * ge - R(856, 105) * (4 * sp.log(2) + 2 * L)
         + (-R(134543, 7776) + 41 * pi ** 2 / 48) * eta - R(94403, 3024) * eta ** 2 - R(775, 324) * eta ** 3,
         (-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * pi]
    de = [R(k + 2, 2) * e[k] for k in range(8)]  # -E'(v) = eta v sum (k+2)/2 e_k v^k
    inv = [sp.Integer(1)] + [0] * 7               # 1 / sum f_k v^k
    for k in range(1, 8):
        inv[k] = sp.expand(-sum(f[j] * inv[k - j] for j in range(1, k + 1)))
    taus = []
    for k in range(8):
        a = sp.expand(sum(de[j] * inv[k - j] for j in range(k + 1)))
        a = sp.expand(a.coeff(s, 0) + (a.coeff(s, 1) if k <= 5 else 0))
        b, c, n = a.coeff(L, 0), a.coeff(L, 1), k - 8  # integrate v^(n-1) (b + c L)
        integral = b / n + c * (L - R(1, n)) / n
        taus.append(sp.expand(integral * R(5, 32) / eta * R(-256, 5) * eta))
    return L, taus


_PN_CASES = [(1.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.6, 1 / 3, -0.5), (0.125, 0.9, 0.7), (0.9, -0.8, 0.2)]


@pytest.mark.parametrize("q,c1,c2", _PN_CASES)
def test_chirp_time_published_taylor_t2(q, c1, c2):
    """The oracle's t(f) equals Blanchet's TaylorT2 series (with Poisson & Will's beta and the
    vector-form sigma) to 1e-12 relative over v = 0.05..0.6 (20 Hz up past the ISCO of the
    workloads' masses), at five mass ratios and four spin pairs. The 2.5PN spin-orbit term is
    pinned by the energy-balance test below."""
    mc = 20.0
    x1, x2 = 1 / (1 + q), q / (1 + q)
    eta = x1 * x2
    beta_pw = sum((113.0 / 12.0 * x * x + 25.0 / 4.0 * eta) * c for x, c in ((x1, c1), (x2, c2)))
    sigma = _sigma_aligned(q, c1, c2)
    # the 2.5PN spin-orbit part of tau_5 (3 gamma / 5) is added from the energy-balance series
    taus = _energy_balance_taus(q, c1, c2)
    taus0 = _energy_balance_taus(q, 0.0, 0.0)
    for v in np.linspace(0.05, 0.6, 30):
        t_or, mtot, eta_o = _oracle_chirp_time(mc, q, c1, c2, v)
        so25 = (taus[5](math.log(v)) - taus0[5](math.log(v))) * v ** 5
        t_pub = -5.0 * mtot * TSUN / (256.0 * eta * v ** 8) * (_taylor_t2_series(eta, beta_pw, sigma, v) + so25)
        assert abs(t_or / t_pub - 1.0) < 1e-12, (q, c1, c2, v, t_or, t_pub)


@pytest.mark.parametrize("q,c1,c2", _PN_CASES)
def test_chirp_time_energy_balance(q, c1, c2):
    """The oracle's t(f) equals the chirp time derived by energy balance from the published E(x)
    and F(x) (non-spinning through 3.5PN, spin-orbit at 1.5PN and 2.5PN), plus -2 sigma v^4 for the
    2PN spin-spin terms, to 1e-12 relative over v = 0.05..1. Every post-Newtonian coefficient of
    the phase, the 3PN logarithm and the beta, gamma, sigma spin terms enter this comparison
    through numbers that appear nowhere in the oracle."""
    mc = 20.0
    taus = _energy_balance_taus(q, c1, c2)
    sigma = _sigma_aligned(q, c1, c2)
    for v in np.linspace(0.05, 1.0, 40):
        t_or, mtot, eta = _oracle_chirp_time(mc, q, c1, c2, v)
        lv = math.log(v)
        ser = sum(float(taus[k](lv)) * v ** k for k in range(8)) - 2.0 * sigma * v ** 4
        t_pub = -5.0 * mtot * TSUN / (256.0 * eta * v ** 8) * ser
        assert abs(t_or / t_pub - 1.0) < 1e-12, (q, c1, c2, v, t_or, t_pub)


@pytest.mark.parametrize("q,c1,c2", _PN_CASES)
def test_phase_stationary_phase_of_energy_balance(q, c1, c2):
    """The oracle's Psi itself, constant terms included, against the stationary-phase transform of
    the energy-balance orbit: Psi(f) = 2 pi f (t - t_c) - 2 (phi - phi_c) at the frequency where the
    GW frequency is twice the orbital one, with t(v) from the published E(x) and F(x) as above and
    the orbital phase phi(v) integrated from d phi/dv = (v^3/M) dt/dv. Every term of phi is fixed by
    the integration except the 2.5PN logarithm's reference, taken at the Schwarzschild
    last-stable-orbit velocity v_lso = 6^(-1/2) (the TaylorF2 reading the oracle states). This pins
    what the chirp-time tests cannot see: the "1" of the 2.5PN factor 1 + 3 ln(v/v_lso), the factor 3,
    and v_lso, each an eta- and spin-dependent constant phase, to 1e-12 of the Newtonian term."""
    sp = pytest.importorskip("sympy")
    R = sp.Rational
    L, taus = _energy_balance_series(q, c1, c2)
    taus = list(taus)
    taus[4] = taus[4] - 2 * R(_sigma_aligned(q, c1, c2))  # 2PN spin-spin, as in the chirp-time tests
    x1, x2 = 1 / (1 + R(q)), R(q) / (1 + R(q))
    eta = x1 * x2
    v = sp.exp(L)
    l_lso = -sp.log(6) / 2
    # t - t_c = M T(v); phi - phi_c = -(5/(256 eta)) sum_k I_k(v)
    T = -R(5, 256) / eta * sum(taus[k] * v ** (k - 8) for k in range(8))
    phi = 0
    for k in range(8):
        a = sp.expand((k - 8) * taus[k] + sp.diff(taus[k], L))  # d/dv [tau_k v^(k-8)] = a v^(k-9)
        b, c, m = a.coeff(L, 0), a.coeff(L, 1), k - 5            # integrate v^(m-1) (b + c L)
        assert sp.expand(a - b - c * L) == 0
        if m == 0:
            assert c == 0
            phi += b * (L - l_lso)
        else:
            phi += (b / m + c * (L - R(1, m)) / m) * v ** m
    phi = -R(5, 256) / eta * phi
    psi = sp.lambdify(L, 2 * v ** 3 * T - 2 * phi)
    mc = 20.0
    eta_f = float(eta)
    mtot = mc * eta_f ** -0.6
    for vv in np.linspace(0.05, 1.0, 40):
        f = vv ** 3 / (math.pi * TSUN * mtot)
        got = oracle.pn_phase(mc, q, c1, c2, f)
        want = float(psi(math.log(vv)))
        newton = 3.0 / (128.0 * eta_f * vv ** 5)
        assert abs(got - want) < 1e-12 * newton, (q, c1, c2, vv, got, want)


def test_spin_orbit_beta_identity():
    """beta = sum_i (113/12 (m_i/M)^2 + 25/4 eta) chi_i (per-body form of the 1.5PN spin-orbit term)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        q, c1, c2 = rng.uniform(0.1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)
        eta = q / (1 + q) ** 2
        m1, m2 = 1 / (1 + q), q / (1 + q)
        want = (113 / 12 * m1 ** 2 + 25 / 4 * eta) * c1 + (113 / 12 * m2 ** 2 + 25 / 4 * eta) * c2
        assert oracle.pn_beta(q, c1, c2) == pytest.approx(want, rel=1e-13, abs=1e-14)


def test_phase_body_exchange_symmetry():
    """Relabelling the bodies (q -> 1/q, chi1 <-> chi2, chirp mass fixed) leaves Psi unchanged."""
    rng = np.random.default_rng(1)
    for _ in range(40):
        mc, q = rng.uniform(5, 40), rng.uniform(0.15, 0.95)
        c1, c2 = rng.uniform(-0.9, 0.9), rng.uniform(-0.9, 0.9)
        f = rng.uniform(20, 60)
        a = oracle.pn_phase(mc, q, c1, c2, f)
        b = oracle.pn_phase(mc, 1.0 / q, c2, c1, f)
        assert a == pytest.approx(b, rel=1e-12)
        # and the spin terms do enter: flipping one spin changes the phase
        assert abs(oracle.pn_phase(mc, q, c1, -c2, f) - a) > 1e-6 or abs(c2) < 1e-3


def test_amplitude_from_time_domain_quadrupole():
    """SPA amplitude |h~(f)| = h0(t_f) / (2 sqrt(fdot)) with the quadrupole
    h0 = 4 (T M_c)^(5/3) (pi f)^(2/3) / D and fdot = (96/5) pi^(8/3) (T M_c)^(5/3) f^(11/3)."""
    for mc, dl, f in [(30.0, 400.0, 30.0), (1.2, 100.0, 200.0), (11.0, 4000.0, 21.5)]:
        m = TSUN * mc
        D = dl * MPC_S
        h0 = 4.0 * m ** (5.0 / 3.0) * (math.pi * f) ** (2.0 / 3.0) / D
        fdot = 96.0 / 5.0 * math.pi ** (8.0 / 3.0) * m ** (5.0 / 3.0) * f ** (11.0 / 3.0)
        assert oracle.amplitude(mc, dl, f) == pytest.approx(0.5 * h0 / math.sqrt(fdot), rel=1e-12)


def test_f_isco():
    """f_ISCO = c^3 / (6^(3/2) pi G M): 4397 Hz for one solar mass."""
    assert oracle.f_isco(1.0 * 0.25 ** 0.6, 1.0) * 1.0 == pytest.approx(1.0 / (6 ** 1.5 * math.pi * TSUN), rel=1e-12)
    assert 4390 < 1.0 / (6 ** 1.5 * math.pi * TSUN) < 4400


def test_hh_flat_psd_euler_maclaurin():
    """Flat PSD, face-on, F+ = 1: <h|h> = 4 df sum_k A0^2 f_k^(-7/3) over bins below f_ISCO,
    against the integral (3/4) A0^2 (f_a^(-4/3) - f_b^(-4/3)) * 4 plus Euler-Maclaurin end terms."""
    w = inputs.tiny()
    model = helpers.oracle_model(w)
    th = np.array([11.0, 0.75, 0.0, 1.0])
    psd = np.ones((1, w.n_bins))
    ev = oracle.EventHolder(np.zeros((1, w.n_bins, 2)), psd, w.f_min, w.df, inputs.detectors(w))
    hh = -2.0 * oracle.loglike(model, ev, th, grad=False)[0]
    a0 = oracle.amplitude(11.0, 400.0, 1.0)
    fis = oracle.f_isco(11.0, 0.75)
    k_last = min(int(math.floor((fis - w.f_min) / w.df)), w.n_bins - 1)
    fa, fb = w.f_min, w.f_min + k_last * w.df
    g = lambda f: f ** (-7.0 / 3.0)
    dg = lambda f: -7.0 / 3.0 * f ** (-10.0 / 3.0)
    integral = 0.75 * (fa ** (-4.0 / 3.0) - fb ** (-4.0 / 3.0))
    s = integral / w.df + 0.5 * (g(fa) + g(fb)) - w.df / 12.0 * (dg(fa) - dg(fb))
    want = 4.0 * w.df * a0 ** 2 * s
    assert hh == pytest.approx(want, rel=1e-8)


# ------------------------------------------------------- antenna patterns
def _textbook(theta, phi, psi):
    c = math.cos(theta)
    fp = 0.5 * (1 + c * c) * math.cos(2 * phi) * math.cos(2 * psi) - c * math.sin(2 * phi) * math.sin(2 * psi)
    fc = 0.5 * (1 + c * c) * math.cos(2 * phi) * math.sin(2 * psi) + c * math.sin(2 * phi) * math.cos(2 * psi)
    return fp, fc


def test_antenna_textbook_frame():
    """Detector at the north pole with arm azimuth a: source polar angle
    theta = pi/2 - dec, azimuth from the first arm phi' = ra - (pi - a).
    The arm frame (azimuth clockwise from north) is left-handed, so the
    textbook formula applies at (theta, -phi', pi/2 - psi)."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        a, ra = rng.uniform(0, 2 * math.pi, 2)
        sd, psi = rng.uniform(-1, 1), rng.uniform(0, math.pi)
        fp, fc, dt = oracle.antenna(dict(lat=math.pi / 2, lon=0.0, azimuth=a), ra, sd, psi)
        tp, tc = _textbook(math.pi / 2 - math.asin(sd), -(ra - (math.pi - a)), math.pi / 2 - psi)
        assert fp == pytest.approx(tp, abs=1e-12)
        assert fc == pytest.approx(tc, abs=1e-12)
        assert dt == pytest.approx(-6.371e6 * sd / 299792458.0, rel=1e-12, abs=1e-18)


def test_antenna_invariants():
    """F+^2 + Fx^2 does not depend on psi; F(psi + pi/2) = -F; |delay| <= R/c."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        det = dict(lat=math.asin(rng.uniform(-1, 1)), lon=rng.uniform(0, 6.28), azimuth=rng.uniform(0, 6.28))
        ra, sd, psi = rng.uniform(0, 6.28), rng.uniform(-1, 1), rng.uniform(0, 3.14)
        a = oracle.antenna(det, ra, sd, psi)
        b = oracle.antenna(det, ra, sd, psi + 0.7)
        c = oracle.antenna(det, ra, sd, psi + math.pi / 2)
        assert a[0] ** 2 + a[1] ** 2 == pytest.approx(b[0] ** 2 + b[1] ** 2, rel=1e-12)
        assert c[0] == pytest.approx(-a[0], abs=1e-12) and c[1] == pytest.approx(-a[1], abs=1e-12)
        assert abs(a[2]) <= 6.371e6 / 299792458.0 * (1 + 1e-12)
        assert a[0] ** 2 + a[1] ** 2 <= 1.0 + 1e-12


# --------------------------------------------------------------- likelihood
def test_loglike_noiseless_maximum():
    """d = h(theta0), no noise: ln L(theta0) = 0 and grad ln L(theta0) = 0."""
    w = inputs.bbh11()
    ev, th, _ = helpers.make_event(w, seed=0, with_noise=False)
    model = helpers.oracle_model(w)
    lnl, g = oracle.loglike(model, ev, th)
    assert abs(lnl[0]) < 1e-9
    widths = np.array(w.hi) - np.array(w.lo)
    assert np.max(np.abs(g[0] * widths)) < 1e-5
    # a nearby point is strictly worse
    th2 = th.copy()
    th2[0] += 1e-3
    assert oracle.loglike(model, ev, th2, grad=False)[0] < -1e-6


def test_loglike_decomposition():
    """Literal -1/2 sum w |d-h|^2 equals Re<d|h> - <h|h>/2 - <d|d>/2 built from the waveform."""
    w = inputs.bbh11()
    ev, th_inj, data = helpers.make_event(w, seed=1)
    model = helpers.oracle_model(w)
    wts = 4.0 * w.df / inputs.psd_array(w)
    thetas = np.vstack([th_inj, inputs.prior_draws(w, 3, 5)])
    lnl = oracle.loglike(model, ev, thetas, grad=False)
    d = data[..., 0] + 1j * data[..., 1]
    for i, th in enumerate(thetas):
        h = oracle.waveform(model, ev, th)
        h = h[..., 0] + 1j * h[..., 1]
        want = np.sum(wts * (np.conj(d) * h).real) - 0.5 * np.sum(wts * abs(h) ** 2) - 0.5 * np.sum(wts * abs(d) ** 2)
        assert lnl[i] == pytest.approx(want, abs=1e-8 * np.sum(wts * abs(d) ** 2))


def test_injection_snr_rescale():
    w = inputs.bbh11()
    model = helpers.oracle_model(w)
    th = helpers.injection(w, 0)
    assert helpers.snr(w, model, th) == pytest.approx(20.0, rel=1e-9) or th[4] in (100.0, 5000.0)


def test_gradient_central_differences():
    """Oracle gradient (forward-mode duals) vs central differences, h = 1e-6 relative, 64 seeded theta
    (prior draws and a ball around the injection). Components whose +-h step changes the set of bins
    below f_ISCO are skipped (the cut is a discontinuity)."""
    w = inputs.bbh11()
    ev, th_inj, _ = helpers.make_event(w, seed=0)
    model = helpers.oracle_model(w)
    thetas = np.vstack([inputs.prior_draws(w, 32, 11), inputs.ball(w, th_inj, 32, 12)])
    lnl, g = oracle.loglike(model, ev, thetas)
    widths = np.array(w.hi) - np.array(w.lo)
    checked = 0
    for i, th in enumerate(thetas):
        pts = []
        hs = []
        for j in range(w.n_dim):
            h = 1e-6 * abs(th[j]) if abs(th[j]) > 1e-3 * widths[j] else 1e-6 * widths[j]
            hs.append(h)
            for s in (+1, -1):
                t = th.copy()
                t[j] += s * h
                pts.append(t)
        vals = oracle.loglike(model, ev, np.array(pts), grad=False).reshape(w.n_dim, 2)
        fd = (vals[:, 0] - vals[:, 1]) / (2 * np.array(hs))
        kis = lambda t: math.floor((oracle.f_isco(t[0], t[1]) - w.f_min) / w.df)
        k0 = kis(th)
        for j in range(w.n_dim):
            if j in (0, 1):
                tp, tm = th.copy(), th.copy()
                tp[j] += hs[j]
                tm[j] -= hs[j]
                if kis(tp) != k0 or kis(tm) != k0:
                    continue
            scale = max(abs(g[i, j]), 1e-3 * np.linalg.norm(g[i] * widths) / widths[j], 1e-8)
            assert abs(fd[j] - g[i, j]) <= 2e-4 * scale, (i, j, fd[j], g[i, j])
            checked += 1
    assert checked > 0.9 * 64 * w.n_dim


# ------------------------------------------------------------------ prior
def test_prior_density_normalised():
    """The prior density integrates to one over the box (power-law d^2 on d_L)."""
    w = inputs.bbh11()
    model = helpers.oracle_model(w)
    x = np.linspace(100, 5000, 200001)
    th = np.tile(inputs.injection(w), (x.size, 1))
    th[:, 4] = x
    lp, g = oracle.prior_logpdf_grad(model, th)
    others = sum(-math.log(h - l) for k, (l, h) in enumerate(zip(w.lo, w.hi)) if k != 4)
    dens = np.exp(lp - others)
    assert np.trapezoid(dens, x) == pytest.approx(1.0, rel=1e-8)
    assert g[:, 4] == pytest.approx(2.0 / x, rel=1e-12)
    out = th[:2].copy()
    out[0, 0] = 50.0
    assert oracle.prior_logpdf_grad(model, out)[0][0] == -np.inf


def test_prior_sample_distribution():
    w = inputs.bbh11()
    model = helpers.oracle_model(w)
    th = oracle.prior_sample(model, 20000, key=5)
    lo, hi = np.array(w.lo), np.array(w.hi)
    assert np.all(th >= lo) and np.all(th <= hi)
    u = (th[:, 0] - lo[0]) / (hi[0] - lo[0])
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    cdf = (th[:, 4] ** 3 - 100.0 ** 3) / (5000.0 ** 3 - 100.0 ** 3)
    assert stats.kstest(cdf, "uniform").pvalue > 1e-3


# --------------------------------------------------- ESS and resampling
def test_ess_special_cases():
    bn, dl, ess, wts = oracle.smc_reweight(np.full(64, -3.0), 0.2, 0.5)
    assert bn == 1.0 and ess == pytest.approx(64.0) and dl == pytest.approx(0.8 * -3.0)
    lnl = np.full(16, -np.inf)
    lnl[5] = -1.0
    bn, dl, ess, wts = oracle.smc_reweight(lnl, 0.0, 0.5)
    assert ess == pytest.approx(1.0) and wts[5] == 1.0 and wts.sum() == 1.0


def test_adaptive_beta_hits_target_ess():
    """Eq. (6): the chosen increment makes ESS = alpha N (to bisection precision)."""
    rng = np.random.default_rng(4)
    lnl = -0.5 * rng.chisquare(11, size=2048) * 30
    bn, dl, ess, wts = oracle.smc_reweight(lnl, 0.0, 0.5)
    assert 0 < bn < 1
    assert ess == pytest.approx(0.5 * 2048, rel=1e-9)
    # evidence increment = log mean of L^dbeta (Eq. 7)
    want = np.log(np.mean(np.exp(bn * (lnl - lnl.max())))) + bn * lnl.max()
    assert dl == pytest.approx(want, rel=1e-12)


def test_systematic_counts_brute_force():
    """For N <= 8 every count lies in {floor(N W_i), ceil(N W_i)} (to one quantum) and sums to N."""
    rng = np.random.default_rng(5)
    for n in range(1, 9):
        for _ in range(200):
            w = rng.uniform(0, 1, n) ** 3
            w /= w.max()
            u = rng.uniform()
            anc = oracle.systematic_resample(w, u)
            counts = np.bincount(anc, minlength=n)
            assert counts.sum() == n and np.all(np.diff(anc) >= 0)
            q = np.floor(w * 2.0 ** 32)
            nw = n * q / q.sum()
            assert np.all(counts >= np.floor(nw - 1e-9)) and np.all(counts <= np.ceil(nw + 1e-9))


def test_systematic_unbiased_over_u_grid():
    """Averaged over a uniform grid of u the counts equal N * Wbar exactly (systematic resampling is
    unbiased); checked with exact integers."""
    rng = np.random.default_rng(6)
    n = 7
    w = rng.uniform(0.05, 1, n)
    w /= w.max()
    q = np.floor(w * 2.0 ** 32).astype(np.int64)
    grid = 1 << 12
    tot = np.zeros(n)
    for g in range(grid):
        anc = oracle.systematic_resample(w, g / grid)
        tot += np.bincount(anc, minlength=n)
    mean = tot / grid
    assert np.allclose(mean, n * q / q.sum(), atol=2.0 * n / grid)


def test_weighted_cov_matches_numpy():
    rng = np.random.default_rng(7)
    th = rng.normal(size=(500, 5)) @ rng.normal(size=(5, 5))
    w = rng.uniform(size=500)
    assert np.allclose(oracle.weighted_cov(th, w), np.cov(th.T, aweights=w, bias=True), rtol=1e-10, atol=1e-12)
