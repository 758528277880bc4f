"""Pins for the oracle's cosmology and time-integration coefficients (CPU only)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import cosmo

THETA = (2.1e-9, 0.965, 0.31, 0.049, 0.68)


def test_growth_matter_dominated_is_exact():
    """App. A: with Omega_m = 1 the growing mode is D1 = a exactly (G1 = 1, G1' = 0)."""
    a = np.array([1e-3, 1 / 64, 0.3, 1.0])
    g, dg = cosmo.growth_g1(a, 1.0)
    assert np.allclose(g, 1.0, rtol=0, atol=1e-13)
    assert np.allclose(dg, 0.0, rtol=0, atol=1e-13)
    d1, dd1, gd, gk = cosmo.growth_factors(a, 1.0)
    # G_D = a^2 H D1' with H = a^-3/2, D1' = a  ->  a^{3/2};  G_K = 3/2 D1
    assert np.allclose(gd, a ** 1.5, rtol=1e-13)
    assert np.allclose(gk, 1.5 * a, rtol=1e-13)


@pytest.mark.parametrize("Om", [0.25, 0.31, 0.35])
def test_growth_lcdm_matches_integral_form(Om):
    """Flat LCDM growing mode D1 = 5/2 Om E(a) int_0^a da / (a E)^3 (Heath 1977),
    normalised to D1 -> a early, as the ODE initial conditions of App. A (Eq. 57)."""
    a = np.array([1 / 64, 0.1, 0.5, 1.0])
    d1, _, _, _ = cosmo.growth_factors(a, Om)
    for ai, di in zip(a, d1):
        val, _ = integrate.quad(lambda x: (x * cosmo.hubble(x, Om)) ** -3, 0, ai,
                                epsabs=0, epsrel=1e-13, limit=200)
        heath = 2.5 * Om * cosmo.hubble(ai, Om) * val
        assert abs(di / heath - 1) < 1e-8


def test_gk_closed_form_equals_eq58():
    """G_K = a^3 H^2 [D1'' + (2 + H'/H) D1'] (App. A, Eq. 58) equals 3/2 Om D1."""
    Om = 0.31
    a = np.array([1 / 64, 0.2, 0.7, 1.0])
    g, dg = cosmo.growth_g1(a, Om)
    om_a = cosmo.omega_m_of_a(a, Om)
    dlnh = -1.5 * om_a
    ddg = -(4 + dlnh) * dg - (3 + dlnh - 1.5 * om_a) * g
    dd1 = a * (g + dg)
    ddd1 = a * (g + 2 * dg + ddg)
    gk58 = a ** 3 * cosmo.hubble(a, Om) ** 2 * (ddd1 + (2 + dlnh) * dd1)
    d1, _, _, gk = cosmo.growth_factors(a, Om)
    assert np.allclose(gk58, gk, rtol=1e-12)
    assert np.allclose(gk, 1.5 * Om * d1, rtol=1e-14)


def test_gd_equals_a2_times_time_derivative_of_d1():
    """G_D = a^2 dD1/dt (Eq. 14) checked by a central difference of D1 in t, dt = da/(aH)."""
    Om = 0.31
    a = 0.4
    eps = 1e-5
    d1p = cosmo.growth_factors(np.array([a * (1 + eps)]), Om)[0][0]
    d1m = cosmo.growth_factors(np.array([a * (1 - eps)]), Om)[0][0]
    dd1_dlna = (d1p - d1m) / (np.log(1 + eps) - np.log(1 - eps))
    gd = cosmo.growth_factors(np.array([a]), Om)[2][0]
    assert abs(gd / (a ** 2 * cosmo.hubble(a, Om) * dd1_dlna) - 1) < 1e-7


def test_kdk_factor_derivative_complex_step_vs_central_fd():
    agrid = cosmo.time_grid(1 / 64, 1.0, 12)
    cs = [cosmo.complex_step(lambda th: cosmo.kdk_factors(agrid, th[2])[j], THETA, 2) for j in range(3)]
    h = 1e-6
    for j in range(3):
        fp = cosmo.kdk_factors(agrid, THETA[2] + h)[j]
        fm = cosmo.kdk_factors(agrid, THETA[2] - h)[j]
        assert np.allclose(cs[j], (fp - fm) / (2 * h), rtol=1e-6)


def test_transfer_limits():
    """T(k) -> 1 as k -> 0 and decreases monotonically (the only pins: parity unpinned)."""
    k = np.logspace(-5, 2, 400)
    t = cosmo.transfer_eh_nowiggle(k, 0.31, 0.049, 0.68)
    assert abs(t[0] - 1) < 1e-3
    assert np.all(np.diff(t) < 0)
    assert np.all(t > 0)


def test_transfer_zero_baryon_scaling():
    """With Omega_b = 0, alpha_Gamma = 1 and Gamma = Omega_m h: T depends on k only
    through q = k Theta^2 / (Omega_m h), so (k, h) -> (c k, c h) leaves T unchanged."""
    k = np.logspace(-3, 1, 50)
    t1 = cosmo.transfer_eh_nowiggle(k, 0.3, 0.0, 0.7)
    t2 = cosmo.transfer_eh_nowiggle(2.0 * k, 0.3, 0.0, 1.4)
    assert np.allclose(t1, t2, rtol=1e-13)


def test_plin_parameter_dependence():
    """Eq. 7: P is linear in A_s, scales as (k/k_pivot)^(n_s-1) and as Omega_m^-2 T^2."""
    k = np.array([0.01, 0.1, 1.0])
    p0 = cosmo.plin(k, THETA)
    th = list(THETA)
    th[0] *= 2
    assert np.allclose(cosmo.plin(k, th), 2 * p0, rtol=1e-14)
    th = list(THETA)
    th[1] += 0.1
    kp = cosmo.K_PIVOT / THETA[4]
    assert np.allclose(cosmo.plin(k, th) / p0, (k / kp) ** 0.1, rtol=1e-12)
    d = cosmo.complex_step(lambda t: np.log(cosmo.plin(k, t)), THETA, 0)
    assert np.allclose(d, 1 / THETA[0], rtol=1e-12)


# ------------------------------------------------------------ second-order growth (2LPT)

def test_second_order_growth_matter_dominated_is_exact():
    """App. A: with Omega_m = 1 the second-order growing mode is D2 = 3/7 a^2 exactly
    (G2 = 3/7 solves Eq. 56 with G1 = 1); D2' = 2 D2 then."""
    a = np.array([1e-3, 1 / 64, 0.3, 1.0])
    g, dg = cosmo.growth_g2(a, 1.0)
    assert np.allclose(g, 3.0 / 7.0, rtol=0, atol=1e-13)
    assert np.allclose(dg, 0.0, rtol=0, atol=1e-13)
    d2, dd2, gd2 = cosmo.growth_factors2(a, 1.0)
    assert np.allclose(dd2, 2.0 * d2, rtol=1e-13)
    assert np.allclose(gd2, a ** 2 * a ** -1.5 * dd2, rtol=1e-13)


@pytest.mark.parametrize("Om", [0.25, 0.31, 0.35])
def test_second_order_growth_matches_d_form_ode(Om):
    """The G-form integration (Eq. 56) against an independent adaptive integration of the
    D-form ODEs (Eq. 52): D'' + (2 + H'/H) D' - 3/2 Om(a) D = {0, 3/2 Om(a) D1^2}, from the
    growing-mode values of Eq. 54 at a_ic."""
    def rhs(lna, y):
        a = np.exp(lna)
        om = cosmo.omega_m_of_a(a, Om)
        dlnh = -1.5 * om
        d1, dd1, d2, dd2 = y
        return [dd1, -(2 + dlnh) * dd1 + 1.5 * om * d1,
                dd2, -(2 + dlnh) * dd2 + 1.5 * om * d2 + 1.5 * om * d1 * d1]
    a = np.array([1 / 64, 0.1, 0.5, 1.0])
    ai = cosmo.A_IC
    sol = integrate.solve_ivp(rhs, (np.log(ai), 0.0), [ai, ai, 3 / 7 * ai ** 2, 6 / 7 * ai ** 2],
                              method="DOP853", t_eval=np.log(a), rtol=1e-12, atol=1e-30)
    d2, dd2, _ = cosmo.growth_factors2(a, Om)
    assert np.allclose(d2, sol.y[2], rtol=1e-8, atol=0)
    assert np.allclose(dd2, sol.y[3], rtol=1e-8, atol=0)
    d1 = cosmo.growth_factors(a, Om)[0]
    assert np.allclose(d1, sol.y[0], rtol=1e-8, atol=0)


def test_second_order_growth_matches_bouchet_fit():
    """Flat LCDM: D2 = 3/7 D1^2 Omega_m(a)^(-1/143) to better than 1e-3 (Bouchet et al.
    1995 fit), so the sign and normalisation of D2 in Eq. 2 are the standard 2LPT ones."""
    a = np.array([1 / 64, 0.2, 0.5, 1.0])
    for Om in (0.25, 0.31):
        d1 = cosmo.growth_factors(a, Om)[0]
        d2 = cosmo.growth_factors2(a, Om)[0]
        fit = 3.0 / 7.0 * d1 ** 2 * cosmo.omega_m_of_a(a, Om) ** (-1.0 / 143.0)
        assert np.all(np.abs(d2 / fit - 1) < 1e-3)


# ------------------------------------------- linear power spectrum against published values
# Planck 2018 results VI (Planck Collaboration, A&A 641, A6, 2020), Table 2, column
# "TT,TE,EE+lowE+lensing": ln(10^10 A_s) = 3.044, n_s = 0.9649, Omega_m = 0.3153,
# Omega_b h^2 = 0.02237, H0 = 67.36 km/s/Mpc; derived sigma_8 = 0.8111 and
# r_drag = 147.09 Mpc.
PLANCK18_H = 0.6736
PLANCK18 = (np.exp(3.044) * 1e-10, 0.9649, 0.3153, 0.02237 / PLANCK18_H ** 2, PLANCK18_H)
PLANCK18_SIGMA8 = 0.8111
PLANCK18_RDRAG_MPC = 147.09


def _sigma8(theta):
    """RMS linear overdensity in spheres of 8 Mpc/h at a = 1: P_lin of Eq. 7 times D1(1)^2
    (P_lin is normalised to D1 = a early), top-hat window 3 (sin x - x cos x) / x^3."""
    d1 = cosmo.growth_factors(np.array([1.0]), theta[2])[0][0]

    def integrand(lnk):
        k = np.exp(lnk)
        x = 8.0 * k
        w = 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3
        return k ** 3 * cosmo.plin(k, theta) / (2.0 * np.pi ** 2) * w * w

    val, _ = integrate.quad(integrand, np.log(1e-5), np.log(1e2), limit=500, epsrel=1e-10)
    return np.sqrt(val) * d1


def test_sigma8_against_planck2018():
    """The amplitude chain of Eq. 7 (4/25 A_s, (c k / H0)^4 / Omega_m^2, the pivot in h
    units, the growth normalisation D1 -> a) and T(k) together give sigma_8 within 5% of
    Planck 2018's 0.8111 at Planck's parameters.  The oracle lands 3% high: Planck's base
    model carries 0.06 eV of neutrino mass (about 2% less sigma_8) and the no-wiggle fit
    is a smooth approximation.  A wrong amplitude factor (2/5 for 4/25), a renormalised
    D1(1) = 1 (+27%) or a wrong power of c/H0 fail it."""
    s8 = _sigma8(PLANCK18)
    assert abs(s8 / PLANCK18_SIGMA8 - 1) < 0.05, s8


def test_sound_horizon_against_planck2018_rdrag():
    """Eisenstein & Hu (1998) Eq. 26 approximates the sound horizon at the drag epoch to a
    few per cent: at Planck 2018's Omega_m h^2 and Omega_b h^2 it is within 3% of the
    published r_drag = 147.09 Mpc (the oracle gives 149.8 Mpc)."""
    h = PLANCK18_H
    s = cosmo.sound_horizon_eh(PLANCK18[2] * h * h, PLANCK18[3] * h * h)
    assert abs(s / PLANCK18_RDRAG_MPC - 1) < 0.03, s


def test_gamma_eff_limits_with_baryons():
    """Eq. 30 of Eisenstein & Hu (1998) at finite f_b: Gamma_eff -> Omega_m h on scales
    much larger than the sound horizon and -> alpha_Gamma Omega_m h on much smaller
    scales, with alpha_Gamma < 1 (baryons suppress small-scale power)."""
    Om, Ob, h = 0.31, 0.049, 0.68
    alpha = cosmo.alpha_gamma(Om * h * h, Ob / Om)
    assert 0.7 < alpha < 0.9
    assert abs(cosmo.gamma_eff(1e-5, Om, Ob, h) / (Om * h) - 1) < 1e-9
    assert abs(cosmo.gamma_eff(1e3, Om, Ob, h) / (alpha * Om * h) - 1) < 1e-9


def test_transfer_zero_baryon_against_bbks():
    """Without baryons the no-wiggle form reduces to a pure CDM transfer function, which
    the Bardeen, Bond, Kaiser & Szalay (1986, ApJ 304, 15, their Eq. G3) fit also
    describes: T = ln(1 + 2.34 q) / (2.34 q) [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3 +
    (6.71 q)^4]^(-1/4), q = k / (Omega_m h) with k in h/Mpc.  The two independent fits agree
    within 7% from 1e-3 to 10 h/Mpc (the largest gap, 5.6%, near k = 0.1)."""
    Om, h = 0.31, 0.68
    k = np.logspace(-3, 1, 60)
    t = cosmo.transfer_eh_nowiggle(k, Om, 0.0, h)
    q = k / (Om * h)
    bbks = np.log(1 + 2.34 * q) / (2.34 * q) * (1 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3
                                                 + (6.71 * q) ** 4) ** -0.25
    assert np.all(np.abs(t / bbks - 1) < 0.07)


def test_pivot_scale_in_h_units():
    """Eq. 7: at the pivot k_pivot = 0.05/Mpc, i.e. k = 0.05/h in h/Mpc, the tilt n_s has
    no effect on P_lin; 0.05 h/Mpc (a pivot in the wrong units) is not invariant."""
    kp = np.array([cosmo.K_PIVOT / THETA[4]])
    th = list(THETA)
    th[1] = 0.90
    assert abs(cosmo.plin(kp, th)[0] / cosmo.plin(kp, THETA)[0] - 1) < 1e-13
    assert abs(cosmo.plin(np.array([0.05]), th)[0] / cosmo.plin(np.array([0.05]), THETA)[0] - 1) > 1e-3
