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
