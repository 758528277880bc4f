"""Oracle (test infrastructure): cosmology and time-integration coefficients in float64.

Units (the paper fixes none): lengths in Mpc/h, wavenumbers in h/Mpc, time in 1/H0 so
that H0 = 1, flat LCDM without radiation, H(a)/H0 = sqrt(Om a^-3 + 1 - Om).  The
parameter vector is theta = (A_s, n_s, Omega_m, Omega_b, h) (Sec. 2.1).  Every function
accepts complex theta so that derivatives can be taken by the complex step
df/dx = Im f(x + i eps) / eps, which is exact to rounding for analytic functions.
"""
import numpy as np

C_OVER_H0 = 2997.92458     # c / (100 km/s/Mpc) in Mpc/h
T_CMB = 2.7255             # K
K_PIVOT = 0.05             # 1/Mpc (not h/Mpc); the paper leaves it unstated
A_IC = 1e-4                # start of the growth integration (App. A leaves it unstated)
LNA_STEP = 1.0 / 512.0     # largest RK4 step in ln a

THETA_NAMES = ("A_s", "n_s", "Omega_m", "Omega_b", "h")


def hubble(a, Om):
    """E(a) = H(a)/H0 for flat LCDM (reading of the units; Sec. 2.1 and App. A)."""
    return np.sqrt(Om * a ** -3 + (1.0 - Om))


def omega_m_of_a(a, Om):
    """Omega_m(a) = Omega_m H0^2 / (a^3 H^2)  (App. A, Eq. 53)."""
    return Om * a ** -3 / hubble(a, Om) ** 2


def _growth_rhs(lna, y, Om):
    """Right-hand side of the first-order suppression-factor ODE (App. A, Eq. 56).

    y = (G1, G1') with ' = d/d ln a.  With H'/H = -3/2 Omega_m(a) for flat LCDM,
    G1'' = -(4 + H'/H) G1' - (3 + H'/H - 3/2 Omega_m(a)) G1.
    """
    a = np.exp(lna)
    om = omega_m_of_a(a, Om)
    dlnh = -1.5 * om
    g, dg = y
    ddg = -(4.0 + dlnh) * dg - (3.0 + dlnh - 1.5 * om) * g
    return np.array([dg, ddg])


def growth_g1(a_targets, Om):
    """G1 = D1/a and G1' = dG1/dln a at each a in ``a_targets`` (App. A, Eqs. 55-57).

    Classical RK4 in ln a from a_ic = 1e-4 with G1 = 1, G1' = 0 (Eq. 57), stepping to
    each target exactly (no interpolation) with steps no larger than 1/512 in ln a.
    Pinned: Omega_m = 1 gives G1 = 1 exactly; for LCDM D1 matches the integral form
    D1 ~ H(a) int da / (a H)^3 (tests/test_oracle_cosmo.py).
    """
    a_targets = np.asarray(a_targets, dtype=np.float64)
    order = np.argsort(a_targets)
    out_g = np.zeros(a_targets.shape, dtype=np.result_type(Om, np.float64))
    out_dg = np.zeros_like(out_g)
    y = np.array([1.0 + 0.0 * Om, 0.0 * Om])
    lna = np.log(A_IC)
    for idx in order:
        target = np.log(a_targets[idx])
        span = target - lna
        nsub = int(np.ceil(span / LNA_STEP)) if span > 0 else 0
        if nsub > 0:
            h = span / nsub
            for _ in range(nsub):
                k1 = _growth_rhs(lna, y, Om)
                k2 = _growth_rhs(lna + 0.5 * h, y + 0.5 * h * k1, Om)
                k3 = _growth_rhs(lna + 0.5 * h, y + 0.5 * h * k2, Om)
                k4 = _growth_rhs(lna + h, y + h * k3, Om)
                y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
                lna = lna + h
            lna = target
        out_g[idx] = y[0]
        out_dg[idx] = y[1]
    return out_g, out_dg


def growth_factors(a, Om):
    """D1, D1' (= dD1/dln a), G_D and G_K at scale factors ``a``.

    D1 = a G1 and D1' = a (G1 + G1') (App. A, Eq. 59 with m = 1);
    G_D = a^2 H D1' (App. A, Eq. 58);
    G_K = a^3 H^2 [D1'' + (2 + H'/H) D1'], which by the D1 growth equation (App. A,
    Eq. 52) equals (3/2) Omega_m H0^2 D1 -- the closed form used here.  The test suite
    checks it against the Eq. 58 form evaluated with D1'' from the ODE.
    """
    a = np.asarray(a, dtype=np.float64)
    g, dg = growth_g1(a, Om)
    d1 = a * g
    dd1 = a * (g + dg)
    gd = a ** 2 * hubble(a, Om) * dd1
    gk = 1.5 * Om * d1
    return d1, dd1, gd, gk


def _growth2_rhs(lna, y, Om):
    """Both suppression-factor ODEs of App. A (Eq. 56) as one first-order system.

    y = (G1, G1', G2, G2'), ' = d/d ln a, H'/H = -3/2 Omega_m(a) (flat LCDM):
      G1'' = -(4 + H'/H) G1' - (3 + H'/H - 3/2 Omega_m(a)) G1
      G2'' = -(6 + H'/H) G2' - (8 + 2 H'/H - 3/2 Omega_m(a)) G2 + 3/2 Omega_m(a) G1^2
    """
    a = np.exp(lna)
    om = omega_m_of_a(a, Om)
    dlnh = -1.5 * om
    g1, dg1, g2, dg2 = y
    ddg1 = -(4.0 + dlnh) * dg1 - (3.0 + dlnh - 1.5 * om) * g1
    ddg2 = -(6.0 + dlnh) * dg2 - (8.0 + 2.0 * dlnh - 1.5 * om) * g2 + 1.5 * om * g1 * g1
    return np.array([dg1, ddg1, dg2, ddg2])


def growth_g2(a_targets, Om):
    """G2 = D2/a^2 and G2' at each a in ``a_targets`` (App. A, Eqs. 55-57, second order).

    The same RK4 scheme as ``growth_g1`` on the joint system (G1, G1', G2, G2') from
    a_ic = 1e-4 with G1 = 1, G1' = 0, G2 = 3/7, G2' = 0 (Eq. 57).  Pinned: Omega_m = 1
    gives G2 = 3/7 exactly; for LCDM D2 matches an independent adaptive integration of
    the D-form ODE (Eq. 52) and the Bouchet et al. (1995) fit D2 ~ 3/7 D1^2
    Omega_m(a)^(-1/143) (tests/test_oracle_cosmo.py).
    """
    a_targets = np.asarray(a_targets, dtype=np.float64)
    order = np.argsort(a_targets)
    out_g = np.zeros(a_targets.shape, dtype=np.result_type(Om, np.float64))
    out_dg = np.zeros_like(out_g)
    y = np.array([1.0 + 0.0 * Om, 0.0 * Om, 3.0 / 7.0 + 0.0 * Om, 0.0 * Om])
    lna = np.log(A_IC)
    for idx in order:
        target = np.log(a_targets[idx])
        span = target - lna
        nsub = int(np.ceil(span / LNA_STEP)) if span > 0 else 0
        if nsub > 0:
            h = span / nsub
            for _ in range(nsub):
                k1 = _growth2_rhs(lna, y, Om)
                k2 = _growth2_rhs(lna + 0.5 * h, y + 0.5 * h * k1, Om)
                k3 = _growth2_rhs(lna + 0.5 * h, y + 0.5 * h * k2, Om)
                k4 = _growth2_rhs(lna + h, y + h * k3, Om)
                y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
                lna = lna + h
            lna = target
        out_g[idx] = y[2]
        out_dg[idx] = y[3]
    return out_g, out_dg


def growth_factors2(a, Om):
    """D2, D2' and G_D2 = a^2 H D2' at scale factors ``a`` (second-order LPT growth).

    D2 = a^2 G2 and D2' = a^2 (2 G2 + G2') (App. A, Eq. 59 for m = 2, read with G_m' in
    place of the printed G_1'); G_D2 is the factor of s2 in the 2LPT momentum,
    p = a^2 H (D1' s1 + D2' s2) (Sec. 2.1, Eq. 2)."""
    a = np.asarray(a, dtype=np.float64)
    g, dg = growth_g2(a, Om)
    d2 = a * a * g
    dd2 = a * a * (2.0 * g + dg)
    return d2, dd2, a ** 2 * hubble(a, Om) * dd2


def time_grid(a0, a1, n_steps):
    """Scale factors a_0..a_n linear in a (Sec. 4, 'time steps linearly spaced in a')."""
    return a0 + (a1 - a0) * np.arange(n_steps + 1, dtype=np.float64) / n_steps


def kdk_factors(a_grid, Om):
    """FastPM kick/drift factors for each step i = 1..n (Sec. 2.3, Eqs. 15-16).

    With a_{i-1/2} the arithmetic mean of a_{i-1} and a_i (the paper does not fix it):
      K1_i = K(t_{i-1}, t_{i-1}, t_{i-1/2}) = [G_D(a_{i-1/2}) - G_D(a_{i-1})] / G_K(a_{i-1})
      D_i  = D(t_{i-1/2}, t_{i-1}, t_i)    = [D1(a_i) - D1(a_{i-1})] / G_D(a_{i-1/2})
      K2_i = K(t_i, t_{i-1/2}, t_i)        = [G_D(a_i) - G_D(a_{i-1/2})] / G_K(a_i)
    Returns arrays (K1, D, K2), each of length n.  Pinned by the Zel'dovich exactness of
    the leapfrog with the linear-theory force (tests/test_oracle_pm.py).
    """
    a_grid = np.asarray(a_grid, dtype=np.float64)
    a_half = 0.5 * (a_grid[:-1] + a_grid[1:])
    d1, _, gd, gk = growth_factors(a_grid, Om)
    d1h, _, gdh, _ = growth_factors(a_half, Om)
    k1 = (gdh - gd[:-1]) / gk[:-1]
    dd = (d1[1:] - d1[:-1]) / gdh
    k2 = (gd[1:] - gdh) / gk[1:]
    return k1, dd, k2


def partial_drift_factor(a, a_grid, j, Om):
    """Drift factor from a_j to a in (a_j, a_{j+1}] with the half-step momentum p_{j+1/2}:
    the FastPM drift D of Sec. 2.3 (Eq. 15) evaluated up to a instead of a_{j+1},
    [D1(a) - D1(a_j)] / G_D(a_{j+1/2}) -- the reading used for positions interpolated
    between two steps (Sec. 2.4 names such snapshots without a formula).  Equals D_{j+1}
    of ``kdk_factors`` at a = a_{j+1}."""
    a_grid = np.asarray(a_grid, dtype=np.float64)
    d1 = growth_factors(np.array([a_grid[j], a]), Om)[0]
    gdh = growth_factors(np.array([0.5 * (a_grid[j] + a_grid[j + 1])]), Om)[2]
    return (d1[1] - d1[0]) / gdh[0]


def sound_horizon_eh(omh2, obh2):
    """Sound horizon at the drag epoch in Mpc (not Mpc/h): the Eisenstein & Hu (1998,
    ApJ 496, 605) fit, their Eq. 26, s = 44.5 ln(9.83 / Omega_m h^2) /
    sqrt(1 + 10 (Omega_b h^2)^(3/4)).  Pinned against Planck 2018's r_drag
    (tests/test_oracle_cosmo.py)."""
    return 44.5 * np.log(9.83 / omh2) / np.sqrt(1.0 + 10.0 * obh2 ** 0.75)


def alpha_gamma(omh2, fb):
    """Small-scale suppression of the shape parameter by baryons, Eisenstein & Hu (1998)
    Eq. 31: alpha_Gamma = 1 - 0.328 ln(431 Omega_m h^2) f_b + 0.38 ln(22.3 Omega_m h^2)
    f_b^2, f_b = Omega_b / Omega_m.  Pinned only through sigma_8 (the f_b^2 term moves
    sigma_8 by 0.2%: parity unpinned beyond that)."""
    return 1.0 - 0.328 * np.log(431.0 * omh2) * fb + 0.38 * np.log(22.3 * omh2) * fb * fb


def gamma_eff(k, Om, Ob, h):
    """Scale-dependent shape parameter of the no-wiggle transfer function, Eisenstein & Hu
    (1998) Eq. 30, k in h/Mpc: Gamma_eff = Omega_m h [alpha + (1 - alpha) /
    (1 + (0.43 k s)^4)] with k s in Mpc units; Omega_m h on large scales, alpha Omega_m h on
    small scales (pinned by those two limits)."""
    omh2 = Om * h * h
    alpha = alpha_gamma(omh2, Ob / Om)
    s = sound_horizon_eh(omh2, Ob * h * h)
    return Om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k * h * s) ** 4))


def transfer_eh_nowiggle(k, Om, Ob, h, tcmb=T_CMB):
    """Eisenstein & Hu (1998) no-wiggle transfer function, k in h/Mpc (Sec. 2.1).

    The paper names the fitting formula but does not print it.  Transcribed from
    Eisenstein & Hu 1998, ApJ 496, 605: sound horizon fit (their Eq. 26), alpha_Gamma
    (Eq. 31), Gamma_eff (Eq. 30), q (Eq. 28), T0(q) = L0 / (L0 + C0 q^2) (Eq. 29).
    Pinned by its limits (T -> 1 as k -> 0, monotone decrease, the zero-baryon case), the
    zero-baryon form against the BBKS fit, the sound horizon against Planck 2018's r_drag
    and sigma_8 against Planck 2018 (tests/test_oracle_cosmo.py); the f_b^2 coefficient
    of alpha_Gamma is parity unpinned.
    """
    theta27 = tcmb / 2.7
    q = k * theta27 ** 2 / gamma_eff(k, Om, Ob, h)
    l0 = np.log(2.0 * np.e + 1.8 * q)
    c0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return l0 / (l0 + c0 * q * q)


def plin(k, theta):
    """Linear matter power spectrum P_lin(k) in (Mpc/h)^3 at D1 = a normalisation.

    Sec. 2.1, Eq. 7:  k^3 P / (2 pi^2) = 4/25 A_s (k/k_pivot)^(n_s-1) T^2(k) c^4 k^4 /
    (Omega_m^2 H0^4), with k in h/Mpc, k_pivot = 0.05/Mpc = 0.05/h h/Mpc and c/H0 in
    Mpc/h.  k must be > 0.
    """
    As, ns, Om, Ob, h = theta
    t = transfer_eh_nowiggle(k, Om, Ob, h)
    return (2.0 * np.pi ** 2 / k ** 3 * 0.16 * As * (k * h / K_PIVOT) ** (ns - 1.0)
            * t * t * (C_OVER_H0 * k) ** 4 / Om ** 2)


def complex_step(fn, theta, j, eps=1e-30):
    """d fn(theta) / d theta_j by the complex step (exact to rounding for analytic fn)."""
    th = np.array(theta, dtype=np.complex128)
    th[j] += 1j * eps
    return np.imag(fn(th)) / eps
