"""Oracle (test infrastructure): particle-mesh forward model and discrete adjoint, float64.

Conventions (the paper leaves them open; the same readings bind the CUDA library):

* Periodic box of side L, mesh of n_mesh^3 nodes at g * l (l = L / n_mesh), particle
  lattice of n_ptcl^3 points q = j * l_p + l/2 (l_p = L / n_ptcl), arrays in C order with the
  last axis fastest; vector fields are (3, N) with component c along array axis c.
* DFT with e^{-i k.x} and no normalisation forward, 1/N^3 on the inverse; k = 2 pi n / L
  with n in [-N/2, N/2); the k = 0 mode of every Green's function is 0; a derivative
  -i k_c (or +i k_c) is zeroed on the Nyquist plane of axis c.
* CIC weights by the floor convention: u = x / l, i = floor(u), t = u - i, weight 1 - t to
  node i and t to node i + 1 per axis; the weight gradient is -1/l and +1/l (the right
  derivative at the kink).
* Particle mass m = n_mesh^3 / n_ptcl^3 so that the mean density is 1 and
  delta = rho - 1.
"""
from dataclasses import dataclass
import itertools

import numpy as np

from . import cosmo


@dataclass(frozen=True)
class PMConfig:
    box: float          # L in Mpc/h
    n_mesh: int         # mesh nodes per side
    n_ptcl: int         # particles per side
    a0: float = 1.0 / 64
    a1: float = 1.0
    n_steps: int = 10
    deconv: bool = False
    lpt_order: int = 1  # 1: Zel'dovich initial conditions, 2: 2LPT (Sec. 2.1, Eq. 2)

    @property
    def cell(self):
        return self.box / self.n_mesh

    @property
    def mass(self):
        return float(self.n_mesh) ** 3 / float(self.n_ptcl) ** 3


# ----------------------------------------------------------------------------- lattice

def lattice(cfg):
    """Lagrangian lattice positions q = j l_p + l/2, shape (3, N) (Sec. 2.1, Eq. 1).

    The half-cell offset (a reading: the paper only says "a Cartesian grid") puts
    unperturbed particles at mesh-cell centres, where the CIC weight of Eq. 10 is
    differentiable, instead of on the nodes, where its kink makes the linear response
    of the density depend on the sign of the displacement."""
    n = cfg.n_ptcl
    idx = np.indices((n, n, n)).reshape(3, -1).astype(np.float64)
    return idx * (cfg.box / n) + 0.5 * cfg.cell


def _kgrid(n, box):
    """Wavevector components on the rfftn layout (last axis halved) and n^2 = |n|^2."""
    f = np.fft.fftfreq(n, d=1.0 / n)                # integers in [-n/2, n/2)
    n0 = f.reshape(n, 1, 1)
    n1 = f.reshape(1, n, 1)
    n2 = np.arange(n // 2 + 1, dtype=np.float64).reshape(1, 1, n // 2 + 1)
    kf = 2.0 * np.pi / box
    return (kf * n0, kf * n1, kf * n2), (n0, n1, n2)


def _derivative_multipliers(n, box):
    """i k_c with the Nyquist plane of axis c zeroed, and k^2 (k = 0 set to 1)."""
    (k0, k1, k2), (n0, n1, n2) = _kgrid(n, box)
    ks = []
    for kc, nc in ((k0, n0), (k1, n1), (k2, n2)):
        ks.append(np.where(np.abs(nc) == n // 2, 0.0, kc))
    k2sum = k0 ** 2 + k1 ** 2 + k2 ** 2
    return ks, k2sum


# ------------------------------------------------------------------ initial conditions

def za_unit_displacement(omega, theta, cfg, dlnp=None):
    """First-order displacement s^(1) on the lattice for unit growth (Sec. 2.1).

    delta1(k) = sqrt(P_lin(k) / l_p^3) * DFT[omega](k)   (Eq. 6 with the lattice
    normalisation <|DFT omega|^2> = N and delta_cont(k) = l_p^3 DFT[delta]);
    s1 = -grad phi_s with laplacian phi_s = delta1 (Eqs. 3-4), i.e.
    s1_c = IDFT[ i k_c / k^2 * delta1(k) ].
    If ``dlnp`` (a callable k -> d ln P / d theta_j) is given, returns
    d s1 / d theta_j = IDFT[ i k_c / k^2 * (1/2 dlnp) * delta1 ] instead.
    Pinned by the ensemble power spectrum of delta1 and by the Zel'dovich growth tests.
    """
    n, box = cfg.n_ptcl, cfg.box
    lp = box / n
    ks, k2 = _derivative_multipliers(n, box)
    k = np.sqrt(k2)
    k_safe = np.where(k2 > 0, k, 1.0)
    amp = np.sqrt(cosmo.plin(k_safe, theta) / lp ** 3)
    if dlnp is not None:
        amp = amp * 0.5 * dlnp(k_safe)
    amp = np.where(k2 > 0, amp, 0.0)
    wk = np.fft.rfftn(np.asarray(omega, dtype=np.float64).reshape(n, n, n))
    dk = amp * wk
    out = np.empty((3, n ** 3))
    for c in range(3):
        out[c] = np.fft.irfftn(1j * ks[c] / np.where(k2 > 0, k2, 1.0) * dk, s=(n, n, n), axes=(0, 1, 2)).ravel()
    return out


def za_initial_state(omega, theta, cfg):
    """Zel'dovich initial conditions at a0: s0 = D1 s1, p0 = G_D s1 (Sec. 2.1, Eq. 2 at
    first order, with p = a^2 H D1' s1 = G_D s1 by Eq. 14/58)."""
    s1 = za_unit_displacement(omega, theta, cfg)
    d1, _, gd, _ = cosmo.growth_factors(np.array([cfg.a0]), theta[2])
    return d1[0] * s1, gd[0] * s1, s1


# ------------------------------------------------------- second-order LPT (Sec. 2.1)

_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def linear_delta_k(omega, theta, cfg, dlnp=None):
    """delta1(k) = sqrt(P_lin(k) / l_p^3) DFT[omega](k) on the rfftn layout of the lattice
    (Eq. 6 with the lattice normalisation of ``za_unit_displacement``), 0 at k = 0.  With
    ``dlnp`` (a callable k -> d ln P / d theta_j) returns d delta1 / d theta_j =
    1/2 dlnp delta1 instead."""
    n, box = cfg.n_ptcl, cfg.box
    lp = box / n
    _, k2 = _derivative_multipliers(n, box)
    k_safe = np.where(k2 > 0, np.sqrt(k2), 1.0)
    amp = np.sqrt(cosmo.plin(k_safe, theta) / lp ** 3)
    if dlnp is not None:
        amp = amp * 0.5 * dlnp(k_safe)
    amp = np.where(k2 > 0, amp, 0.0)
    return amp * np.fft.rfftn(np.asarray(omega, dtype=np.float64).reshape(n, n, n))


def lpt2_hessian(delta_k, cfg):
    """The six second derivatives phi_ij = d_i d_j phi^(1) of the first-order potential,
    laplacian phi^(1) = delta1 (Eq. 4): phi_ij = IDFT[(i k_i)(i k_j)(-1/k^2) delta1(k)] with
    each i k_c zeroed on the Nyquist plane of axis c.  Returns {(i, j): real field}."""
    n = cfg.n_ptcl
    ks, k2 = _derivative_multipliers(n, cfg.box)
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    return {(i, j): np.fft.irfftn(ks[i] * ks[j] * inv * delta_k, s=(n, n, n), axes=(0, 1, 2))
            for i, j in _PAIRS}


def lpt2_source(hess, hess_b=None):
    """The 2LPT source S = sum_{i<j} (phi_ii phi_jj - phi_ij phi_ji) (Eq. 4, second line).
    With ``hess_b`` returns the symmetric bilinear form whose diagonal is S:
    1/2 sum_{i<j} (phi_ii phi'_jj + phi'_ii phi_jj - 2 phi_ij phi'_ij)."""
    hb = hess if hess_b is None else hess_b
    out = 0.0
    for i, j in ((0, 1), (0, 2), (1, 2)):
        out = out + 0.5 * (hess[i, i] * hb[j, j] + hb[i, i] * hess[j, j]) - hess[i, j] * hb[i, j]
    return out


def lpt2_displacement_from_source(src, cfg):
    """s2 = -grad phi^(2) with laplacian phi^(2) = S (Eqs. 3-4):
    s2_c = IDFT[i k_c / k^2 DFT[S]], (3, N)."""
    n = cfg.n_ptcl
    ks, k2 = _derivative_multipliers(n, cfg.box)
    sk = np.fft.rfftn(src)
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    return np.stack([np.fft.irfftn(1j * ks[c] * inv * sk, s=(n, n, n), axes=(0, 1, 2)).ravel()
                     for c in range(3)])


def lpt2_unit_displacement(omega, theta, cfg, dlnp=None):
    """Second-order displacement s2 on the lattice for unit growth (Sec. 2.1, Eqs. 2-4).
    With ``dlnp`` returns d s2 / d theta_j through P_lin: s2 is quadratic in delta1, so
    the derivative is twice the bilinear source of (delta1, d delta1 / d theta_j)."""
    dk = linear_delta_k(omega, theta, cfg)
    hess = lpt2_hessian(dk, cfg)
    if dlnp is None:
        src = lpt2_source(hess)
    else:
        src = 2.0 * lpt2_source(hess, lpt2_hessian(linear_delta_k(omega, theta, cfg, dlnp=dlnp), cfg))
    return lpt2_displacement_from_source(src, cfg)


def lpt2_transpose(sbar2, omega, theta, cfg):
    """Vector-Jacobian product of omega -> s2 at ``omega`` with sbar2 (3, N):

      S_bar      = sum_c IDFT[conj(i k_c / k^2) DFT[sbar2_c]]   (transpose of the s2 map)
      phi_bar_ii = S_bar sum_{j != i} phi_jj,  phi_bar_ij = -2 phi_ij S_bar (i < j)
      omega_bar  = sum_ij IDFT[amp k_i k_j / k^2 DFT[phi_bar_ij]]  (real even multipliers)
    with amp = sqrt(P/l_p^3).  Pinned by central differences, exact for the quadratic map."""
    n, box = cfg.n_ptcl, cfg.box
    lp = box / n
    ks, k2 = _derivative_multipliers(n, box)
    inv = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    hess = lpt2_hessian(linear_delta_k(omega, theta, cfg), cfg)
    sk = 0.0
    for c in range(3):
        sk = sk + np.conj(1j * ks[c] * inv) * np.fft.rfftn(sbar2[c].reshape(n, n, n))
    sbar = np.fft.irfftn(sk, s=(n, n, n), axes=(0, 1, 2))
    bars = {}
    for i in range(3):
        bars[i, i] = sbar * sum(hess[j, j] for j in range(3) if j != i)
    for i, j in ((0, 1), (0, 2), (1, 2)):
        bars[i, j] = -2.0 * hess[i, j] * sbar
    k_safe = np.where(k2 > 0, np.sqrt(k2), 1.0)
    amp = np.where(k2 > 0, np.sqrt(cosmo.plin(k_safe, theta) / lp ** 3), 0.0)
    acc = 0.0
    for i, j in _PAIRS:
        acc = acc + amp * ks[i] * ks[j] * inv * np.fft.rfftn(bars[i, j])
    return np.fft.irfftn(acc, s=(n, n, n), axes=(0, 1, 2)).ravel()


def lpt_initial_state(omega, theta, cfg):
    """Initial state at a0 of order ``cfg.lpt_order`` (Sec. 2.1, Eq. 2):
    s0 = D1 s1 + D2 s2, p0 = a^2 H (D1' s1 + D2' s2) = G_D s1 + G_D2 s2; the s2 terms are
    absent at first order (Zel'dovich)."""
    s0, p0, _ = za_initial_state(omega, theta, cfg)
    if cfg.lpt_order == 2:
        s2 = lpt2_unit_displacement(omega, theta, cfg)
        d2, _, gd2 = cosmo.growth_factors2(np.array([cfg.a0]), theta[2])
        s0 = s0 + d2[0] * s2
        p0 = p0 + gd2[0] * s2
    return s0, p0


# ------------------------------------------------------------------------------- CIC

def _cic_corners(x, cfg):
    """Yield (flat node index, weight, weight gradient (3, N)) for the 8 CIC corners of
    every particle (Sec. 2.2, Eq. 10, floor convention)."""
    n, l = cfg.n_mesh, cfg.cell
    u = x / l
    i = np.floor(u)
    t = u - i
    i = i.astype(np.int64)
    for d in itertools.product((0, 1), repeat=3):
        w1 = [t[c] if d[c] else 1.0 - t[c] for c in range(3)]
        dw1 = [(1.0 / l if d[c] else -1.0 / l) * np.ones_like(t[c]) for c in range(3)]
        w = w1[0] * w1[1] * w1[2]
        grad = np.stack([dw1[0] * w1[1] * w1[2], w1[0] * dw1[1] * w1[2], w1[0] * w1[1] * dw1[2]])
        idx = (((i[0] + d[0]) % n) * n + (i[1] + d[1]) % n) * n + (i[2] + d[2]) % n
        yield idx, w, grad


def cic_scatter(x, values, cfg):
    """Mesh field sum_j values_j W(x_g, x_j) (Sec. 2.2, Eq. 10)."""
    m = cfg.n_mesh ** 3
    out = np.zeros(m)
    for idx, w, _ in _cic_corners(x, cfg):
        out += np.bincount(idx, weights=values * w, minlength=m)
    return out.reshape((cfg.n_mesh,) * 3)


def cic_gather(mesh, x, cfg):
    """Particle values sum_g W(x_g, x_j) mesh(g) (Sec. 2.2, the gather with Eq. 10)."""
    flat = mesh.ravel()
    out = np.zeros(x.shape[1])
    for idx, w, _ in _cic_corners(x, cfg):
        out += w * flat[idx]
    return out


def cic_gather_grad(mesh, x, cfg):
    """sum_g grad_{x_j} W(x_g, x_j) mesh(g), shape (3, N): derivative of the gather with
    respect to the particle position (the weight-gradient term of the force VJP)."""
    flat = mesh.ravel()
    out = np.zeros((3, x.shape[1]))
    for idx, _, grad in _cic_corners(x, cfg):
        out += grad * flat[idx]
    return out


def density(x, cfg):
    """Overdensity delta = rho - 1 with rho = m sum_j W (Sec. 2.1 definition of delta)."""
    return cic_scatter(x, np.full(x.shape[1], cfg.mass), cfg) - 1.0


def density_at(x, cfg, cells):
    """The same overdensity at the flat mesh indices ``cells`` only, by direct summation
    of m W over the particles whose CIC corners include them (for meshes too large to
    deposit whole)."""
    cells = np.asarray(cells, dtype=np.int64)
    order = np.argsort(cells)
    srt = cells[order]
    mark = np.zeros(cfg.n_mesh ** 3, dtype=bool)
    mark[srt] = True
    n, l = cfg.n_mesh, cfg.cell
    u = x / l
    i = np.floor(u)
    t = u - i
    i = i.astype(np.int64)
    acc = np.zeros(len(cells))
    for d in itertools.product((0, 1), repeat=3):      # the 8 corners of Eq. 10
        idx = (((i[0] + d[0]) % n) * n + (i[1] + d[1]) % n) * n + (i[2] + d[2]) % n
        hit = mark[idx]
        w = 1.0
        for c in range(3):
            tc = t[c][hit]
            w = w * (tc if d[c] else 1.0 - tc)
        np.add.at(acc, np.searchsorted(srt, idx[hit]), cfg.mass * w)
    out = np.empty(len(cells))
    out[order] = acc - 1.0
    return out


# ----------------------------------------------------------------------------- force

def _green(cfg, Om):
    """Fourier multipliers H_c(k) = -i k_c G(k), G(k) = -3/2 Omega_m / k^2, G(0) = 0
    (Sec. 2.2, Eq. 11 and the -i k gradient), optionally divided by the CIC window
    prod_c sinc^4(k_c l / 2) (deconvolution for scatter and gather)."""
    n = cfg.n_mesh
    ks, k2 = _derivative_multipliers(n, cfg.box)
    g = np.where(k2 > 0, -1.5 * Om / np.where(k2 > 0, k2, 1.0), 0.0)
    if cfg.deconv:
        (k0, k1, k2c), _ = _kgrid(n, cfg.box)
        win = 1.0
        for kc in (k0, k1, k2c):
            win = win * np.sinc(kc * cfg.cell / (2.0 * np.pi)) ** 4
        g = g / win
    return [-1j * kc * g for kc in ks]


def force_meshes(delta, Om, cfg):
    """Force field f_c = -d_c varphi on the mesh from delta (Sec. 2.2): one forward DFT,
    the multiplier -i k_c G(k), three inverse DFTs."""
    n = cfg.n_mesh
    dk = np.fft.rfftn(delta)
    return np.stack([np.fft.irfftn(h * dk, s=(n, n, n), axes=(0, 1, 2)) for h in _green(cfg, Om)])


def pm_force(x, Om, cfg):
    """Particle accelerations a = -grad varphi(x) (Sec. 2.2; operator F of Eq. 16)."""
    f = force_meshes(density(x, cfg), Om, cfg)
    return np.stack([cic_gather(f[c], x, cfg) for c in range(3)]), f


def force_vjp(x, pi, f, Om, cfg):
    """alpha = pi . d a / d x (Sec. 3.6, Eq. 49 second line of F), written out:

    alpha_j = sum_g grad_{x_j} W(x_g, x_j) [ pi_j . f(g) + m psi(g) ],
    psi = sum_c L_c^T scatter(pi_c), L_c^T = IDFT conj(H_c) DFT (the transpose of the
    real operator delta -> f_c).  The first term is the gather-weight derivative, the
    second the dependence of the density on the positions.
    """
    n = cfg.n_mesh
    alpha = np.zeros_like(pi)
    for c in range(3):
        alpha += pi[c] * cic_gather_grad(f[c], x, cfg)
    hs = _green(cfg, Om)
    psi_k = 0.0
    for c in range(3):
        psi_k = psi_k + np.conj(hs[c]) * np.fft.rfftn(cic_scatter(x, pi[c], cfg))
    psi = np.fft.irfftn(psi_k, s=(n, n, n), axes=(0, 1, 2))
    alpha += cfg.mass * cic_gather_grad(psi, x, cfg)
    return alpha


# ------------------------------------------------------------------------- integrate

def forward(omega, theta, cfg, store_every=0, force_fn=None, snapshots=(), snapshot_a=()):
    """Zel'dovich ICs then the FastPM kick-drift-kick leapfrog (Sec. 2.3, Eq. 16).

    a_0 = F_0 first; then for i = 1..n: p += a K1_i; s += p D_i; a = F_i; p += a K2_i.
    Returns a dict with the final displacement s, momentum p, acceleration a, the
    density delta_n at a_n, and (store_every > 0) the states (s_j, p_j) at steps
    j = 0, k, 2k, ... for the checkpointed adjoint.  ``force_fn(x, s)`` replaces the PM
    force (used by the Zel'dovich-exactness pin with the linear-theory force).
    ``snapshots``: steps j whose displacement s_j, density delta_j and momentum p_j are
    returned in "snap" as {j: (s_j, delta_j, p_j)} -- observations of intermediate states
    (Sec. 2.4: the objective may depend on every z_0..z_n).  ``snapshot_a``: scale factors
    a in (a_0, a_n] whose positions are interpolated between the two enclosing steps,
    s(a) = s_j + p_{j+1/2} Dp_j(a) with the partial drift factor of
    ``cosmo.partial_drift_factor``; returned in "snap_a" as {a: (s(a), delta(a))}.
    """
    q = lattice(cfg)
    Om = theta[2]
    if force_fn is None:
        def force_fn(x, _s):
            return pm_force(x, Om, cfg)[0]
    s, p = lpt_initial_state(omega, theta, cfg)
    k1, dd, k2 = cosmo.kdk_factors(cosmo.time_grid(cfg.a0, cfg.a1, cfg.n_steps), Om)
    store = {}
    snap = {}
    if store_every:
        store[0] = (s.copy(), p.copy())
    snap_a = {}
    agrid = cosmo.time_grid(cfg.a0, cfg.a1, cfg.n_steps)
    if 0 in snapshots:
        snap[0] = (s.copy(), density(q + s, cfg), p.copy())
    a = force_fn(q + s, s)
    for i in range(1, cfg.n_steps + 1):
        p = p + a * k1[i - 1]
        for a_s in snapshot_a:
            if agrid[i - 1] < a_s <= agrid[i]:
                s_a = s + p * cosmo.partial_drift_factor(a_s, agrid, i - 1, Om)
                snap_a[a_s] = (s_a, density(q + s_a, cfg))
        s = s + p * dd[i - 1]
        a = force_fn(q + s, s)
        p = p + a * k2[i - 1]
        if store_every and i % store_every == 0:
            store[i] = (s.copy(), p.copy())
        if i in snapshots:
            snap[i] = (s.copy(), density(q + s, cfg), p.copy())
    return dict(s=s, p=p, a=a, delta=density(q + s, cfg), store=store, snap=snap, snap_a=snap_a)


def mse_loss(delta, target):
    """Objective J = mean_g (delta(g) - target(g))^2 on the final density mesh (Sec. 2.4,
    Eq. 17 as a field-level MSE) and its derivative dJ/d delta."""
    diff = delta - target
    return float(np.mean(diff * diff)), 2.0 * diff / diff.size


def _dlnp_funcs(theta):
    """d ln P_lin / d theta_j (j = 0..4) by the complex step, as callables of k."""
    def make(j):
        return lambda k: cosmo.complex_step(lambda th: np.log(cosmo.plin(k, th)), theta, j)
    return [make(j) for j in range(5)]


def _observation_cotangent(x, dj_ddelta, dj_ds, cfg):
    """dJ/dx of an observation of the positions x: the density cotangent through the CIC
    weight gradient, m sum_g grad W dJ/d delta(g), plus the direct displacement term."""
    out = np.zeros_like(x)
    if dj_ddelta is not None:
        out += cfg.mass * cic_gather_grad(np.asarray(dj_ddelta).reshape((cfg.n_mesh,) * 3), x, cfg)
    if dj_ds is not None:
        out += dj_ds
    return out


def adjoint(omega, theta, cfg, fwd, dj_ddelta=None, dj_ds=None, dj_dp=None, ckpt=None, obs=None, obs_a=None):
    """Discrete adjoint with reverse time integration (Sec. 3.6, Eqs. 49-51).

    Starts from the final state in ``fwd`` and integrates the leapfrog backward jointly
    with (xi, pi).  Initial conditions (Eq. 50): xi_n = dJ/dx_n, pi_n = dJ/dp_n, and
    a_n, alpha_n, zeta_n from F_n.  For i = n..1:
      K_i^{i-1/2}:  p -= a K2_i;  xi += alpha K2_i;  g += (pi.a) dK2_i + zeta K2_i
      D_i^{i-1}:    g += (xi.p) dD_i;  s -= p D_i;  pi += xi D_i
      F_{i-1}:      a, alpha = pi . da/dx, zeta = pi . da/dtheta = (pi.a)/Omega_m e_Om
      K_{i-1/2}^{i-1}: p -= a K1_i;  xi += alpha K1_i;  g += (pi.a) dK1_i + zeta K1_i
    (D(t_c,t_b,t_a) = -D(t_c,t_a,t_b) turns the printed signs into these.)  Finally
    (Eq. 51) dJ/domega = (D1 xi_0 + G_D pi_0) . ds1/domega and the theta terms of the
    initial conditions; with 2LPT also (D2 xi_0 + G_D2 pi_0) . ds2/domega and the s2 terms.
    ``obs`` maps steps j to cotangents (dJ/d delta_j or None, dJ/ds_j or None[, dJ/dp_j])
    of observed intermediate states; the position terms are added to xi when the reverse
    pass holds x_j (after the last reverse kick that ends at step j, before the reverse
    drift of step j); dJ/dp_j is added to pi there, and the force VJP that the next reverse
    kick (K2_j, the one that made p_j) uses is extended by its share, alpha(pi + v) =
    alpha(pi) + alpha(v).  ``obs_a`` maps interpolated scale factors a (see ``forward``) to
    (dJ/d delta(a) or None, dJ/ds(a) or None): with u their position cotangent at x(a),
    xi_j += u and pi_{j+1/2} += Dp_j(a) u right after the reverse drift of step j + 1 (before
    the force VJP at x_j), and the theta term (u . p_{j+1/2}) dDp_j/dOmega_m.  ``ckpt`` maps step j to a stored (s_j, p_j) that replaces the
    reverse-integrated state when step j is reached (piecewise resumption, Sec. 3.5).
    Returns dict(grad_omega (n_ptcl^3,), grad_theta (5,), s0, p0 (reverse-integrated)).
    """
    q = lattice(cfg)
    Om = theta[2]
    n = cfg.n_steps
    agrid = cosmo.time_grid(cfg.a0, cfg.a1, n)
    k1, dd, k2 = cosmo.kdk_factors(agrid, Om)
    dk1, ddd, dk2 = (cosmo.complex_step(lambda th: cosmo.kdk_factors(agrid, th[2])[j], theta, 2)
                     for j in range(3))
    ckpt = ckpt or {}
    s = fwd["s"].copy()
    p = fwd["p"].copy()
    g_om = 0.0
    x = q + s
    obs = obs or {}
    obs_a = obs_a or {}
    xi = _observation_cotangent(x, dj_ddelta, dj_ds, cfg)
    pi = np.zeros_like(s) if dj_dp is None else np.array(dj_dp, dtype=np.float64)
    if n in obs:
        xi += _observation_cotangent(x, *obs[n][:2], cfg)
        if len(obs[n]) > 2 and obs[n][2] is not None:
            pi = pi + obs[n][2]
    a, f = pm_force(x, Om, cfg)
    alpha = force_vjp(x, pi, f, Om, cfg)
    for i in range(n, 0, -1):
        pa = float(np.sum(pi * a))
        p = p - a * k2[i - 1]
        xi = xi + alpha * k2[i - 1]
        g_om += pa * dk2[i - 1] + (pa / Om) * k2[i - 1]
        g_om += float(np.sum(xi * p)) * ddd[i - 1]
        s = s - p * dd[i - 1]
        pi = pi + xi * dd[i - 1]
        if (i - 1) in ckpt:
            s = ckpt[i - 1][0].copy()
        for a_s, (djd, djs) in obs_a.items():
            if agrid[i - 1] < a_s <= agrid[i]:
                fac = cosmo.partial_drift_factor(a_s, agrid, i - 1, Om)
                dfac = cosmo.complex_step(lambda th: cosmo.partial_drift_factor(a_s, agrid, i - 1, th[2]), theta, 2)
                u = _observation_cotangent(q + s + p * fac, djd, djs, cfg)
                xi = xi + u
                pi = pi + fac * u
                g_om += float(np.sum(u * p)) * dfac
        x = q + s
        a, f = pm_force(x, Om, cfg)
        alpha = force_vjp(x, pi, f, Om, cfg)
        pa = float(np.sum(pi * a))
        p = p - a * k1[i - 1]
        xi = xi + alpha * k1[i - 1]
        g_om += pa * dk1[i - 1] + (pa / Om) * k1[i - 1]
        if (i - 1) in ckpt:
            p = ckpt[i - 1][1].copy()
        if (i - 1) in obs:
            xi = xi + _observation_cotangent(x, *obs[i - 1][:2], cfg)
            if len(obs[i - 1]) > 2 and obs[i - 1][2] is not None:
                pi = pi + obs[i - 1][2]
                alpha = alpha + force_vjp(x, obs[i - 1][2], f, Om, cfg)
    # initial conditions (Eq. 51): x0 = q + D1(a0) s1, p0 = G_D(a0) s1
    d1, _, gd, _ = cosmo.growth_factors(np.array([cfg.a0]), Om)
    dd1 = cosmo.complex_step(lambda th: cosmo.growth_factors(np.array([cfg.a0]), th[2])[0], theta, 2)[0]
    dgd = cosmo.complex_step(lambda th: cosmo.growth_factors(np.array([cfg.a0]), th[2])[2], theta, 2)[0]
    s1 = za_unit_displacement(omega, theta, cfg)
    sbar = d1[0] * xi + gd[0] * pi
    grad_theta = np.zeros(5)
    for j, dlnp in enumerate(_dlnp_funcs(theta)):
        grad_theta[j] = float(np.sum(sbar * za_unit_displacement(omega, theta, cfg, dlnp=dlnp)))
    grad_theta[2] += g_om + float(np.sum(xi * s1)) * dd1 + float(np.sum(pi * s1)) * dgd
    grad_omega = za_transpose(sbar, theta, cfg)
    if cfg.lpt_order == 2:
        # 2LPT: x0 += D2(a0) s2, p0 += G_D2(a0) s2 with s2 quadratic in delta1
        d2, _, gd2 = cosmo.growth_factors2(np.array([cfg.a0]), Om)
        dd2, dgd2 = (cosmo.complex_step(lambda th: cosmo.growth_factors2(np.array([cfg.a0]), th[2])[q], theta, 2)[0]
                     for q in (0, 2))
        s2 = lpt2_unit_displacement(omega, theta, cfg)
        sbar2 = d2[0] * xi + gd2[0] * pi
        for j, dlnp in enumerate(_dlnp_funcs(theta)):
            grad_theta[j] += float(np.sum(sbar2 * lpt2_unit_displacement(omega, theta, cfg, dlnp=dlnp)))
        grad_theta[2] += float(np.sum(xi * s2)) * dd2 + float(np.sum(pi * s2)) * dgd2
        grad_omega = grad_omega + lpt2_transpose(sbar2, omega, theta, cfg)
    return dict(grad_omega=grad_omega, grad_theta=grad_theta, s0=s, p0=p, xi0=xi, pi0=pi)


def za_transpose(sbar, theta, cfg):
    """Transpose of the linear map omega -> s1 applied to sbar (3, N):
    sum_c IDFT[ conj(i k_c sqrt(P/l_p^3) / k^2) DFT[sbar_c] ] (adjoint of Sec. 2.1's
    Eq. 6 chain).  Pinned by the dot-product test <v, s1(w)> = <ZA^T(v), w>."""
    n, box = cfg.n_ptcl, cfg.box
    lp = box / n
    ks, k2 = _derivative_multipliers(n, box)
    k_safe = np.where(k2 > 0, np.sqrt(k2), 1.0)
    amp = np.where(k2 > 0, np.sqrt(cosmo.plin(k_safe, theta) / lp ** 3), 0.0)
    acc = 0.0
    for c in range(3):
        b = 1j * ks[c] / np.where(k2 > 0, k2, 1.0) * amp
        acc = acc + np.conj(b) * np.fft.rfftn(sbar[c].reshape(n, n, n))
    return np.fft.irfftn(acc, s=(n, n, n), axes=(0, 1, 2)).ravel()


def loss_and_gradient(omega, theta, target, cfg, ckpt_every=0):
    """J(omega, theta) = MSE(delta_n, target) and (dJ/domega, dJ/dtheta) by the adjoint.
    ``ckpt_every`` > 0 resumes the reverse pass from states stored every k steps."""
    fwd = forward(omega, theta, cfg, store_every=ckpt_every)
    loss, dj = mse_loss(fwd["delta"], target)
    ckpt = fwd["store"] if ckpt_every else None
    adj = adjoint(omega, theta, cfg, fwd, dj_ddelta=dj, ckpt=ckpt)
    return loss, adj, fwd


def power_spectrum(delta, box):
    """Shell-averaged power spectrum of a real mesh field (the summary statistic of
    Sec. 2.4): P(k_b) = V / M^2 <|DFT delta(k)|^2> over modes with b <= |n| < b + 1,
    b = 0 .. n/2 - 1, averaged over the full k-space sphere (each half-spectrum mode
    off the kx = 0 and kx = n/2 planes stands for itself and its conjugate).
    Returns (mean |k| per bin in h/Mpc, P per bin, number of modes per bin)."""
    n = delta.shape[0]
    dk = np.fft.rfftn(delta)
    (k0, k1, k2), (n0, n1, n2) = _kgrid(n, box)
    nn = np.sqrt(n0 ** 2 + n1 ** 2 + n2 ** 2)
    w = np.where((n2 == 0) | (n2 == n // 2), 1.0, 2.0) * np.ones_like(nn)
    b = np.floor(nn).astype(np.int64)
    keep = b < n // 2
    nb = n // 2
    cnt = np.bincount(b[keep], weights=w[keep], minlength=nb)
    pw = np.bincount(b[keep], weights=(w * np.abs(dk) ** 2)[keep], minlength=nb)
    ks = np.bincount(b[keep], weights=(w * nn)[keep], minlength=nb)
    m = float(n) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        pk = box ** 3 / m ** 2 * pw / cnt
        kmean = 2 * np.pi / box * ks / cnt
    return kmean, pk, cnt


def power_loss(delta, box, target_pk, weights):
    """Objective on the shell-averaged power spectrum (a summary-statistic objective,
    Sec. 2.4): J = sum_b w_b (P_b - T_b)^2 with P_b from ``power_spectrum`` (bins
    b < n/2), and dJ/d delta.

    With F = DFT delta and C_b the number of full-k-space modes in shell b,
    P_b = V / (M^2 C_b) sum_{k in b} |F(k)|^2, so d P_b / d delta(x) =
    2 V / (M^2 C_b) sum_{k in b} F(k) e^{i k.x}: the unnormalised inverse DFT of F
    restricted to the shell.  Hence dJ/d delta = IDFT_unnorm[g_b(k) F(k)] with
    g_b = 2 w_b (P_b - T_b) 2 V / (M^2 C_b), and modes with |n| >= n/2 do not enter.
    Returns (J, dJ/d delta as an (n, n, n) array).  Pinned by central differences."""
    n = delta.shape[0]
    _, pk, cnt = power_spectrum(delta, box)
    diff = pk - np.asarray(target_pk, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    loss = float(np.sum(w * diff * diff))
    m = float(n) ** 3
    with np.errstate(invalid="ignore", divide="ignore"):
        g = np.where(cnt > 0, 2.0 * w * diff * 2.0 * box ** 3 / (m * m * cnt), 0.0)
    _, (n0, n1, n2) = _kgrid(n, box)
    b = np.floor(np.sqrt(n0 ** 2 + n1 ** 2 + n2 ** 2)).astype(np.int64)
    coef = np.where(b < n // 2, g[np.minimum(b, n // 2 - 1)], 0.0)
    grad = np.fft.irfftn(coef * np.fft.rfftn(delta), s=(n, n, n), axes=(0, 1, 2)) * m
    return loss, grad
