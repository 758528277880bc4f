"""Pins for the oracle's particle-mesh forward model and adjoint (CPU only).

Each test checks the oracle against something other than itself: exact invariants of
CIC and of the antisymmetric force operator, a brute-force DFT, Newton's law, the
Zel'dovich solution, linear growth, reversibility and central finite differences.
"""
import itertools

import numpy as np
import pytest

from oracle import cosmo, pm
from paper_2211_09815_gb300 import inputs

THETA = inputs.THETA_FIDUCIAL


def _rand_positions(rng, n, box):
    return rng.uniform(0, box, size=(3, n))


# ------------------------------------------------------------------------------ CIC

def test_cic_mass_conservation_and_lattice_node():
    cfg = pm.PMConfig(box=10.0, n_mesh=8, n_ptcl=4)
    rng = np.random.default_rng(0)
    x = _rand_positions(rng, 64, cfg.box)
    rho = pm.cic_scatter(x, np.full(64, cfg.mass), cfg)
    assert abs(rho.sum() - 64 * cfg.mass) < 1e-12 * 64 * cfg.mass
    # a particle on a node puts all its mass into that node
    xn = np.array([[3 * cfg.cell], [5 * cfg.cell], [7 * cfg.cell]])
    rho1 = pm.cic_scatter(xn, np.array([1.0]), cfg)
    assert rho1[3, 5, 7] == pytest.approx(1.0, abs=1e-15)
    assert abs(rho1.sum() - 1.0) < 1e-15
    # gather of a constant field is that constant (weights sum to 1)
    assert np.allclose(pm.cic_gather(np.full((8, 8, 8), 2.5), x, cfg), 2.5, atol=1e-14)


def test_cic_periodic_wrap():
    cfg = pm.PMConfig(box=10.0, n_mesh=8, n_ptcl=4)
    x = np.array([[cfg.box - 0.25 * cfg.cell], [0.0], [0.0]])
    rho = pm.cic_scatter(x, np.array([1.0]), cfg)
    assert rho[7, 0, 0] == pytest.approx(0.25)
    assert rho[0, 0, 0] == pytest.approx(0.75)


def test_scatter_is_transpose_of_gather():
    cfg = pm.PMConfig(box=10.0, n_mesh=8, n_ptcl=4)
    rng = np.random.default_rng(1)
    x = _rand_positions(rng, 50, cfg.box)
    v = rng.normal(size=50)
    mesh = rng.normal(size=(8, 8, 8))
    lhs = np.dot(pm.cic_gather(mesh, x, cfg), v)
    rhs = np.sum(mesh * pm.cic_scatter(x, v, cfg))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_gather_gradient_matches_finite_difference():
    cfg = pm.PMConfig(box=10.0, n_mesh=8, n_ptcl=4)
    rng = np.random.default_rng(2)
    x = _rand_positions(rng, 20, cfg.box)
    mesh = rng.normal(size=(8, 8, 8))
    g = pm.cic_gather_grad(mesh, x, cfg)
    h = 1e-7
    for c in range(3):
        xp, xm = x.copy(), x.copy()
        xp[c] += h
        xm[c] -= h
        fd = (pm.cic_gather(mesh, xp, cfg) - pm.cic_gather(mesh, xm, cfg)) / (2 * h)
        assert np.allclose(fd, g[c], rtol=1e-6, atol=1e-7)


def test_gather_gradient_at_a_cell_face_is_the_right_derivative():
    """At a cell face (u = x/l an integer) the CIC weight of Eq. 10 has a kink; the floor
    convention takes the right derivative, and the one-sided differences from the left
    and the right differ by the jump of the weight gradient (the discontinuity behind
    the FP32/FP64 gradient differences of trajectories that cross a face)."""
    cfg = pm.PMConfig(box=10.0, n_mesh=8, n_ptcl=4)
    rng = np.random.default_rng(3)
    mesh = rng.normal(size=(8, 8, 8))
    x = np.array([[3.0 * cfg.cell], [2.4 * cfg.cell], [5.7 * cfg.cell]])
    g = pm.cic_gather_grad(mesh, x, cfg)[0, 0]
    h = 1e-7
    xr, xl = x.copy(), x.copy()
    xr[0] += h
    xl[0] -= h
    right = (pm.cic_gather(mesh, xr, cfg)[0] - pm.cic_gather(mesh, x, cfg)[0]) / h
    left = (pm.cic_gather(mesh, x, cfg)[0] - pm.cic_gather(mesh, xl, cfg)[0]) / h
    assert abs(g - right) < 1e-6 * max(1.0, abs(g))
    assert abs(right - left) > 1e-2 * max(abs(right), abs(left))


# -------------------------------------------------------------------------- Fourier

def _naive_force(delta, Om, box):
    """Brute-force O(N^6) evaluation of f_c(x) = 1/N^3 sum_k H_c(k) sum_y delta(y)
    e^{-ik(y-x)} over the full k grid, H_c = -i k_c (-3/2 Om / k^2), Nyquist of axis c
    zeroed, k = 0 dropped (Sec. 2.2, Eq. 11 and the -ik gradient)."""
    n = delta.shape[0]
    idx = np.array(list(itertools.product(range(n), repeat=3)))          # (N, 3)
    freq = np.where(idx >= n // 2, idx - n, idx).astype(float)            # n in [-N/2, N/2)
    k = 2 * np.pi / box * freq
    k2 = np.sum(k * k, axis=1)
    phase = np.exp(-2j * np.pi * (freq @ idx.T) / n)                      # (k, y)
    dk = phase @ delta.ravel()
    out = []
    for c in range(3):
        kc = np.where(np.abs(freq[:, c]) == n // 2, 0.0, k[:, c])
        h = np.where(k2 > 0, -1j * kc * (-1.5 * Om) / np.where(k2 > 0, k2, 1), 0)
        out.append(np.real(np.conj(phase).T @ (h * dk)) / n ** 3)
    return np.stack(out)


def test_force_mesh_matches_naive_dft_8cubed():
    cfg = pm.PMConfig(box=50.0, n_mesh=8, n_ptcl=4)
    rng = np.random.default_rng(3)
    delta = rng.normal(size=(8, 8, 8))
    f = pm.force_meshes(delta, 0.31, cfg)
    ref = _naive_force(delta, 0.31, cfg.box)
    assert np.allclose(f.reshape(3, -1), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_force_operator_is_antisymmetric():
    """<u, L_c v> = -<L_c u, v>: the -ik_c G kernel is odd, so the net force vanishes."""
    cfg = pm.PMConfig(box=50.0, n_mesh=16, n_ptcl=8)
    rng = np.random.default_rng(4)
    u = rng.normal(size=(16, 16, 16))
    v = rng.normal(size=(16, 16, 16))
    fu = pm.force_meshes(u, 0.31, cfg)
    fv = pm.force_meshes(v, 0.31, cfg)
    for c in range(3):
        a = np.sum(u * fv[c])
        b = np.sum(fu[c] * v)
        assert abs(a + b) < 1e-12 * (abs(a) + 1e-30)


def test_zero_net_force_and_zero_self_force():
    cfg = pm.PMConfig(box=50.0, n_mesh=16, n_ptcl=8)
    rng = np.random.default_rng(5)
    x = _rand_positions(rng, 300, cfg.box)
    a, _ = pm.pm_force(x, 0.31, cfg)
    scale = np.abs(a).sum(axis=1)
    assert np.all(np.abs(a.sum(axis=1)) < 1e-12 * scale)
    a1, _ = pm.pm_force(np.array([[13.3], [7.1], [40.2]]), 0.31, cfg)
    assert np.all(np.abs(a1) < 1e-14)


@pytest.mark.parametrize("r_cells", [4.0, 6.0, 12.0])
def test_pair_force_matches_newton(r_cells):
    """Two particles at separation r, l < r << L: averaged over random positions and
    orientations, the PM acceleration equals the Newtonian 3/2 Om m l^3 / (4 pi r^2)
    (Poisson Eq. 9 for a point mass) times the periodic-box background correction
    1 - 4 pi/3 (r/L)^3, within 5%.  Single axis-aligned pairs ring (the exact -ik
    gradient keeps the mesh's high-k modes), hence the average."""
    cfg = pm.PMConfig(box=64.0, n_mesh=64, n_ptcl=2)
    l = cfg.cell
    rng = np.random.default_rng(9)
    newton = 1.5 * 0.31 * cfg.mass * l ** 3 / (4 * np.pi * (r_cells * l) ** 2)
    newton *= 1 - 4 * np.pi / 3 * (r_cells * l / cfg.box) ** 3
    ratios = []
    for _ in range(48):
        x0 = rng.uniform(0, cfg.box, 3)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        x = np.stack([x0, x0 + r_cells * l * d], axis=1)
        a, _ = pm.pm_force(x, 0.31, cfg)
        assert np.allclose(a[:, 0], -a[:, 1], rtol=1e-10, atol=1e-10 * newton)
        ratios.append(-(a[:, 1] @ d) / newton)
    assert abs(np.mean(ratios) - 1) < 0.05


# ------------------------------------------------------------------ time integration

def test_leapfrog_reproduces_zeldovich_exactly():
    """Sec. 2.3: with the linear-theory force a = 3/2 Om s, FastPM KDK reproduces ZA,
    s_i = D1(a_i) s1 and p_i = G_D(a_i) s1, for any step count (pins Eqs. 14-16)."""
    cfg = pm.PMConfig(box=64.0, n_mesh=16, n_ptcl=8, n_steps=7)
    om = inputs.white_noise(8, 11).astype(np.float64)
    Om = THETA[2]
    out = pm.forward(om, THETA, cfg, force_fn=lambda x, s: 1.5 * Om * s)
    s1 = pm.za_unit_displacement(om, THETA, cfg)
    d1, _, gd, _ = cosmo.growth_factors(np.array([cfg.a1]), Om)
    assert np.allclose(out["s"], d1[0] * s1, rtol=1e-12, atol=1e-13 * np.abs(s1).max())
    assert np.allclose(out["p"], gd[0] * s1, rtol=1e-12, atol=1e-13 * np.abs(s1).max())


def test_linear_growth_with_pm_force():
    """Small-amplitude ZA ICs under the real PM force: the lowest axis-aligned displacement
    modes grow as D1(a)/D1(a0) within 1e-3 (pins the force sign, normalisation and FFT
    scaling).

    Run with one mesh cell per particle and the CIC deconvolution on: there the PM
    response of a displaced lattice at low k is linear theory up to O((k l)^2).  With
    two cells per particle the exact -ik gradient keeps the lattice alias at the mesh
    Nyquist, which strengthens the low-k force by a constant few per cent (a property
    of the discretisation, not a pin)."""
    cfg = pm.PMConfig(box=256.0, n_mesh=32, n_ptcl=32, a0=1 / 64, a1=1.0, n_steps=10,
                      deconv=True)
    th = (THETA[0] * 1e-8,) + tuple(THETA[1:])
    om = inputs.white_noise(32, 12).astype(np.float64)
    out = pm.forward(om, th, cfg)
    s1 = pm.za_unit_displacement(om, th, cfg)
    d1 = cosmo.growth_factors(np.array([cfg.a1]), th[2])[0][0]
    n = cfg.n_ptcl
    (k0, k1, k2), _ = pm._kgrid(n, cfg.box)
    kk2 = k0 ** 2 + k1 ** 2 + k2 ** 2
    # axis-aligned modes |n| <= 2 (diagonal modes carry an O(1e-2) anisotropic alias)
    axis = ((k0 != 0).astype(int) + (k1 != 0).astype(int) + (k2 != 0).astype(int)) == 1
    low = axis & (kk2 <= (2 * np.pi / cfg.box) ** 2 * 4.01)
    for c in range(3):
        got = np.fft.rfftn(out["s"][c].reshape(n, n, n))[low]
        want = d1 * np.fft.rfftn(s1[c].reshape(n, n, n))[low]
        assert np.max(np.abs(got - want)) < 1e-3 * np.max(np.abs(want))


def test_reversibility_fp64():
    """Forward 10 steps then reverse 10 steps recovers the ICs to 1e-10 relative
    (the paper's FP64 reversibility is 7e-13 to 1.3e-10)."""
    cfg = pm.PMConfig(box=64.0, n_mesh=16, n_ptcl=8, n_steps=10)
    om = inputs.white_noise(8, 13).astype(np.float64)
    fwd = pm.forward(om, THETA, cfg)
    adj = pm.adjoint(om, THETA, cfg, fwd)
    s0, p0, _ = pm.za_initial_state(om, THETA, cfg)
    assert np.sqrt(np.mean((adj["s0"] - s0) ** 2)) < 1e-10 * np.std(s0)
    assert np.sqrt(np.mean((adj["p0"] - p0) ** 2)) < 1e-10 * np.std(p0)


# ------------------------------------------------------------------------ gradients

def test_za_map_transpose_dot_product():
    cfg = pm.PMConfig(box=64.0, n_mesh=16, n_ptcl=8)
    rng = np.random.default_rng(6)
    w = rng.normal(size=(8, 8, 8))
    v = rng.normal(size=(3, 512))
    lhs = np.sum(v * pm.za_unit_displacement(w, THETA, cfg))
    rhs = np.sum(pm.za_transpose(v, THETA, cfg) * w.ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_force_vjp_matches_finite_difference():
    cfg = pm.PMConfig(box=40.0, n_mesh=16, n_ptcl=8)
    rng = np.random.default_rng(7)
    x = _rand_positions(rng, 40, cfg.box)
    pi = rng.normal(size=(3, 40))
    dx = rng.normal(size=(3, 40))
    a, f = pm.pm_force(x, 0.31, cfg)
    alpha = pm.force_vjp(x, pi, f, 0.31, cfg)
    h = 1e-7
    ap, _ = pm.pm_force(x + h * dx, 0.31, cfg)
    am, _ = pm.pm_force(x - h * dx, 0.31, cfg)
    fd = np.sum(pi * (ap - am)) / (2 * h)
    assert abs(fd - np.sum(alpha * dx)) < 1e-6 * abs(fd)


FD_CFG = pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8, n_steps=4)


def _loss(om, th, target):
    fwd = pm.forward(om, th, FD_CFG)
    return pm.mse_loss(fwd["delta"], target)[0]


@pytest.fixture(scope="module")
def fd_case():
    om = inputs.white_noise(8, 1).astype(np.float64)
    target = pm.forward(inputs.white_noise(8, 2).astype(np.float64), THETA, FD_CFG)["delta"]
    loss, adj, _ = pm.loss_and_gradient(om, THETA, target, FD_CFG)
    return om, target, loss, adj


def test_adjoint_gradient_omega_vs_central_fd(fd_case):
    """Sec. 3.6: dJ/domega by the adjoint equals central FD along random directions."""
    om, target, _, adj = fd_case
    rng = np.random.default_rng(8)
    for _ in range(2):
        v = rng.normal(size=om.shape)
        h = 1e-6
        fd = (_loss(om + h * v, THETA, target) - _loss(om - h * v, THETA, target)) / (2 * h)
        ad = np.sum(adj["grad_omega"] * v.ravel())
        assert abs(fd - ad) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("j", range(5))
def test_adjoint_gradient_theta_vs_central_fd(fd_case, j):
    """Sec. 3.6, Eq. 51: dJ/dtheta_j by the adjoint equals central FD in theta_j."""
    om, target, _, adj = fd_case
    h = 1e-6 * abs(THETA[j])
    tp = list(THETA)
    tm = list(THETA)
    tp[j] += h
    tm[j] -= h
    fd = (_loss(om, tp, target) - _loss(om, tm, target)) / (2 * h)
    assert abs(fd - adj["grad_theta"][j]) <= 1e-6 * abs(fd) + 1e-12


def test_adjoint_with_deconvolution_vs_central_fd():
    """With the CIC deconvolution (a real, even factor on the Green's function) the force
    VJP's conj(H_c) carries the same factor: dJ/domega and dJ/dOmega_m against FD."""
    cfg = pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8, n_steps=3, deconv=True)
    om = inputs.white_noise(8, 1).astype(np.float64)
    target = pm.forward(inputs.white_noise(8, 2).astype(np.float64), THETA, cfg)["delta"]
    _, adj, _ = pm.loss_and_gradient(om, THETA, target, cfg)

    def loss(w, th):
        return pm.mse_loss(pm.forward(w, th, cfg)["delta"], target)[0]
    v = np.random.default_rng(27).normal(size=om.shape)
    h = 1e-6
    fd = (loss(om + h * v, THETA) - loss(om - h * v, THETA)) / (2 * h)
    assert abs(fd - np.sum(adj["grad_omega"] * v.ravel())) <= 1e-6 * abs(fd)
    ht = 1e-6 * THETA[2]
    tp, tm = list(THETA), list(THETA)
    tp[2] += ht
    tm[2] -= ht
    fdt = (loss(om, tp) - loss(om, tm)) / (2 * ht)
    assert abs(fdt - adj["grad_theta"][2]) <= 1e-6 * abs(fdt)


def test_reverse_time_adjoint_equals_stored_trajectory(fd_case):
    """Reverse time integration (Sec. 3.5) gives the stored-trajectory gradient to ~1e-10
    in FP64; resuming from checkpoints every step is the stored trajectory."""
    om, target, _, adj = fd_case
    _, adj_st, _ = pm.loss_and_gradient(om, THETA, target, FD_CFG, ckpt_every=1)
    g, gs = adj["grad_omega"], adj_st["grad_omega"]
    assert np.linalg.norm(g - gs) < 1e-9 * np.linalg.norm(gs)
    assert np.allclose(adj["grad_theta"], adj_st["grad_theta"], rtol=1e-9)


# ------------------------------------------------------------------- 2LPT (Sec. 2.1)

def _lpt2_of_field(delta1, cfg):
    return pm.lpt2_displacement_from_source(pm.lpt2_source(pm.lpt2_hessian(np.fft.rfftn(delta1), cfg)), cfg)


def test_lpt2_two_perpendicular_waves_closed_form():
    """delta1 = A cos(k q0) + B cos(k q1): phi_00 = A cos(k q0), phi_11 = B cos(k q1), so
    S = AB cos(k q0) cos(k q1) (Eq. 4), phi2 = -S / (2 k^2) and s2 = -grad phi2 gives
    s2_0 = -AB sin(k q0) cos(k q1) / (2k), s2_1 = -AB cos(k q0) sin(k q1) / (2k), s2_2 = 0."""
    n, box = 16, 64.0
    cfg = pm.PMConfig(box=box, n_mesh=32, n_ptcl=n)
    q = np.indices((n, n, n)).astype(np.float64) * (box / n)
    k, A, B = 2 * np.pi / box * 2, 0.7, -1.3
    s2 = _lpt2_of_field(A * np.cos(k * q[0]) + B * np.cos(k * q[1]), cfg)
    want = np.stack([-A * B * np.sin(k * q[0]) * np.cos(k * q[1]) / (2 * k),
                     -A * B * np.cos(k * q[0]) * np.sin(k * q[1]) / (2 * k), 0 * q[2]]).reshape(3, -1)
    assert np.max(np.abs(s2 - want)) < 1e-13 * np.max(np.abs(want))


def test_lpt2_diagonal_wave_uses_the_mixed_derivatives():
    """delta1 = A cos(k (q0 + q1)) + B cos(k q2): phi_00 = phi_11 = phi_01 = A/2 cos u, so
    the mixed term cancels the phi_00 phi_11 product and S = AB cos u cos v (u = k(q0+q1),
    v = k q2); with |k|^2 = 3k^2, s2 = grad S / (3k^2).  A dropped or mis-signed phi_01^2
    term fails here."""
    n, box = 16, 64.0
    cfg = pm.PMConfig(box=box, n_mesh=32, n_ptcl=n)
    q = np.indices((n, n, n)).astype(np.float64) * (box / n)
    k, A, B = 2 * np.pi / box, 0.9, 0.4
    u, v = k * (q[0] + q[1]), k * q[2]
    s2 = _lpt2_of_field(A * np.cos(u) + B * np.cos(v), cfg)
    sx = -A * B * np.sin(u) * np.cos(v) / (3 * k)
    want = np.stack([sx, sx, -A * B * np.cos(u) * np.sin(v) / (3 * k)]).reshape(3, -1)
    assert np.max(np.abs(s2 - want)) < 1e-13 * np.max(np.abs(want))


def test_lpt2_vanishes_for_one_dimensional_fields():
    """A field that varies along one axis only has phi_ij = 0 unless i = j = that axis, so
    S = 0 and 2LPT adds nothing (Zel'dovich is exact in one dimension)."""
    n = 16
    cfg = pm.PMConfig(box=50.0, n_mesh=32, n_ptcl=n)
    line = np.random.default_rng(4).normal(size=n)
    s2 = _lpt2_of_field(np.broadcast_to(line[None, :, None], (n, n, n)).copy(), cfg)
    assert np.max(np.abs(s2)) < 1e-15 * n ** 3


def test_lpt2_transpose_equals_exact_central_difference():
    """s2 is quadratic in omega, so the central difference along v is exact up to
    rounding: <sbar, (s2(w + h v) - s2(w - h v)) / 2h> = <lpt2_transpose(sbar), v>."""
    cfg = pm.PMConfig(box=64.0, n_mesh=32, n_ptcl=16)
    rng = np.random.default_rng(3)
    w = inputs.white_noise(16, 1).astype(np.float64)
    v = rng.normal(size=w.shape)
    sb = rng.normal(size=(3, 16 ** 3))
    h = 1e-3
    fd = np.sum(sb * (pm.lpt2_unit_displacement(w + h * v, THETA, cfg)
                      - pm.lpt2_unit_displacement(w - h * v, THETA, cfg))) / (2 * h)
    ad = np.sum(pm.lpt2_transpose(sb, w, THETA, cfg) * v.ravel())
    assert abs(fd - ad) < 1e-11 * abs(fd)


@pytest.mark.parametrize("j", range(5))
def test_lpt2_theta_derivative_vs_central_fd(j):
    """d s2 / d theta_j through P_lin (twice the bilinear source) against central FD."""
    cfg = pm.PMConfig(box=64.0, n_mesh=32, n_ptcl=16)
    w = inputs.white_noise(16, 5).astype(np.float64)
    an = pm.lpt2_unit_displacement(w, THETA, cfg, dlnp=pm._dlnp_funcs(THETA)[j])
    h = 1e-6 * abs(THETA[j])
    tp, tm = list(THETA), list(THETA)
    tp[j] += h
    tm[j] -= h
    fd = (pm.lpt2_unit_displacement(w, tp, cfg) - pm.lpt2_unit_displacement(w, tm, cfg)) / (2 * h)
    assert np.linalg.norm(an - fd) < 1e-8 * np.linalg.norm(fd)


def test_lpt2_density_matches_second_order_perturbation_theory():
    """Physics pin of the whole 2LPT chain (Eqs. 2-4 with the App. A growth at Omega_m = 1,
    D1 = a, D2 = 3/7 a^2): for delta1 = eps (cos k q0 + cos k q1) the particle density's
    Fourier coefficient at k1 + k2 is 2 F2(k1, k2) (eps/2)^2 + O(eps^4), with the
    Eulerian perturbation-theory kernel F2 = 5/7 for perpendicular equal modes, i.e.
    (5/14) eps^2; the Zel'dovich displacement alone gives the kernel 1/2, i.e. eps^2 / 4.
    A wrong sign of the source or of D2 gives 1/7."""
    n, box = 32, 100.0
    cfg = pm.PMConfig(box=box, n_mesh=n, n_ptcl=n)
    q = np.indices((n, n, n)).reshape(3, -1).astype(np.float64) * (box / n)
    k, eps = 2 * np.pi / box, 1e-3
    d1 = eps * (np.cos(k * q[0]) + np.cos(k * q[1])).reshape(n, n, n)
    s1 = pm.lpt2_displacement_from_source(d1, cfg)        # the same ik/k^2 map as s1 from delta1
    s2 = _lpt2_of_field(d1, cfg)
    a = np.array([1.0])
    dd1 = cosmo.growth_factors(a, 1.0)[0][0]
    dd2 = cosmo.growth_factors2(a, 1.0)[0][0]

    def coefficient(x):
        return np.mean(np.exp(-1j * (k * x[0] + k * x[1]))) / eps ** 2

    assert abs(coefficient(q + dd1 * s1) - 0.25) < 1e-5
    assert abs(coefficient(q + dd1 * s1 + dd2 * s2) - 5.0 / 14.0) < 1e-5


def _second_order_coefficient_after_pm(n_steps):
    n, box, eps = 32, 256.0, 1e-2
    cfg = pm.PMConfig(box=box, n_mesh=n, n_ptcl=n, n_steps=n_steps, deconv=True)
    q = pm.lattice(cfg)
    k = 2 * np.pi / box
    d1 = eps * (np.cos(k * q[0]) + np.cos(k * q[1])).reshape(n, n, n)
    s1 = pm.lpt2_displacement_from_source(d1, cfg)
    s2 = _lpt2_of_field(d1, cfg)
    a0 = np.array([cfg.a0])
    dd1, _, gd, _ = cosmo.growth_factors(a0, 1.0)
    dd2, _, gd2 = cosmo.growth_factors2(a0, 1.0)
    s = dd1[0] * s1 + dd2[0] * s2
    p = gd[0] * s1 + gd2[0] * s2
    k1, dd, k2 = cosmo.kdk_factors(cosmo.time_grid(cfg.a0, cfg.a1, n_steps), 1.0)
    acc = pm.pm_force(q + s, 1.0, cfg)[0]
    for i in range(n_steps):
        p = p + acc * k1[i]
        s = s + p * dd[i]
        acc = pm.pm_force(q + s, 1.0, cfg)[0]
        p = p + acc * k2[i]
    x = q + s
    first = np.mean(np.exp(-1j * k * x[0])).real / eps
    second = np.mean(np.exp(-1j * (k * x[0] + k * x[1]))).real / eps ** 2
    return first, second


def test_pm_dynamics_grow_the_second_order_density():
    """Two perpendicular waves from 2LPT initial conditions at a0 = 1/64, evolved to a = 1
    with Omega_m = 1 (D1 = a) by the PM force and the FastPM leapfrog (Sec. 2.2-2.3): the
    first-order coefficient stays D1 / 2 (1e-4) and the mode coupling builds the
    perturbation-theory second-order coefficient (5/14) D1^2 at k1 + k2, within 1.5% at
    20 steps and 0.5% at 40 (the time-integration error of the second-order mode halves
    with the step size)."""
    f20, s20 = _second_order_coefficient_after_pm(20)
    f40, s40 = _second_order_coefficient_after_pm(40)
    assert abs(f20 - 0.5) < 1e-4 and abs(f40 - 0.5) < 1e-4
    want = 5.0 / 14.0
    assert abs(s20 / want - 1) < 1.5e-2 and abs(s40 / want - 1) < 5e-3
    assert abs(s40 - want) < 0.6 * abs(s20 - want)


FD_CFG2 = pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8, n_steps=4, lpt_order=2)


def _loss2(om, th, target):
    return pm.mse_loss(pm.forward(om, th, FD_CFG2)["delta"], target)[0]


@pytest.fixture(scope="module")
def fd_case2():
    om = inputs.white_noise(8, 1).astype(np.float64)
    target = pm.forward(inputs.white_noise(8, 2).astype(np.float64), THETA, FD_CFG2)["delta"]
    loss, adj, _ = pm.loss_and_gradient(om, THETA, target, FD_CFG2)
    return om, target, loss, adj


def test_lpt2_changes_the_initial_state_by_the_second_order_term():
    om = inputs.white_noise(8, 1).astype(np.float64)
    s1, p1 = pm.lpt_initial_state(om, THETA, pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8))
    s2, p2 = pm.lpt_initial_state(om, THETA, FD_CFG2)
    d2, _, gd2 = cosmo.growth_factors2(np.array([FD_CFG2.a0]), THETA[2])
    u = pm.lpt2_unit_displacement(om, THETA, FD_CFG2)
    assert np.allclose(s2 - s1, d2[0] * u, rtol=0, atol=1e-14 * np.abs(s1).max())
    assert np.allclose(p2 - p1, gd2[0] * u, rtol=0, atol=1e-14 * np.abs(p1).max())


def test_lpt2_adjoint_gradient_omega_vs_central_fd(fd_case2):
    """dJ/domega with 2LPT initial conditions (the s2 VJP added to Eq. 51) against FD."""
    om, target, _, adj = fd_case2
    rng = np.random.default_rng(9)
    v = rng.normal(size=om.shape)
    h = 1e-6
    fd = (_loss2(om + h * v, THETA, target) - _loss2(om - h * v, THETA, target)) / (2 * h)
    assert abs(fd - np.sum(adj["grad_omega"] * v.ravel())) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("j", range(5))
def test_lpt2_adjoint_gradient_theta_vs_central_fd(fd_case2, j):
    """dJ/dtheta_j with 2LPT initial conditions (P_lin through s2, D2 and G_D2 through
    Omega_m) against central FD."""
    om, target, _, adj = fd_case2
    h = 1e-6 * abs(THETA[j])
    tp, tm = list(THETA), list(THETA)
    tp[j] += h
    tm[j] -= h
    fd = (_loss2(om, tp, target) - _loss2(om, tm, target)) / (2 * h)
    assert abs(fd - adj["grad_theta"][j]) <= 1e-6 * abs(fd) + 1e-12


def test_lpt2_reversibility_fp64():
    """Reverse integration recovers the 2LPT initial state to 1e-10 relative."""
    cfg = pm.PMConfig(box=64.0, n_mesh=16, n_ptcl=8, n_steps=10, lpt_order=2)
    om = inputs.white_noise(8, 13).astype(np.float64)
    adj = pm.adjoint(om, THETA, cfg, pm.forward(om, THETA, cfg))
    s0, p0 = pm.lpt_initial_state(om, THETA, cfg)
    assert np.sqrt(np.mean((adj["s0"] - s0) ** 2)) < 1e-10 * np.std(s0)
    assert np.sqrt(np.mean((adj["p0"] - p0) ** 2)) < 1e-10 * np.std(p0)


def test_white_noise_power_recovers_plin():
    """Eq. 5-6: <|delta1(k)|^2> l_p^6 / V = P_lin(k), averaged over seeds and shells."""
    cfg = pm.PMConfig(box=200.0, n_mesh=32, n_ptcl=16)
    n = cfg.n_ptcl
    lp = cfg.box / n
    (k0, k1, k2), _ = pm._kgrid(n, cfg.box)
    kk = np.sqrt(k0 ** 2 + k1 ** 2 + k2 ** 2)
    shell = (kk > 0.06) & (kk < 0.16)     # below the lattice Nyquist 0.25 h/Mpc
    pk = []
    for seed in range(24):
        om = inputs.white_noise(n, 100 + seed).astype(np.float64)
        s1 = pm.za_unit_displacement(om, THETA, cfg)
        # delta1 = -div s1  in Fourier: -i k . s1(k)
        dk = sum(-1j * kc * np.fft.rfftn(s1[c].reshape(n, n, n)) for c, kc in enumerate((k0, k1, k2)))
        pk.append(np.abs(dk[shell]) ** 2 * lp ** 6 / cfg.box ** 3 / cosmo.plin(kk[shell], THETA))
    ratio = np.mean(pk)
    assert abs(ratio - 1) < 0.05


def test_power_spectrum_of_a_plane_wave():
    """A single cosine mode of amplitude A at |n| = 3 along x puts V A^2 / 4 (per of the
    two +-k modes) into bin 3 and nothing elsewhere; bin 3 holds 6 * ... modes, so the
    shell average is (2 modes with power (A M / 2)^2 V / M^2) / (modes in the shell)."""
    n, box = 16, 50.0
    x = np.arange(n) * box / n
    A = 0.7
    delta = A * np.cos(2 * np.pi * 3 * x / box)[:, None, None] * np.ones((n, n, n))
    kmean, pk, cnt = pm.power_spectrum(delta, box)
    total = pk * cnt
    expect = 2 * (A * n ** 3 / 2) ** 2 * box ** 3 / n ** 6
    assert abs(total[3] / expect - 1) < 1e-12
    assert np.all(np.abs(np.delete(total, 3)) < 1e-20 * expect + 1e-25)
    # mode counts cover the half-open shells exactly
    (k0, k1, k2), (n0, n1, n2) = pm._kgrid(n, box)
    nn = np.sqrt(n0 ** 2 + n1 ** 2 + n2 ** 2)
    full = np.sum(np.floor(np.sqrt(np.add.outer(np.add.outer(np.fft.fftfreq(n, 1 / n) ** 2, np.fft.fftfreq(n, 1 / n) ** 2), np.fft.fftfreq(n, 1 / n) ** 2))) == 3)
    assert cnt[3] == full


def test_density_at_sampled_cells_equals_full_deposit():
    """The sampled-cell form used at full mesh sizes against the whole-mesh deposit."""
    cfg = pm.PMConfig(box=32.0, n_mesh=16, n_ptcl=8, n_steps=1)
    rng = np.random.default_rng(21)
    x = pm.lattice(cfg) + rng.normal(scale=3.0, size=(3, 8 ** 3))
    full = pm.density(x, cfg).ravel()
    cells = rng.choice(16 ** 3, size=200, replace=False)
    np.testing.assert_allclose(pm.density_at(x, cfg, cells), full[cells], rtol=0, atol=1e-12)


def test_power_loss_gradient_vs_central_fd():
    """J = sum_b w_b (P_b - T_b)^2 on the shell power (Sec. 2.4 summary statistic): the
    closed-form dJ/d delta against central differences along random directions, with
    weights on every bin (including bins whose modes sit on the kx = 0 and kx = n/2
    planes) and a target away from the field's own spectrum."""
    n, box = 16, 50.0
    rng = np.random.default_rng(21)
    delta = rng.normal(size=(n, n, n))
    _, pk, _ = pm.power_spectrum(delta, box)
    target = pk * rng.uniform(0.5, 1.5, size=pk.shape)
    w = rng.uniform(0.5, 2.0, size=pk.shape) / pk ** 2
    loss, grad = pm.power_loss(delta, box, target, w)
    for _ in range(3):
        v = rng.normal(size=delta.shape)
        h = 1e-5
        fd = (pm.power_loss(delta + h * v, box, target, w)[0] - pm.power_loss(delta - h * v, box, target, w)[0]) / (2 * h)
        assert abs(fd - np.sum(grad * v)) < 1e-7 * abs(fd)


def test_power_loss_single_bin_value():
    """With one bin weighted the objective is that bin's squared deviation, and the
    gradient of a field's own spectrum as target is zero."""
    n, box = 16, 50.0
    delta = np.random.default_rng(22).normal(size=(n, n, n))
    _, pk, _ = pm.power_spectrum(delta, box)
    w = np.zeros_like(pk)
    w[3] = 1.0
    loss, _ = pm.power_loss(delta, box, np.zeros_like(pk), w)
    assert loss == pytest.approx(pk[3] ** 2, rel=1e-14)
    loss0, grad0 = pm.power_loss(delta, box, pk, np.ones_like(pk))
    assert loss0 == 0.0 and np.max(np.abs(grad0)) == 0.0


SNAP_CFG = pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8, n_steps=4)


def _snapshot_loss(om, th, targets, u):
    """J = sum_j MSE(delta_j, target_j) over observed steps + <u, s_3> (intermediate
    observations of Sec. 2.4)."""
    fwd = pm.forward(om, th, SNAP_CFG, snapshots=(0, 2, 3))
    j = sum(pm.mse_loss(fwd["snap"][k][1], targets[k])[0] for k in (0, 2))
    return j + float(np.sum(u * fwd["snap"][3][0]))


@pytest.fixture(scope="module")
def snapshot_case():
    om = inputs.white_noise(8, 1).astype(np.float64)
    other = pm.forward(inputs.white_noise(8, 2).astype(np.float64), THETA, SNAP_CFG, snapshots=(0, 2))
    targets = {k: other["snap"][k][1] for k in (0, 2)}
    u = np.random.default_rng(23).normal(size=(3, 8 ** 3))
    fwd = pm.forward(om, THETA, SNAP_CFG, snapshots=(0, 2, 3))
    obs = {k: (pm.mse_loss(fwd["snap"][k][1], targets[k])[1], None) for k in (0, 2)}
    obs[3] = (None, u)
    adj = pm.adjoint(om, THETA, SNAP_CFG, fwd, obs=obs)
    return om, targets, u, adj


def test_snapshot_states_equal_shorter_runs():
    """The state observed at step j is the final state of a j-step run over the same
    time grid (a1 = a_j)."""
    om = inputs.white_noise(8, 1).astype(np.float64)
    fwd = pm.forward(om, THETA, SNAP_CFG, snapshots=(2,))
    agrid = cosmo.time_grid(SNAP_CFG.a0, SNAP_CFG.a1, SNAP_CFG.n_steps)
    short = pm.PMConfig(box=24.0, n_mesh=16, n_ptcl=8, n_steps=2, a1=float(agrid[2]))
    ref = pm.forward(om, THETA, short)
    assert np.allclose(fwd["snap"][2][0], ref["s"], rtol=0, atol=1e-12 * np.abs(ref["s"]).max())
    assert np.allclose(fwd["snap"][2][1], ref["delta"], rtol=0, atol=1e-12)


def test_snapshot_objective_gradient_omega_vs_central_fd(snapshot_case):
    """Cotangents of observed intermediate densities and displacements, injected when the
    reverse pass reaches their step, give dJ/domega of the whole objective (central FD)."""
    om, targets, u, adj = snapshot_case
    v = np.random.default_rng(24).normal(size=om.shape)
    h = 1e-6
    fd = (_snapshot_loss(om + h * v, THETA, targets, u) - _snapshot_loss(om - h * v, THETA, targets, u)) / (2 * h)
    assert abs(fd - np.sum(adj["grad_omega"] * v.ravel())) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("j", [0, 2])
def test_snapshot_objective_gradient_theta_vs_central_fd(snapshot_case, j):
    om, targets, u, adj = snapshot_case
    h = 1e-6 * abs(THETA[j])
    tp, tm = list(THETA), list(THETA)
    tp[j] += h
    tm[j] -= h
    fd = (_snapshot_loss(om, tp, targets, u) - _snapshot_loss(om, tm, targets, u)) / (2 * h)
    assert abs(fd - adj["grad_theta"][j]) <= 1e-6 * abs(fd) + 1e-12


A_OBS = (0.33, 0.8)     # between steps of SNAP_CFG's grid (1/64, 0.26, 0.51, 0.75, 1)


def _interp_loss(om, th, target, u, v):
    """J = MSE(delta(0.33), target) + <u, s(0.8)> + <v, p_2>: positions interpolated between
    steps and a momentum observed at an intermediate step."""
    fwd = pm.forward(om, th, SNAP_CFG, snapshots=(2,), snapshot_a=A_OBS)
    j = pm.mse_loss(fwd["snap_a"][A_OBS[0]][1], target)[0]
    return j + float(np.sum(u * fwd["snap_a"][A_OBS[1]][0])) + float(np.sum(v * fwd["snap"][2][2]))


@pytest.fixture(scope="module")
def interp_case():
    om = inputs.white_noise(8, 1).astype(np.float64)
    target = pm.forward(inputs.white_noise(8, 2).astype(np.float64), THETA, SNAP_CFG,
                        snapshot_a=A_OBS)["snap_a"][A_OBS[0]][1]
    rng = np.random.default_rng(25)
    u = rng.normal(size=(3, 8 ** 3))
    v = rng.normal(size=(3, 8 ** 3)) * 10.0
    fwd = pm.forward(om, THETA, SNAP_CFG, snapshots=(2,), snapshot_a=A_OBS)
    obs_a = {A_OBS[0]: (pm.mse_loss(fwd["snap_a"][A_OBS[0]][1], target)[1], None), A_OBS[1]: (None, u)}
    adj = pm.adjoint(om, THETA, SNAP_CFG, fwd, obs={2: (None, None, v)}, obs_a=obs_a)
    return om, target, u, v, adj


def test_interpolated_snapshot_at_a_step_is_that_step():
    """The interpolated position at a = a_j is the state after step j (the partial drift
    factor equals the full one there)."""
    om = inputs.white_noise(8, 1).astype(np.float64)
    agrid = cosmo.time_grid(SNAP_CFG.a0, SNAP_CFG.a1, SNAP_CFG.n_steps)
    fwd = pm.forward(om, THETA, SNAP_CFG, snapshots=(3,), snapshot_a=(float(agrid[3]),))
    assert np.allclose(fwd["snap_a"][float(agrid[3])][0], fwd["snap"][3][0], rtol=0, atol=1e-12)


def test_interpolated_and_momentum_observations_gradient_vs_central_fd(interp_case):
    om, target, u, v, adj = interp_case
    w = np.random.default_rng(26).normal(size=om.shape)
    h = 1e-6
    fd = (_interp_loss(om + h * w, THETA, target, u, v) - _interp_loss(om - h * w, THETA, target, u, v)) / (2 * h)
    assert abs(fd - np.sum(adj["grad_omega"] * w.ravel())) <= 1e-6 * abs(fd)


@pytest.mark.parametrize("j", [0, 2])
def test_interpolated_and_momentum_observations_theta_vs_central_fd(interp_case, j):
    """Omega_m enters the partial drift factors as well as the dynamics."""
    om, target, u, v, adj = interp_case
    h = 1e-6 * abs(THETA[j])
    tp, tm = list(THETA), list(THETA)
    tp[j] += h
    tm[j] -= h
    fd = (_interp_loss(om, tp, target, u, v) - _interp_loss(om, tm, target, u, v)) / (2 * h)
    assert abs(fd - adj["grad_theta"][j]) <= 1e-6 * abs(fd) + 1e-12
