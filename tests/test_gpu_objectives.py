"""Objectives other than the field MSE (Sec. 2.4: observables compared at the level of
the fields or of summary statistics), through the C ABI against the FP64 oracle:

* the shell power spectrum objective J = sum_b w_b (P_b - T_b)^2 (pm_loss_power) as an
  operator on a given density and through the whole adjoint;
* objectives on the final particle state: cotangents dJ/dx_n, dJ/dp_n passed to pm_adjoint.
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL


def _za_density(box, nm, npc, growth):
    cfg = oracle_cfg(box, nm, npc, 1)
    s1 = opm.za_unit_displacement(inputs.white_noise(npc, 3).astype(np.float64), THETA, cfg)
    return opm.density(opm.lattice(cfg) + growth * s1, cfg)


@pytest.mark.parametrize("precision", [1, 0])
def test_power_loss_operator_matches_oracle(precision):
    torch = torch_cuda()
    box, nm, npc = 100.0, 64, 32
    delta = _za_density(box, nm, npc, 0.5)
    _, pk, _ = opm.power_spectrum(delta, box)
    rng = np.random.default_rng(31)
    target = pk * rng.uniform(0.7, 1.3, size=pk.shape)
    w = 1.0 / target ** 2
    w[0] = 0.0        # bin 0 is the k = 0 mode alone, whose power is rounding noise (mean delta = 0)
    loss_o, grad_o = opm.power_loss(delta, box, target, w)
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=precision)
    d = torch.from_numpy(delta.ravel()).to("cuda", ctx.dtype)
    djdd = torch.empty_like(d)
    loss = ctx.loss_power(target[None], w[None], djdd, dens=d)
    ctx.close()
    tol = 1e-11 if precision else 2e-5
    assert abs(loss[0] / loss_o - 1) < tol
    assert rel_l2(djdd.cpu().numpy(), grad_o.ravel()) < tol


@pytest.mark.parametrize("precision", [1, 0])
def test_power_objective_gradient_matches_oracle(precision):
    """J on P(k) of the final density, back-propagated through the reverse-time adjoint."""
    torch = torch_cuda()
    c = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)
    cfg = oracle_cfg(**c)
    om = inputs.white_noise(c["n_ptcl"], 1).astype(np.float64)
    tgt_delta = opm.forward(inputs.white_noise(c["n_ptcl"], 2).astype(np.float64), THETA, cfg)["delta"]
    _, target, _ = opm.power_spectrum(tgt_delta, c["box"])
    w = 1.0 / target ** 2
    w[0] = 0.0        # the k = 0 mode carries no power
    fwd = opm.forward(om, THETA, cfg)
    loss_o, djdd_o = opm.power_loss(fwd["delta"], c["box"], target, w)
    adj = opm.adjoint(om, THETA, cfg, fwd, dj_ddelta=djdd_o.ravel())

    ctx, *_ = make_ctx(c["box"], c["n_mesh"], c["n_ptcl"], c["n_steps"], precision=precision)
    M, N = c["n_mesh"] ** 3, c["n_ptcl"] ** 3
    ctx.forward(dens=torch.empty(M, device="cuda", dtype=ctx.dtype))
    djdd = torch.empty(M, device="cuda", dtype=ctx.dtype)
    loss = ctx.loss_power(target[None], w[None], djdd)
    gw = torch.empty(N, device="cuda", dtype=ctx.dtype)
    gt = torch.zeros(5, dtype=torch.float64)
    ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
    ctx.close()
    g = gw.cpu().numpy()
    if precision:
        assert abs(loss[0] / loss_o - 1) < 1e-9
        assert rel_l2(g, adj["grad_omega"]) < 1e-8
        assert np.allclose(gt.numpy(), adj["grad_theta"], rtol=1e-8, atol=0)
    else:
        assert abs(loss[0] / loss_o - 1) < 1e-3
        assert cosine(g, adj["grad_omega"]) >= 0.999
        assert np.all(np.abs(gt.numpy() / adj["grad_theta"] - 1) < 1e-2)


@pytest.mark.parametrize("precision", [1, 0])
def test_particle_state_objective_gradient_matches_oracle(precision):
    """J = <u, x_n> + <v, p_n> with seeded u, v: the cotangents dJ/dx_n = u and dJ/dp_n = v
    enter the adjoint initial conditions (Eq. 50) directly."""
    torch = torch_cuda()
    c = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)
    cfg = oracle_cfg(**c)
    N = c["n_ptcl"] ** 3
    rng = np.random.default_rng(41)
    u = rng.normal(size=(3, N))
    v = rng.normal(size=(3, N))
    om = inputs.white_noise(c["n_ptcl"], 1).astype(np.float64)
    adj = opm.adjoint(om, THETA, cfg, opm.forward(om, THETA, cfg), dj_ds=u, dj_dp=v)

    ctx, *_ = make_ctx(c["box"], c["n_mesh"], c["n_ptcl"], c["n_steps"], precision=precision)
    ctx.forward()
    gw = torch.empty(N, device="cuda", dtype=ctx.dtype)
    gt = torch.zeros(5, dtype=torch.float64)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel())).to("cuda", ctx.dtype)
    ctx.adjoint(djdx=to(u), djdp=to(v), grad_omega=gw, grad_theta=gt)
    ctx.close()
    g = gw.cpu().numpy()
    if precision:
        assert rel_l2(g, adj["grad_omega"]) < 1e-8
        assert np.allclose(gt.numpy(), adj["grad_theta"], rtol=1e-8, atol=0)
    else:
        assert cosine(g, adj["grad_omega"]) >= 0.999
        assert rel_l2(g, adj["grad_omega"]) <= 1e-2


SNAP = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)
SNAP_STEPS = (0, 2, 5, 6)


def _snapshot_cotangents():
    """Seeded cotangents of the observed densities and displacements (the same on both
    sides; none derived from either path's outputs)."""
    rng = np.random.default_rng(51)
    N, M = SNAP["n_ptcl"] ** 3, SNAP["n_mesh"] ** 3
    ddens = rng.normal(size=(len(SNAP_STEPS), M)) / M
    ddisp = rng.normal(size=(len(SNAP_STEPS), 3, N)) * 1e-3
    return ddens, ddisp


@pytest.mark.parametrize("precision,ckpt", [(1, 0), (1, 2), (0, 0)])
def test_snapshot_observations_match_oracle(precision, ckpt):
    """pm_set_snapshots: the forward writes s_j and delta_j at the observed steps, and the
    adjoint adds their cotangents when the reverse pass reaches each step (reverse time
    integration, or resumption from checkpoints every 2 steps)."""
    torch = torch_cuda()
    cfg = oracle_cfg(**SNAP)
    om = inputs.white_noise(SNAP["n_ptcl"], 1).astype(np.float64)
    fwd = opm.forward(om, THETA, cfg, store_every=ckpt, snapshots=SNAP_STEPS)
    ddens, ddisp = _snapshot_cotangents()
    obs = {j: (ddens[q], ddisp[q]) for q, j in enumerate(SNAP_STEPS)}
    adj = opm.adjoint(om, THETA, cfg, fwd, obs=obs, ckpt=fwd["store"] if ckpt else None)

    ctx, *_ = make_ctx(SNAP["box"], SNAP["n_mesh"], SNAP["n_ptcl"], SNAP["n_steps"], precision=precision,
                       ckpt_every=ckpt)
    N, M, ns = SNAP["n_ptcl"] ** 3, SNAP["n_mesh"] ** 3, len(SNAP_STEPS)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel())).to("cuda", ctx.dtype)
    disp = torch.empty(ns * 3 * N, device="cuda", dtype=ctx.dtype)
    dens = torch.empty(ns * M, device="cuda", dtype=ctx.dtype)
    gd, gx = to(ddens), to(ddisp)
    ctx.set_snapshots(SNAP_STEPS, disp=disp, dens=dens, ddisp=gx, ddens=gd)
    ctx.forward()
    gw = torch.empty(N, device="cuda", dtype=ctx.dtype)
    gt = torch.zeros(5, dtype=torch.float64)
    ctx.adjoint(grad_omega=gw, grad_theta=gt)
    ctx.set_snapshots([])
    ctx.close()
    disp = disp.cpu().numpy().reshape(ns, 3, N)
    dens = dens.cpu().numpy().reshape(ns, M)
    g = gw.cpu().numpy()
    if precision:
        for q, j in enumerate(SNAP_STEPS):
            assert rel_l2(disp[q], fwd["snap"][j][0]) < 1e-9
            assert np.max(np.abs(dens[q] - fwd["snap"][j][1].ravel())) < 1e-8
        assert rel_l2(g, adj["grad_omega"]) < 1e-8
        assert np.allclose(gt.numpy(), adj["grad_theta"], rtol=1e-8, atol=0)
    else:
        cell = SNAP["box"] / SNAP["n_mesh"]
        for q, j in enumerate(SNAP_STEPS):
            assert np.sqrt(np.mean((disp[q] - fwd["snap"][j][0]) ** 2)) < 1e-3 * cell
        assert cosine(g, adj["grad_omega"]) >= 0.999
        assert rel_l2(g, adj["grad_omega"]) <= 1e-2


def test_set_snapshots_rejects_bad_step_lists():
    torch_cuda()
    from paper_2211_09815_gb300 import pm
    ctx, *_ = make_ctx(50.0, 32, 16, 4)
    for bad in ([3, 2], [1, 1], [-1], [5], list(range(65))):
        with pytest.raises(pm.PMError):
            ctx.set_snapshots(bad)
    ctx.set_snapshots([0, 4])
    ctx.set_snapshots([])
    ctx.close()


@pytest.mark.parametrize("precision,ckpt", [(1, 0), (1, 2), (0, 0)])
def test_momentum_and_interpolated_observations_match_oracle(precision, ckpt):
    """Momenta observed at intermediate steps (pm_set_snapshot_momenta: the force VJP of
    step j split between its two reverse kicks) and positions observed between steps
    (pm_set_interp_snapshots: the drift of the step stopped at a), together with the step
    snapshots: the forward outputs p_j, s(a), delta(a) and the whole gradient against the
    oracle's FD-pinned adjoint (obs with dJ/dp_j, obs_a)."""
    torch = torch_cuda()
    cfg = oracle_cfg(**SNAP)
    om = inputs.white_noise(SNAP["n_ptcl"], 1).astype(np.float64)
    agrid = np.linspace(cfg.a0, cfg.a1, SNAP["n_steps"] + 1)
    a_obs = [0.5 * (agrid[1] + agrid[2]), agrid[3] + 0.2 * (agrid[4] - agrid[3]), agrid[5]]
    fwd = opm.forward(om, THETA, cfg, store_every=ckpt, snapshots=SNAP_STEPS, snapshot_a=a_obs)
    N, M, ns, na = SNAP["n_ptcl"] ** 3, SNAP["n_mesh"] ** 3, len(SNAP_STEPS), len(a_obs)
    rng = np.random.default_rng(41)
    ddens, ddisp = _snapshot_cotangents()
    dmom = rng.normal(size=(ns, 3, N)) * 1e-3
    adens = rng.normal(size=(na, M)) / M
    adisp = rng.normal(size=(na, 3, N)) * 1e-3
    obs = {j: (ddens[q], ddisp[q], dmom[q]) for q, j in enumerate(SNAP_STEPS)}
    obs_a = {a: (adens[k], adisp[k]) for k, a in enumerate(a_obs)}
    adj = opm.adjoint(om, THETA, cfg, fwd, obs=obs, obs_a=obs_a, ckpt=fwd["store"] if ckpt else None)

    ctx, *_ = make_ctx(SNAP["box"], SNAP["n_mesh"], SNAP["n_ptcl"], SNAP["n_steps"], precision=precision,
                       ckpt_every=ckpt)
    to = lambda a: torch.from_numpy(np.ascontiguousarray(a.ravel())).to("cuda", ctx.dtype)
    mom = torch.empty(ns * 3 * N, device="cuda", dtype=ctx.dtype)
    sa = torch.empty(na * 3 * N, device="cuda", dtype=ctx.dtype)
    da = torch.empty(na * M, device="cuda", dtype=ctx.dtype)
    ctx.set_snapshots(SNAP_STEPS, ddisp=to(ddisp), ddens=to(ddens))
    gm = to(dmom)
    ctx.set_snapshot_momenta(mom=mom, dmom=gm)
    ctx.set_interp_snapshots(a_obs, disp=sa, dens=da, ddisp=to(adisp), ddens=to(adens))
    ctx.forward()
    gw = torch.empty(N, device="cuda", dtype=ctx.dtype)
    gt = torch.zeros(5, dtype=torch.float64)
    ctx.adjoint(grad_omega=gw, grad_theta=gt)
    ctx.close()
    mom = mom.cpu().numpy().reshape(ns, 3, N)
    sa = sa.cpu().numpy().reshape(na, 3, N)
    da = da.cpu().numpy().reshape(na, M)
    g = gw.cpu().numpy()
    if precision:
        for q, j in enumerate(SNAP_STEPS):
            assert rel_l2(mom[q], fwd["snap"][j][2]) < 1e-9
        for k, a in enumerate(a_obs):
            assert rel_l2(sa[k], fwd["snap_a"][a][0]) < 1e-9
            assert np.max(np.abs(da[k] - fwd["snap_a"][a][1].ravel())) < 1e-8
        assert rel_l2(g, adj["grad_omega"]) < 1e-8
        assert np.allclose(gt.numpy(), adj["grad_theta"], rtol=1e-8, atol=0)
    else:
        cell = SNAP["box"] / SNAP["n_mesh"]
        for k, a in enumerate(a_obs):
            assert np.sqrt(np.mean((sa[k] - fwd["snap_a"][a][0]) ** 2)) < 1e-3 * cell
        assert cosine(g, adj["grad_omega"]) >= 0.999
        assert rel_l2(g, adj["grad_omega"]) <= 1e-2


def test_observation_setters_reject_bad_arguments():
    torch_cuda()
    from paper_2211_09815_gb300 import pm
    ctx, *_ = make_ctx(50.0, 32, 16, 4)
    with pytest.raises(pm.PMError):      # no snapshots set
        pm._check(pm.load_library().pm_set_snapshot_momenta(ctx._h, None, None), "x")
    for bad in ([1 / 64], [0.5, 0.4], [0.3, 0.3], [1.5]):
        with pytest.raises(pm.PMError):
            ctx.set_interp_snapshots(bad)
    ctx.set_interp_snapshots([0.5, 1.0])
    ctx.set_interp_snapshots([])
    ctx.close()
