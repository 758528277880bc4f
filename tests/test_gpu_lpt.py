"""GPU parity of the 2LPT initial conditions (Sec. 2.1, Eqs. 2-4; App. A) and of the
gradient through them, against the FP64 oracle, through the C ABI (pm_op_ic, pm_forward,
pm_loss_mse, pm_adjoint with lpt_order = 2).

Tolerances: FP64 to rounding (1e-11 for the initial state, 1e-8 for gradients after the
dynamics); FP32 to the accuracy targets of the method's FP32 form.  The second-order part
is also checked on its own (the 2LPT state minus the Zel'dovich state), since at a0 =
1/64 it is a small correction to s0.
"""
import numpy as np
import pytest

from oracle import cosmo
from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL
THETA_B = (2.3e-9, 0.95, 0.28, 0.049, 0.68)


def _gpu_ic(box, nm, npc, precision, lpt_order, batch=1, theta=THETA):
    torch = torch_cuda()
    ctx, *_ = make_ctx(box, nm, npc, 2, precision=precision, batch=batch, theta=theta, lpt_order=lpt_order)
    s0 = torch.empty(batch * 3 * npc ** 3, device="cuda", dtype=ctx.dtype)
    p0 = torch.empty_like(s0)
    ctx.op_ic(s0, p0)
    out = s0.cpu().numpy().reshape(batch, 3, -1), p0.cpu().numpy().reshape(batch, 3, -1)
    ctx.close()
    return out


# (box, n_mesh, n_ptcl): two mesh cells per particle; one cell per particle at a size
# whose lattice transforms take the TMA-staged column passes
IC_CASES = [(64.0, 32, 16), (200.0, 128, 64), (128.0, 128, 128)]


@pytest.mark.parametrize("box,nm,npc", IC_CASES)
@pytest.mark.parametrize("precision", [1, 0])
def test_lpt2_initial_state_matches_oracle(box, nm, npc, precision):
    cfg2 = oracle_cfg(box, nm, npc, 2, lpt_order=2)
    om = inputs.white_noise(npc, 1).astype(np.float64)
    s_o, p_o = opm.lpt_initial_state(om, THETA, cfg2)
    s_g, p_g = _gpu_ic(box, nm, npc, precision, 2)
    tol = 1e-11 if precision else 2e-6
    assert rel_l2(s_g[0], s_o) < tol and rel_l2(p_g[0], p_o) < tol
    # the second-order part alone: (2LPT state) - (Zel'dovich state) = D2 s2, G_D2 s2
    s_1, p_1 = _gpu_ic(box, nm, npc, precision, 1)
    d2, _, gd2 = cosmo.growth_factors2(np.array([cfg2.a0]), THETA[2])
    s2 = opm.lpt2_unit_displacement(om, THETA, cfg2)
    tol2 = 1e-9 if precision else 2e-3
    assert rel_l2(s_g[0].astype(np.float64) - s_1[0], d2[0] * s2) < tol2
    assert rel_l2(p_g[0].astype(np.float64) - p_1[0], gd2[0] * s2) < tol2


def test_lpt2_initial_state_batched_cosmologies():
    box, nm, npc = 64.0, 32, 16
    th = np.array([THETA, THETA_B])
    s_g, p_g = _gpu_ic(box, nm, npc, 1, 2, batch=2, theta=th)
    cfg2 = oracle_cfg(box, nm, npc, 2, lpt_order=2)
    for b in range(2):
        s_o, p_o = opm.lpt_initial_state(inputs.white_noise(npc, 1 + b).astype(np.float64), th[b], cfg2)
        assert rel_l2(s_g[b], s_o) < 1e-11 and rel_l2(p_g[b], p_o) < 1e-11


# small, nonlinear gradient case; a0 = 0.1 makes the s2 path about 6% of dJ/domega
G2 = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)


def _gpu_grad(cfg, precision, a0, target, batch=1, theta=THETA):
    torch = torch_cuda()
    ctx, *_ = make_ctx(cfg["box"], cfg["n_mesh"], cfg["n_ptcl"], cfg["n_steps"], precision=precision, a0=a0,
                       lpt_order=2, batch=batch, theta=theta)
    N, M = cfg["n_ptcl"] ** 3, cfg["n_mesh"] ** 3
    dens = torch.empty(batch * M, device="cuda", dtype=ctx.dtype)
    ctx.forward(dens=dens)
    tgt = torch.from_numpy(np.ascontiguousarray(target)).to("cuda", ctx.dtype)
    djdd = torch.empty(batch * M, device="cuda", dtype=ctx.dtype)
    loss = ctx.loss_mse(tgt, djdd)
    gw = torch.empty(batch * N, device="cuda", dtype=ctx.dtype)
    gt = torch.zeros(batch * 5, dtype=torch.float64)
    ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
    out = dict(loss=loss.numpy().copy(), grad_omega=gw.cpu().numpy().reshape(batch, N),
               grad_theta=gt.numpy().reshape(batch, 5))
    ctx.close()
    return out


def _oracle_grad(a0):
    cfg = oracle_cfg(**G2, a0=a0, lpt_order=2)
    om = inputs.white_noise(G2["n_ptcl"], 1).astype(np.float64)
    target = opm.forward(inputs.white_noise(G2["n_ptcl"], 2).astype(np.float64), THETA, cfg)["delta"]
    loss, adj, _ = opm.loss_and_gradient(om, THETA, target, cfg)
    return target, loss, adj


@pytest.mark.parametrize("a0", [1 / 64, 0.1])
def test_lpt2_adjoint_fp64_matches_oracle(a0):
    target, loss, adj = _oracle_grad(a0)
    g = _gpu_grad(G2, 1, a0, target.ravel()[None])
    assert abs(g["loss"][0] / loss - 1) < 1e-10
    assert rel_l2(g["grad_omega"][0], adj["grad_omega"]) < 1e-8
    assert np.allclose(g["grad_theta"][0], adj["grad_theta"], rtol=1e-8, atol=0)


def test_lpt2_adjoint_fp32_gradient_accuracy():
    target, loss, adj = _oracle_grad(1 / 64)
    g = _gpu_grad(G2, 0, 1 / 64, target.ravel()[None])
    assert abs(g["loss"][0] / loss - 1) < 1e-4
    assert cosine(g["grad_omega"][0], adj["grad_omega"]) >= 0.999
    assert rel_l2(g["grad_omega"][0], adj["grad_omega"]) <= 1e-3
    assert np.all(np.abs(g["grad_theta"][0] / adj["grad_theta"] - 1) < 1e-3)


def test_lpt2_batched_gradient_equals_single_runs():
    th = np.array([THETA, THETA_B])
    tgt = np.zeros((2, G2["n_mesh"] ** 3))
    both = _gpu_grad(G2, 0, 1 / 64, tgt, batch=2, theta=th)
    for b in range(2):
        torch = torch_cuda()
        ctx, *_ = make_ctx(G2["box"], G2["n_mesh"], G2["n_ptcl"], G2["n_steps"], precision=0, lpt_order=2,
                           seed=1 + b, theta=th[b])
        N, M = G2["n_ptcl"] ** 3, G2["n_mesh"] ** 3
        ctx.forward(dens=torch.empty(M, device="cuda"))
        djdd = torch.empty(M, device="cuda")
        ctx.loss_mse(torch.zeros(M, device="cuda"), djdd)
        gw = torch.empty(N, device="cuda")
        gt = torch.zeros(5, dtype=torch.float64)
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        assert np.array_equal(gw.cpu().numpy(), both["grad_omega"][b])
        assert np.array_equal(gt.numpy(), both["grad_theta"][b])
        ctx.close()
