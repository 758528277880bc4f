"""torch.autograd.Function over the C ABI: gradients against central finite differences
(FP64), against the FP64 oracle (FP32: cosine >= 0.999, relative L2 <= 1e-3) and against
the library's own loss path."""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, ensure_built, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL
C0 = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)


def _setup(precision):
    torch = torch_cuda()
    ensure_built()
    from paper_2211_09815_gb300 import pm
    dt = torch.float32 if precision == 0 else torch.float64
    cfg = oracle_cfg(**C0)
    target = opm.forward(inputs.white_noise(C0["n_ptcl"], 2).astype(np.float64), THETA, cfg)["delta"].ravel()
    om = torch.from_numpy(inputs.white_noise(C0["n_ptcl"], 1).astype(np.float64)).to("cuda", dt)
    ctx = pm.PMContext(C0["box"], C0["n_mesh"], C0["n_ptcl"], C0["n_steps"], [THETA], om, precision=precision)
    tgt = torch.from_numpy(target).to("cuda", dt)
    return torch, ctx, om, tgt, target


def _loss(torch, simulate, ctx, om, th, tgt):
    dens, _, _ = simulate(ctx, om, th)
    return torch.mean((dens[0] - tgt) ** 2)


def test_autograd_fp64_matches_central_finite_differences():
    from paper_2211_09815_gb300.autograd import simulate
    torch, ctx, om, tgt, _ = _setup(1)
    om = om.clone().requires_grad_(True)
    th = torch.tensor([THETA], dtype=torch.float64, requires_grad=True)
    loss = _loss(torch, simulate, ctx, om, th, tgt)
    loss.backward()
    g_om, g_th = om.grad.clone(), th.grad.clone()
    rng = np.random.default_rng(5)
    v = torch.from_numpy(rng.normal(size=om.shape)).to("cuda", torch.float64)
    h = 1e-6
    with torch.no_grad():
        lp = _loss(torch, simulate, ctx, om + h * v, th, tgt).item()
        lm = _loss(torch, simulate, ctx, om - h * v, th, tgt).item()
    fd = (lp - lm) / (2 * h)
    ad = float((g_om * v).sum())
    assert abs(fd - ad) <= 1e-6 * abs(fd)
    for j in (0, 2):
        hj = 1e-6 * abs(THETA[j])
        tp, tm = th.detach().clone(), th.detach().clone()
        tp[0, j] += hj
        tm[0, j] -= hj
        with torch.no_grad():
            fdj = (_loss(torch, simulate, ctx, om, tp, tgt).item() - _loss(torch, simulate, ctx, om, tm, tgt).item()) / (2 * hj)
        assert abs(fdj - float(g_th[0, j])) <= 1e-6 * abs(fdj)
    ctx.close()


def test_autograd_fp32_matches_oracle_and_library_loss_path():
    from paper_2211_09815_gb300.autograd import simulate
    torch, ctx, om, tgt, target = _setup(0)
    om = om.clone().requires_grad_(True)
    th = torch.tensor([THETA], dtype=torch.float64, requires_grad=True)
    loss = _loss(torch, simulate, ctx, om, th, tgt)
    loss.backward()
    cfg = oracle_cfg(**C0)
    _, adj, _ = opm.loss_and_gradient(inputs.white_noise(C0["n_ptcl"], 1).astype(np.float64), THETA,
                                      target.reshape((C0["n_mesh"],) * 3), cfg)
    g = om.grad.detach().cpu().numpy().ravel()
    assert cosine(g, adj["grad_omega"]) >= 0.999
    assert rel_l2(g, adj["grad_omega"]) <= 1e-3
    assert np.all(np.abs(th.grad.numpy()[0] / adj["grad_theta"] - 1) < 1e-3)
    # the library's own MSE + adjoint path gives the same gradient
    ctx.set_inputs(theta=[THETA], omega=om.detach())
    ctx.forward()
    djdd = torch.empty_like(tgt)
    ctx.loss_mse(tgt, djdd)
    gw = torch.empty_like(om.detach().reshape(-1))
    ctx.adjoint(djdd=djdd, grad_omega=gw)
    assert rel_l2(gw.cpu().numpy(), g) < 1e-5
    ctx.close()


def test_backward_after_the_context_state_was_replaced_raises():
    """Two simulate() calls on one context, then backward through the first: the context
    now holds the second call's final state, so the backward refuses instead of returning
    the gradient at the second call's inputs; the second graph's backward still works."""
    from paper_2211_09815_gb300.autograd import simulate
    torch, ctx, om, tgt, _ = _setup(1)
    om1 = om.clone().requires_grad_(True)
    om2 = (om * 1.01).requires_grad_(True)
    th = torch.tensor([THETA], dtype=torch.float64, requires_grad=True)
    loss1 = _loss(torch, simulate, ctx, om1, th, tgt)
    loss2 = _loss(torch, simulate, ctx, om2, th, tgt)
    with pytest.raises(RuntimeError, match="forward state was replaced"):
        loss1.backward()
    loss2.backward()
    assert om2.grad is not None and bool(torch.isfinite(om2.grad).all())
    ctx.close()
