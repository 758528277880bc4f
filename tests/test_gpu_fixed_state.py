"""The exactly reversible fixed-point particle state (pm_config.fixed_state): 64-bit integer
displacements and momenta whose kicks and drifts the reverse pass undoes exactly.

Pins: reverse time integration recovers the initial fixed-point state bit for bit (meshes
below 128^3 take the unstaged transforms, 128^3 the TMA-staged passes and the fused
deposit), and the gradient matches the FP64 oracle (FP64: 1e-8; FP32: the accuracy targets
of the FP32 form, and at least as close as a stored-trajectory FP32 run).
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL


def _fixed_ctx(box, nm, npc, n, precision, **kw):
    torch = torch_cuda()
    from paper_2211_09815_gb300 import pm
    dt = torch.float32 if precision == 0 else torch.float64
    om = torch.from_numpy(inputs.white_noise(npc, 1).astype(np.float64)).to("cuda", dt)
    return pm.PMContext(box, nm, npc, n, [THETA], om, precision=precision, fixed_state=True, **kw)


@pytest.mark.parametrize("precision,box,nm,npc,n", [(0, 32.0, 32, 16, 6), (0, 64.0, 64, 32, 10), (1, 64.0, 64, 32, 10),
                                                    (0, 200.0, 128, 64, 12)])
def test_reverse_pass_recovers_the_initial_state_bitwise(precision, box, nm, npc, n):
    torch = torch_cuda()
    ctx = _fixed_ctx(box, nm, npc, n, precision)
    N, M = npc ** 3, nm ** 3
    u0 = torch.empty(3 * N, device="cuda", dtype=torch.int64)
    w0 = torch.empty_like(u0)
    ctx.op_ic()
    ctx.get_fixed_state(u0, w0)
    dens = torch.empty(M, device="cuda", dtype=ctx.dtype)
    uf = torch.empty_like(u0)
    ctx.forward(dens=dens)
    ctx.get_fixed_state(uf)
    tgt = torch.zeros(M, device="cuda", dtype=ctx.dtype)
    djdd = torch.empty_like(dens)
    ctx.loss_mse(tgt, djdd)
    gw = torch.empty(N, device="cuda", dtype=ctx.dtype)
    ctx.adjoint(djdd=djdd, grad_omega=gw)
    u1, w1 = torch.empty_like(u0), torch.empty_like(u0)
    ctx.get_fixed_state(u1, w1)
    ctx.close()
    assert not torch.equal(uf, u0)                   # the particles did move
    assert torch.equal(u1, u0) and torch.equal(w1, w0)


@pytest.mark.parametrize("precision", [1, 0])
def test_fixed_state_gradient_matches_oracle(precision):
    torch = torch_cuda()
    box, nm, npc, n = 32.0, 32, 16, 6
    cfg = oracle_cfg(box, nm, npc, n)
    om = inputs.white_noise(npc, 1).astype(np.float64)
    target = opm.forward(inputs.white_noise(npc, 2).astype(np.float64), THETA, cfg)["delta"]
    loss_ref, adj, _ = opm.loss_and_gradient(om, THETA, target, cfg)

    def grad(**kw):
        ctx = _fixed_ctx(box, nm, npc, n, precision) if kw.pop("fixed") else \
            make_ctx(box, nm, npc, n, precision=precision, **kw)[0]
        dt = ctx.dtype
        ctx.forward()
        djdd = torch.empty(nm ** 3, device="cuda", dtype=dt)
        loss = ctx.loss_mse(torch.from_numpy(target.ravel()).to("cuda", dt), djdd)
        gw = torch.empty(npc ** 3, device="cuda", dtype=dt)
        gt = torch.zeros(5, dtype=torch.float64)
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        ctx.close()
        return float(loss[0]), gw.cpu().numpy().astype(np.float64), gt.numpy()

    loss, g, gt = grad(fixed=True)
    if precision:
        assert abs(loss / loss_ref - 1) < 1e-10
        assert rel_l2(g, adj["grad_omega"]) < 1e-8
        assert np.allclose(gt, adj["grad_theta"], rtol=1e-8, atol=0)
    else:
        assert abs(loss / loss_ref - 1) < 1e-4
        assert cosine(g, adj["grad_omega"]) >= 0.999
        assert rel_l2(g, adj["grad_omega"]) <= 1e-3
        assert np.all(np.abs(gt / adj["grad_theta"] - 1) < 1e-3)
        # the stored trajectory (checkpoints every step) of the floating-point FP32 state
        _, g_st, _ = grad(fixed=False, ckpt_every=1)
        assert rel_l2(g, adj["grad_omega"]) <= 2.0 * rel_l2(g_st, adj["grad_omega"]) + 1e-6
