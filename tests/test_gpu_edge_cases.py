"""Edge cases of the path against the FP64 oracle, through the C ABI: the smallest mesh and
lattice the library accepts (8^3 cells, 4^3 particles), one particle per cell, a single
step, a very short step, and zero white noise (no displacement at all: every particle at
its cell centre, a zero density contrast and zero force)."""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL


def _gradient(box, nm, npc, n, omega, target, a0=1 / 64, a1=1.0):
    torch = torch_cuda()
    ctx, *_ = make_ctx(box, nm, npc, n, precision=1, a0=a0, a1=a1, omega=omega[None])
    disp = torch.empty(3 * npc ** 3, device="cuda", dtype=torch.float64)
    ctx.forward(disp=disp)
    djdd = torch.empty(nm ** 3, device="cuda", dtype=torch.float64)
    loss = ctx.loss_mse(torch.from_numpy(target.ravel()).cuda(), djdd)
    gw = torch.empty(npc ** 3, device="cuda", dtype=torch.float64)
    gt = torch.zeros(5, dtype=torch.float64)
    ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
    ctx.close()
    return disp.cpu().numpy().reshape(3, -1), float(loss[0]), gw.cpu().numpy(), gt.numpy()


@pytest.mark.parametrize("box,nm,npc,n,a0,a1", [
    (16.0, 8, 4, 1, 1 / 64, 1.0),        # smallest mesh and lattice, one step
    (32.0, 16, 16, 3, 1 / 64, 1.0),      # one particle per cell
    (32.0, 16, 8, 2, 0.5, 0.5001),       # a very short time span
])
def test_small_and_degenerate_configurations_match_oracle(box, nm, npc, n, a0, a1):
    cfg = oracle_cfg(box, nm, npc, n, a0=a0, a1=a1)
    om = inputs.white_noise(npc, 5).astype(np.float64)
    target = opm.forward(inputs.white_noise(npc, 6).astype(np.float64), THETA, cfg)["delta"]
    loss_ref, adj, fwd = opm.loss_and_gradient(om, THETA, target, cfg)
    s, loss, g, gt = _gradient(box, nm, npc, n, om, target, a0, a1)
    assert rel_l2(s, fwd["s"]) < 1e-9
    assert abs(loss / loss_ref - 1) < 1e-10
    assert rel_l2(g, adj["grad_omega"]) < 1e-8
    assert np.allclose(gt, adj["grad_theta"], rtol=1e-8, atol=1e-12 * np.max(np.abs(adj["grad_theta"])))


def test_zero_white_noise():
    """omega = 0 with half as many particles as cells per side: every particle sits midway
    between two cell centres on each axis, so CIC spreads its mass 1/8 over 8 cells and the
    density contrast is exactly 0; the force vanishes at every step and nothing moves.  The
    loss is the target's mean square, dJ/domega is the oracle's (the ZA map is linear, so it
    does not vanish), and dJ/dtheta is 0 (every term of it carries omega or a force)."""
    box, nm, npc, n = 32.0, 16, 8, 3
    cfg = oracle_cfg(box, nm, npc, n)
    om = np.zeros(npc ** 3)
    target = opm.forward(inputs.white_noise(npc, 6).astype(np.float64), THETA, cfg)["delta"]
    loss_ref, adj, fwd = opm.loss_and_gradient(om, THETA, target, cfg)
    s, loss, g, gt = _gradient(box, nm, npc, n, om, target)
    assert np.all(s == 0.0)
    assert abs(loss - float(np.mean(target ** 2))) <= 1e-12 * loss
    assert abs(loss / loss_ref - 1) < 1e-12
    assert rel_l2(g, adj["grad_omega"]) < 1e-8
    assert np.all(adj["grad_theta"] == 0.0)
    assert np.max(np.abs(gt)) < 1e-6
