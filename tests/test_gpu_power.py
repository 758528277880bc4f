"""GPU power spectrum (pm_power_spectrum) against the oracle: the reduction itself on a
given field (FP64, 1e-12), and the FP32 simulation's final P(k) per shell against the FP64
oracle's (1e-4 relative, the accuracy target for P(k) of the FP32 form)."""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import make_ctx, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL


@pytest.mark.parametrize("precision", [1, 0])
def test_power_spectrum_reduction_matches_oracle(precision):
    torch = torch_cuda()
    nm, box = 32, 80.0
    ctx, *_ = make_ctx(box, nm, 16, 1, precision=precision)
    rng = np.random.default_rng(7)
    delta = rng.normal(size=(nm, nm, nm))
    if precision == 0:
        delta = delta.astype(np.float32).astype(np.float64)
    d = torch.from_numpy(delta.ravel()).to("cuda", ctx.dtype)
    km, pk, nmodes = ctx.power_spectrum(d)
    k_ref, p_ref, c_ref = opm.power_spectrum(delta, box)
    assert np.array_equal(nmodes, c_ref)
    ok = c_ref > 0
    tol = 1e-12 if precision else 1e-6
    assert np.max(np.abs(pk[0][ok] / p_ref[ok] - 1)) < tol
    kk = ok & (k_ref > 0)
    assert np.max(np.abs(km[kk] / k_ref[kk] - 1)) < 1e-6
    ctx.close()


def test_fp32_simulation_power_spectrum_within_1e4_of_oracle():
    torch = torch_cuda()
    box, nm, npc, n = 100.0, 64, 32, 10
    ctx, *_ = make_ctx(box, nm, npc, n, precision=0)
    ctx.forward()
    km, pk, nmodes = ctx.power_spectrum()
    ctx.close()
    cfg = opm.PMConfig(box=box, n_mesh=nm, n_ptcl=npc, n_steps=n)
    ref = opm.forward(inputs.white_noise(npc, 1).astype(np.float64), THETA, cfg)
    _, p_ref, c_ref = opm.power_spectrum(ref["delta"], box)
    ok = c_ref > 0
    ok[0] = False                       # k = 0 carries no power
    assert np.max(np.abs(pk[0][ok] / p_ref[ok] - 1)) < 1e-4
