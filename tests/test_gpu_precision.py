"""FP32 against FP64 on the GPU where the oracle is too slow: 128^3 particles, 256^3 mesh,
200 Mpc/h, 63 steps (the FP64 GPU path is pinned to the oracle at the small sizes of
test_gpu_pm and serves as the reference here).

Per output: final displacement RMS <= 1e-3 cell, per-shell P(k) <= 1e-4 relative, dJ/domega
cosine >= 0.999.  The relative L2 of dJ/domega is not held to 1e-3 here: the exact gradient
of the CIC objective jumps by ~1/l wherever a particle-step crosses a cell face (Eq. 10),
so it is not a continuous function of the trajectory, and any trajectory difference of
FP32 size moves it by more than 1e-3 at this size.  The test shows that this, and not the
FP32 arithmetic of the adjoint, sets the error: an FP64 run whose inputs are moved so that
its trajectory differs from the reference by as much as the FP32 run's does (omega moved
by a multiple of one FP32 ulp, scaled from a one-ulp run) moves the gradient by a similar
amount; the FP32 error must stay within three times that (the crossings are few and
random, so two such realisations differ by a factor of order one)."""
import numpy as np
import pytest

from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
BOX, NM, NP, NS = 200.0, 256, 128, 63


def _run(precision, omega, target):
    torch = torch_cuda()
    ctx, *_ = make_ctx(BOX, NM, NP, NS, precision=precision, omega=omega[None])
    dt = ctx.dtype
    N, M = NP ** 3, NM ** 3
    disp = torch.empty(3 * N, device="cuda", dtype=dt)
    ctx.forward(disp=disp)
    _, pk, nmodes = ctx.power_spectrum()
    djdd = torch.empty(M, device="cuda", dtype=dt)
    ctx.loss_mse(torch.from_numpy(target).to("cuda", dt), djdd)
    gw = torch.empty(N, device="cuda", dtype=dt)
    gt = torch.zeros(5, dtype=torch.float64)
    ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
    ctx.close()
    return (disp.cpu().numpy().astype(np.float64), pk[0], nmodes, gw.cpu().numpy().astype(np.float64), gt.numpy())


def _moved(omega, ulps):
    """omega with every value moved by `ulps` FP32 spacings, signs seeded."""
    sign = np.where(inputs.uniform01(77, omega.size).reshape(omega.shape) < 0.5, -1.0, 1.0)
    return omega + ulps * sign * np.spacing(np.abs(omega.astype(np.float32))).astype(np.float64)


def test_fp32_against_fp64_at_128_cubed():
    torch = torch_cuda()
    om = inputs.white_noise(NP, 1).astype(np.float64)
    ctx, *_ = make_ctx(BOX, NM, NP, NS, precision=1, omega=inputs.white_noise(NP, 2).astype(np.float64)[None])
    t = torch.empty(NM ** 3, device="cuda", dtype=torch.float64)
    ctx.forward(dens=t)
    target = t.cpu().numpy()
    ctx.close()
    cell = BOX / NM
    s64, pk64, nmodes, g64, gt64 = _run(1, om, target)
    s32, pk32, _, g32, gt32 = _run(0, om, target)
    d32 = np.sqrt(np.mean((s32 - s64) ** 2))
    assert d32 <= 1e-3 * cell
    ok = nmodes > 0
    ok[0] = False
    assert np.max(np.abs(pk32[ok] / pk64[ok] - 1)) <= 1e-4
    assert cosine(g32, g64) >= 0.999
    assert np.all(np.abs(gt32 / gt64 - 1) <= 1e-2)
    # the conditioning control: FP64 with a trajectory difference of the FP32 size
    s1, _, _, _, _ = _run(1, _moved(om, 1.0), target)
    d1 = np.sqrt(np.mean((s1 - s64) ** 2))
    k = d32 / d1
    sk, _, _, gk, _ = _run(1, _moved(om, k), target)
    dk = np.sqrt(np.mean((sk - s64) ** 2))
    assert 0.5 * d32 <= dk <= 2.0 * d32          # the displacement difference scales with the move
    floor = rel_l2(gk, g64)
    err = rel_l2(g32, g64)
    print(f"FP32 vs FP64: disp {d32 / cell:.2e} cell, dJ/domega rel-L2 {err:.2e}; FP64 moved by {k:.1f} FP32 ulps: "
          f"disp {dk / cell:.2e} cell, dJ/domega rel-L2 {floor:.2e}")
    assert err <= 3.0 * floor
