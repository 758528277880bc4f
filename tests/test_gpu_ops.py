"""GPU parity of the hot-path rows against the FP64 oracle, called through the C ABI.

Sizes span several FFT tiles and ragged tails (tile widths are 8..256 sequences); each
operator is compared element by element.  Tolerances: FP64 runs to ~1e-10 relative,
FP32 runs to a few float32 ulps amplified by the transform length (derived per test).
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL


@pytest.mark.parametrize("precision,n,batch", [(1, 8, 1), (1, 16, 2), (0, 32, 1), (0, 64, 2), (1, 128, 1),
                                               (0, 128, 2), (0, 256, 1)])
def test_fft_roundtrip_matches_numpy(precision, n, batch):
    torch = torch_cuda()
    ctx, *_ = make_ctx(100.0, n, min(n, 8), 1, precision=precision, batch=batch)
    rng = np.random.default_rng(n)
    x = rng.normal(size=(batch, n, n, n))
    dt = torch.float32 if precision == 0 else torch.float64
    xt = torch.from_numpy(x).to("cuda", dt).contiguous()
    spec = torch.empty(batch, n, n, n // 2 + 1, 2, device="cuda", dtype=dt)
    ctx.op_fft(-1, xt, spec)
    ref = np.fft.rfftn(x.astype(np.float32 if precision == 0 else np.float64).astype(np.float64), axes=(1, 2, 3))
    got = spec.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    tol = 1e-12 if precision else 2e-6 * np.log2(n ** 3)
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    back = torch.empty(batch, n, n, n, device="cuda", dtype=dt)
    ctx.op_fft(+1, spec, back)
    assert np.max(np.abs(back.cpu().numpy() / n ** 3 - x)) <= tol * np.max(np.abs(x))
    ctx.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_za_displacement_matches_oracle(precision):
    torch = torch_cuda()
    box, nm, npc = 64.0, 32, 16
    ctx, _, omega, _ = make_ctx(box, nm, npc, 1, precision=precision)
    s1 = torch.empty(3 * npc ** 3, device="cuda", dtype=ctx.dtype)
    ctx.op_za(s1)
    ref = opm.za_unit_displacement(omega[0].astype(np.float64), THETA, oracle_cfg(box, nm, npc, 1))
    got = s1.cpu().numpy().reshape(3, -1)
    tol = 1e-10 if precision else 2e-5
    assert rel_l2(got, ref) < tol
    ctx.close()


@pytest.mark.parametrize("precision,nm,npc", [(1, 16, 8), (0, 32, 16), (1, 32, 8)])
def test_density_matches_oracle(precision, nm, npc):
    torch = torch_cuda()
    box = 50.0
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=precision)
    rng = np.random.default_rng(3)
    disp = rng.normal(scale=3.0, size=(3, npc ** 3))
    d = torch.from_numpy(disp).to("cuda", ctx.dtype).contiguous()
    out = torch.empty(nm ** 3, device="cuda", dtype=ctx.dtype)
    ctx.op_density(d, out)
    cfg = oracle_cfg(box, nm, npc, 1)
    x = opm.lattice(cfg) + d.cpu().numpy().astype(np.float64)
    ref = opm.density(x, cfg).ravel()
    got = out.cpu().numpy().astype(np.float64)
    tol = 1e-11 if precision else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    # mass conservation: sum(delta) = 0 up to the fixed-point quantum
    assert abs(got.sum()) < (1e-9 if precision else 1e-3) * nm ** 3
    ctx.close()


@pytest.mark.parametrize("precision,nm,npc", [(1, 16, 8), (0, 32, 16), (0, 128, 64), (1, 128, 32), (0, 256, 64)])
def test_force_and_vjp_match_oracle(precision, nm, npc):
    """Meshes of 128^3 and more take the TMA-staged persistent column and fused passes."""
    torch = torch_cuda()
    box = 40.0
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=precision)
    rng = np.random.default_rng(4)
    disp = rng.normal(scale=2.0, size=(3, npc ** 3))
    pi = rng.normal(size=(3, npc ** 3))
    d = torch.from_numpy(disp).to("cuda", ctx.dtype).contiguous()
    p = torch.from_numpy(pi).to("cuda", ctx.dtype).contiguous()
    acc = torch.empty(3 * npc ** 3, device="cuda", dtype=ctx.dtype)
    alpha = torch.empty_like(acc)
    ctx.op_force(d, acc)
    cfg = oracle_cfg(box, nm, npc, 1)
    x = opm.lattice(cfg) + d.cpu().numpy().astype(np.float64)
    a_ref, f = opm.pm_force(x, THETA[2], cfg)
    tol = 1e-10 if precision else 3e-5
    assert rel_l2(acc.cpu().numpy().reshape(3, -1), a_ref) < tol
    acc2 = torch.empty_like(acc)
    ctx.op_force_vjp(d, p, acc2, alpha)
    al_ref = opm.force_vjp(x, p.cpu().numpy().astype(np.float64), f, THETA[2], cfg)
    assert rel_l2(acc2.cpu().numpy().reshape(3, -1), a_ref) < tol
    assert rel_l2(alpha.cpu().numpy().reshape(3, -1), al_ref) < tol
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_density_of_collapsed_particles_matches_oracle(precision):
    """All 64^3 particles collapsed into a few cells: one mesh tile receives more than 2^16
    particle visits, which takes the exact 64-bit accumulation path of the deposit."""
    torch = torch_cuda()
    box, nm, npc = 64.0, 64, 64
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=precision)
    cfg = oracle_cfg(box, nm, npc, 1)
    q = opm.lattice(cfg)
    rng = np.random.default_rng(8)
    target = np.array([[20.3], [33.7], [41.1]])
    disp = target - q + rng.normal(scale=0.6, size=q.shape)
    d = torch.from_numpy(disp).to("cuda", ctx.dtype).contiguous()
    out = torch.empty(nm ** 3, device="cuda", dtype=ctx.dtype)
    ctx.op_density(d, out)
    ref = opm.density(q + d.cpu().numpy().astype(np.float64), cfg).ravel()
    got = out.cpu().numpy().astype(np.float64)
    tol = 1e-11 if precision else 1e-6
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
    assert abs((got + 1).sum() - nm ** 3) <= (1e-9 if precision else 1e-5) * nm ** 3
    ctx.close()
