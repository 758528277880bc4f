"""GPU parity of the whole forward model and the adjoint gradient against the FP64 oracle,
through the C ABI (pm_forward, pm_loss_mse, pm_adjoint).

Tolerances: FP64 runs agree with the oracle to rounding amplified by the dynamics
(<= 1e-8 relative here).  FP32 runs are held to the accuracy targets of the method's
FP32 form: displacement RMS <= 1e-3 cell, gradient cosine >= 0.999 and relative L2
<= 1e-3, theta gradient relative error <= 1e-3.
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu
THETA = inputs.THETA_FIDUCIAL

# the small FP64 configuration: 32^3 particles, 64^3 mesh, 100 Mpc/h, 10 steps
C1 = dict(box=100.0, n_mesh=64, n_ptcl=32, n_steps=10)
# a smaller, more nonlinear case for the gradient checks
C0 = dict(box=32.0, n_mesh=32, n_ptcl=16, n_steps=6)


def _gpu_run(cfg, precision, seed=1, ckpt_every=0, batch=1, theta=THETA, target=None, omega=None):
    torch = torch_cuda()
    ctx, om_t, omega, th = make_ctx(cfg["box"], cfg["n_mesh"], cfg["n_ptcl"], cfg["n_steps"], precision=precision,
                                    seed=seed, ckpt_every=ckpt_every, batch=batch, theta=theta, omega=omega)
    N, M = cfg["n_ptcl"] ** 3, cfg["n_mesh"] ** 3
    disp = torch.empty(batch * 3 * N, device="cuda", dtype=ctx.dtype)
    mom = torch.empty_like(disp)
    dens = torch.empty(batch * M, device="cuda", dtype=ctx.dtype)
    ctx.forward(disp, mom, dens)
    out = dict(s=disp.cpu().numpy().reshape(batch, 3, N), p=mom.cpu().numpy().reshape(batch, 3, N),
               delta=dens.cpu().numpy().reshape(batch, M), omega=omega, theta=th)
    if target is not None:
        tgt = torch.from_numpy(np.ascontiguousarray(target)).to("cuda", ctx.dtype)
        djdd = torch.empty(batch * M, device="cuda", dtype=ctx.dtype)
        loss = ctx.loss_mse(tgt, djdd)
        gw = torch.empty(batch * N, device="cuda", dtype=ctx.dtype)
        gt = torch.zeros(batch * 5, dtype=torch.float64)
        ctx.adjoint(djdd=djdd, grad_omega=gw, grad_theta=gt)
        out.update(loss=loss.numpy().copy(), grad_omega=gw.cpu().numpy().reshape(batch, N),
                   grad_theta=gt.numpy().reshape(batch, 5))
    ctx.close()
    return out


@pytest.fixture(scope="module")
def oracle_c1():
    cfg = oracle_cfg(**C1)
    om = inputs.white_noise(C1["n_ptcl"], 1).astype(np.float64)
    return opm.forward(om, THETA, cfg)


def test_forward_fp64_matches_oracle(oracle_c1):
    g = _gpu_run(C1, 1)
    assert rel_l2(g["s"][0], oracle_c1["s"]) < 1e-9
    assert rel_l2(g["p"][0], oracle_c1["p"]) < 1e-9
    assert np.max(np.abs(g["delta"][0] - oracle_c1["delta"].ravel())) < 1e-8


def test_forward_fp32_displacement_rms_below_1e3_cell(oracle_c1):
    g = _gpu_run(C1, 0)
    cell = C1["box"] / C1["n_mesh"]
    rms = np.sqrt(np.mean((g["s"][0].astype(np.float64) - oracle_c1["s"]) ** 2))
    assert rms < 1e-3 * cell
    assert rel_l2(g["p"][0], oracle_c1["p"]) < 1e-3


def test_forward_is_bitwise_deterministic():
    a = _gpu_run(C1, 0)
    b = _gpu_run(C1, 0)
    assert np.array_equal(a["s"], b["s"]) and np.array_equal(a["p"], b["p"])
    assert np.array_equal(a["delta"], b["delta"])


@pytest.fixture(scope="module")
def oracle_grad_c0():
    cfg = oracle_cfg(**C0)
    om = inputs.white_noise(C0["n_ptcl"], 1).astype(np.float64)
    target = opm.forward(inputs.white_noise(C0["n_ptcl"], 2).astype(np.float64), THETA, cfg)["delta"]
    loss, adj, _ = opm.loss_and_gradient(om, THETA, target, cfg)
    return target, loss, adj


def test_adjoint_fp64_matches_oracle(oracle_grad_c0):
    target, loss, adj = oracle_grad_c0
    g = _gpu_run(C0, 1, target=target.ravel()[None])
    assert abs(g["loss"][0] / loss - 1) < 1e-10
    assert rel_l2(g["grad_omega"][0], adj["grad_omega"]) < 1e-8
    assert np.allclose(g["grad_theta"][0], adj["grad_theta"], rtol=1e-8, atol=0)


def test_adjoint_fp32_gradient_accuracy(oracle_grad_c0):
    target, loss, adj = oracle_grad_c0
    g = _gpu_run(C0, 0, target=target.ravel()[None])
    assert abs(g["loss"][0] / loss - 1) < 1e-4
    assert cosine(g["grad_omega"][0], adj["grad_omega"]) >= 0.999
    assert rel_l2(g["grad_omega"][0], adj["grad_omega"]) <= 1e-3
    assert np.all(np.abs(g["grad_theta"][0] / adj["grad_theta"] - 1) < 1e-3)


def test_adjoint_checkpoint_mode_fp64_matches_oracle():
    cfg = oracle_cfg(**C0)
    om = inputs.white_noise(C0["n_ptcl"], 1).astype(np.float64)
    target = opm.forward(inputs.white_noise(C0["n_ptcl"], 2).astype(np.float64), THETA, cfg)["delta"]
    _, adj, _ = opm.loss_and_gradient(om, THETA, target, cfg, ckpt_every=2)
    g = _gpu_run(C0, 1, ckpt_every=2, target=target.ravel()[None])
    assert rel_l2(g["grad_omega"][0], adj["grad_omega"]) < 1e-8
    assert np.allclose(g["grad_theta"][0], adj["grad_theta"], rtol=1e-8)


def test_batched_instances_equal_single_runs():
    theta2 = np.array([THETA, (2.3e-9, 0.95, 0.28, 0.049, 0.68)])
    cfg = dict(C0)
    tgt = np.zeros((2, cfg["n_mesh"] ** 3))
    both = _gpu_run(cfg, 0, batch=2, theta=theta2, target=tgt)
    for b in range(2):
        one = _gpu_run(cfg, 0, seed=1 + b, theta=theta2[b], target=tgt[b:b + 1])
        assert np.array_equal(one["s"][0], both["s"][b])
        assert np.array_equal(one["grad_omega"][0], both["grad_omega"][b])
        assert np.array_equal(one["grad_theta"][0], both["grad_theta"][b])


def test_graph_replay_equals_eager_batched():
    """pm_gradient_graph (captured once, replayed with new omega) gives the eager result
    bit for bit, for a batch of two instances with different cosmologies."""
    torch = torch_cuda()
    from paper_2211_09815_gb300 import pm
    cfg = dict(C0)
    N, M = cfg["n_ptcl"] ** 3, cfg["n_mesh"] ** 3
    theta2 = [THETA, (2.3e-9, 0.95, 0.28, 0.049, 0.68)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        om = torch.from_numpy(np.stack([inputs.white_noise(cfg["n_ptcl"], s) for s in (1, 2)])).cuda()
        ctx = pm.PMContext(cfg["box"], cfg["n_mesh"], cfg["n_ptcl"], cfg["n_steps"], theta2, om, batch=2,
                           stream=stream)
        tgt = torch.zeros(2 * M, device="cuda")
        loss = torch.zeros(2, dtype=torch.float64, device="cuda")
        gw = torch.empty(2 * N, device="cuda")
        gt = torch.zeros(10, dtype=torch.float64, device="cuda")
        results = []
        for seeds in ((1, 2), (3, 4), (1, 2)):
            om2 = torch.from_numpy(np.stack([inputs.white_noise(cfg["n_ptcl"], s) for s in seeds])).cuda()
            ctx.set_inputs(omega=om2)
            ctx.gradient_graph(tgt, loss=loss, grad_omega=gw, grad_theta=gt)
            stream.synchronize()
            g_graph = (gw.cpu().numpy().copy(), gt.cpu().numpy().copy(), loss.cpu().numpy().copy())
            ctx.set_inputs(omega=om2)
            ctx.forward()
            djdd = torch.empty(2 * M, device="cuda")
            ctx.loss_mse(tgt, djdd)
            gw2 = torch.empty(2 * N, device="cuda")
            gt2 = torch.zeros(10, dtype=torch.float64, device="cuda")
            ctx.adjoint(djdd=djdd, grad_omega=gw2, grad_theta=gt2)
            stream.synchronize()
            assert np.array_equal(g_graph[0], gw2.cpu().numpy())
            assert np.array_equal(g_graph[1], gt2.cpu().numpy())
            results.append(g_graph)
        assert not np.array_equal(results[0][0], results[1][0])
        assert np.array_equal(results[0][0], results[2][0])
        ctx.close()
