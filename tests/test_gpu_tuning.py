"""Launch-shape tuning (pm_get_tuning / pm_set_tuning / pm_autotune) through the C ABI.

The tunable shapes change speed, never results: the CIC deposit sums exact integers for
any tile shape, so densities must be bitwise equal across shapes, and the staged and
unstaged column passes run the same radix stages.  The autotuner must leave the forward
state usable for the adjoint.
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import cosine, make_ctx, oracle_cfg, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def test_set_tuning_rejects_invalid_shapes():
    torch_cuda()
    from paper_2211_09815_gb300 import pm
    ctx, *_ = make_ctx(50.0, 32, 16, 2)
    t = ctx.get_tuning()
    assert t["threads_density"] in (256, 512) and t["threads_adjoint"] in (256, 512)
    for bad in ({"tile_log2_density": [4, 4, 5]},       # 2^13 cells
                {"tile_log2_adjoint": [4, 4, 4]},       # 2^12 cells with the pi sums
                {"tile_log2_adjoint": [2, 2, 2]},       # 2^6 cells
                {"threads_density": 128},
                {"tma_columns": 1},                     # no staged passes below 128^3
                {"fused_x": 3}):                        # no fused deposit below 128^3
        with pytest.raises(pm.PMError):
            ctx.set_tuning(bad)
    assert ctx.get_tuning() == t
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_density_bitwise_equal_across_tile_shapes(precision):
    torch = torch_cuda()
    box, nm, npc = 64.0, 64, 32
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=precision)
    rng = np.random.default_rng(11)
    # clustered: half the particles pulled towards a few points
    disp = rng.normal(scale=4.0, size=(3, npc ** 3))
    disp[:, ::2] *= 0.05
    d = torch.from_numpy(disp).to("cuda", ctx.dtype).contiguous()
    outs = []
    for tile, nt in (([3, 4, 4], 256), ([3, 3, 5], 512), ([3, 3, 3], 256), ([2, 4, 5], 512), ([4, 4, 4], 256)):
        ctx.set_tuning({"tile_log2_density": tile, "threads_density": nt})
        out = torch.empty(nm ** 3, device="cuda", dtype=ctx.dtype)
        ctx.op_density(d, out)
        outs.append(out.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    cfg = oracle_cfg(box, nm, npc, 1)
    ref = opm.density(opm.lattice(cfg) + disp, cfg).ravel()
    tol = 1e-11 if precision else 1e-5
    assert np.max(np.abs(outs[0] - ref)) <= tol * np.max(np.abs(ref))
    ctx.close()


def test_force_vjp_equal_across_shapes_and_column_forms():
    """128^3 mesh: the adjoint deposit shapes and the staged/unstaged column passes."""
    torch = torch_cuda()
    box, nm, npc = 60.0, 128, 64
    ctx, *_ = make_ctx(box, nm, npc, 1, precision=0)
    rng = np.random.default_rng(5)
    d = torch.from_numpy(rng.normal(scale=2.0, size=(3, npc ** 3))).to("cuda", torch.float32).contiguous()
    p = torch.from_numpy(rng.normal(size=(3, npc ** 3))).to("cuda", torch.float32).contiguous()
    res = []
    for tune in ({"tile_log2_adjoint": [3, 4, 4], "threads_adjoint": 512, "tma_columns": 1},
                 {"tile_log2_adjoint": [2, 4, 5], "threads_adjoint": 256, "tma_columns": 1},
                 {"tile_log2_adjoint": [3, 3, 4], "threads_adjoint": 512, "tma_columns": 0}):
        ctx.set_tuning(tune)
        acc = torch.empty(3 * npc ** 3, device="cuda")
        alpha = torch.empty_like(acc)
        ctx.op_force_vjp(d, p, acc, alpha)
        res.append((acc.cpu().numpy(), alpha.cpu().numpy()))
    # deposit shapes alone: bitwise; column form: the same stages, FP32 rounding at most
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert rel_l2(res[2][0], res[0][0]) < 1e-6 and rel_l2(res[2][1], res[0][1]) < 1e-6
    ctx.close()


def test_autotune_keeps_forward_state_and_gradient():
    torch = torch_cuda()
    cfg = dict(box=64.0, n_mesh=128, n_ptcl=64, n_steps=4)
    N, M = cfg["n_ptcl"] ** 3, cfg["n_mesh"] ** 3
    ctx, *_ = make_ctx(cfg["box"], cfg["n_mesh"], cfg["n_ptcl"], cfg["n_steps"], precision=0)
    tgt = torch.from_numpy(inputs.white_noise(cfg["n_mesh"], 9).ravel() * 0.1).to("cuda", torch.float32)

    default = ctx.get_tuning()
    chosen = {}

    def gradient(tune_between):
        dens = torch.empty(M, device="cuda")
        ctx.forward(dens=dens)
        if tune_between:
            t, ms = ctx.autotune(reps=2)
            assert t["threads_density"] in (256, 512) and all(m > 0 for m in ms)
            assert sum(t["tile_log2_adjoint"]) in (9, 10, 11) and t["fused_x"] in (0, 1, 2, 3)
            chosen.update(t)
        djdd = torch.empty(M, device="cuda")
        loss = ctx.loss_mse(tgt, djdd)
        gw = torch.empty(N, device="cuda")
        ctx.adjoint(djdd=djdd, grad_omega=gw)
        return dens.cpu().numpy(), float(loss[0]), gw.cpu().numpy()

    d0, l0, g0 = gradient(False)
    d1, l1, g1 = gradient(True)
    assert np.array_equal(d0, d1) and l0 == l1
    if chosen["tma_columns"] == default["tma_columns"] and chosen["fused_x"] == default["fused_x"]:
        # deposit shapes only: exact integer sums, the same gradient bit for bit
        assert np.array_equal(g1, g0)
    else:
        # the other column-pass or x-pass form rounds differently in the last bit; the FP32
        # reverse integration amplifies that to the FP32 accuracy class of the gradient
        assert cosine(g1, g0) > 0.9999 and rel_l2(g1, g0) < 1e-3
    ctx.close()


@pytest.mark.parametrize("precision,nm,npc", [(0, 128, 64), (1, 128, 32), (0, 256, 64)])
def test_fused_deposit_and_x_pass_match_separate_passes(precision, nm, npc):
    """The deposit fused with the R2C x pass (whole-row tiles, spectra written from shared
    memory) against the separate deposit and x pass: the same exact integer sums, the same
    conversion and radix stages.  The final density of a forward run is bitwise equal; the
    forces, the VJP and the forward state equal to the last-bit rounding of the transform
    (relative 1e-6), and both match the oracle."""
    torch = torch_cuda()
    box = 60.0
    ctx, *_ = make_ctx(box, nm, npc, 3, precision=precision)
    rng = np.random.default_rng(6)
    d = torch.from_numpy(rng.normal(scale=2.0 * box / nm, size=(3, npc ** 3))).to("cuda", ctx.dtype).contiguous()
    p = torch.from_numpy(rng.normal(size=(3, npc ** 3))).to("cuda", ctx.dtype).contiguous()
    res = []
    for fused in (3, 0):
        ctx.set_tuning({"fused_x": fused})
        assert ctx.get_tuning()["fused_x"] == fused
        acc = torch.empty(3 * npc ** 3, device="cuda", dtype=ctx.dtype)
        acc2, alpha = torch.empty_like(acc), torch.empty_like(acc)
        ctx.op_force(d, acc)
        ctx.op_force_vjp(d, p, acc2, alpha)
        dens = torch.empty(nm ** 3, device="cuda", dtype=ctx.dtype)
        disp = torch.empty(3 * npc ** 3, device="cuda", dtype=ctx.dtype)
        ctx.forward(disp=disp, dens=dens)
        res.append([x.cpu().numpy() for x in (acc, acc2, alpha, dens, disp)])
    tol = 1e-13 if precision else 1e-6
    for a, b in zip(res[0][:3], res[1][:3]):
        assert rel_l2(a, b) < tol
    assert rel_l2(res[0][4], res[1][4]) < tol
    # the final density is the deposit's real output at the last step's positions
    if np.array_equal(res[0][4], res[1][4]):
        assert np.array_equal(res[0][3], res[1][3])
    cfg = oracle_cfg(box, nm, npc, 1)
    x = opm.lattice(cfg) + d.cpu().numpy().astype(np.float64)
    a_ref, _ = opm.pm_force(x, inputs.THETA_FIDUCIAL[2], cfg)
    assert rel_l2(res[0][0].reshape(3, -1), a_ref) < (1e-10 if precision else 3e-5)
    ctx.close()
