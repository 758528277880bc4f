"""pm_density_noalloc -- the CIC density for callers that cannot call cudaMalloc (their
device memory belongs to their own pool allocator, or they cannot afford the device
synchronisation of an allocation) -- against the context-based pm_op_density (the same
fixed-point quantum, so bit for bit) and against the FP64 oracle's CIC density.

Runs last (file name) so that a failure here cannot hide the other tests; it builds the
library itself, so it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from oracle import pm as opm

from gpu_util import ensure_built, oracle_cfg, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_mesh,n_ptcl", [(32, 16), (128, 64)])
def test_noalloc_density_matches_context_density_on_two_calls(n_mesh, n_ptcl):
    torch = torch_cuda()
    ensure_built()
    from paper_2211_09815_gb300 import inputs, pm
    box = 100.0
    N = n_ptcl ** 3
    rng = np.random.default_rng(n_mesh)
    om = torch.from_numpy(inputs.white_noise(n_ptcl, 1)).cuda()
    ctx = pm.PMContext(box, n_mesh, n_ptcl, 1, [inputs.THETA_FIDUCIAL], om)
    for call in range(2):   # two calls in a row: the shared array must be cleared each time
        disp = torch.from_numpy(rng.normal(scale=2.0 + call, size=3 * N).astype(np.float32)).cuda()
        ref = torch.empty(n_mesh ** 3, device="cuda")
        ctx.op_density(disp, ref)
        got = torch.full((n_mesh ** 3,), float("nan"), device="cuda")
        pm.density_noalloc(box, n_mesh, n_ptcl, disp, got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        # the same fixed-point deposit with the same quantum: equal bit for bit
        assert np.array_equal(g, r)
        # and the CIC density of the oracle to FP32 rounding of the weights
        cfg = oracle_cfg(box, n_mesh, n_ptcl, 1)
        x = opm.lattice(cfg) + disp.cpu().numpy().astype(np.float64).reshape(3, -1)
        o = opm.density(x, cfg).ravel()
        assert np.max(np.abs(g - o)) <= 1e-5 * np.max(np.abs(o))
    ctx.close()


def test_noalloc_rejects_meshes_beyond_the_fixed_array():
    torch = torch_cuda()
    ensure_built()
    from paper_2211_09815_gb300 import pm
    lib = pm.load_library()
    disp = torch.zeros(3 * 64 ** 3, device="cuda")
    dens = torch.zeros(8, device="cuda")
    import ctypes
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = lib.pm_density_noalloc(100.0, 256, 64, ctypes.c_void_p(disp.data_ptr()),
                                    ctypes.c_void_p(dens.data_ptr()), st)
    assert status == 1    # PM_ERR_ARG: 256^3 cells exceed PM_NOALLOC_MAX_CELLS
    with pytest.raises(ValueError):
        pm.density_noalloc(100.0, 256, 64, disp, dens)
