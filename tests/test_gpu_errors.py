"""Error paths on the GPU without a GPU fault: a bounded device wait that gives up
(PM_ERR_TIMEOUT) and a failing device allocation (PM_ERR_OOM), both injected from the host
through the library's test hooks, followed by a clean, correct call.
"""
import ctypes

import numpy as np
import pytest

from paper_2211_09815_gb300 import inputs

from gpu_util import ensure_built, make_ctx, torch_cuda

pytestmark = pytest.mark.gpu
PM_ERR_OOM, PM_ERR_TIMEOUT = 2, 6


def test_tma_wait_timeout_is_reported_and_the_next_call_is_correct():
    """The first mbarrier wait of every CTA of the TMA-staged column passes (128^3 mesh)
    is given a spin limit of 0: each CTA sets the device flag, drains the copies it has in
    flight (bounded wait) and returns.  pm_check reports PM_ERR_TIMEOUT once and clears the
    flag; with the normal limit restored the same transform matches numpy."""
    torch = torch_cuda()
    from paper_2211_09815_gb300 import pm
    lib = pm.load_library()
    n = 128
    ctx, *_ = make_ctx(100.0, n, 16, 1)
    x = torch.from_numpy(np.random.default_rng(5).normal(size=(n, n, n)).astype(np.float32)).cuda()
    spec = torch.empty(n, n, n // 2 + 1, 2, device="cuda")
    assert lib.pm_debug_first_wait(ctx._h, 0) == 0
    with pytest.raises(pm.PMError) as e:
        ctx.op_fft(-1, x, spec)
    assert e.value.status == PM_ERR_TIMEOUT
    assert lib.pm_check(ctx._h) == 0                    # reported once, then cleared
    # a call that synchronises for a host output reports it directly
    ctx.check_errors = False
    tgt = torch.zeros(n ** 3, dtype=torch.float32).pin_memory()
    loss = torch.zeros(1, dtype=torch.float64).pin_memory()
    status = lib.pm_gradient(ctx._h, None, ctypes.c_void_p(tgt.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                             None, None)
    assert status == PM_ERR_TIMEOUT
    ctx.check_errors = True
    assert lib.pm_debug_first_wait(ctx._h, -1) == 0
    ctx.op_fft(-1, x, spec)
    ref = np.fft.rfftn(x.cpu().numpy().astype(np.float64))
    got = spec.cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.log2(n ** 3) * np.max(np.abs(ref))
    ctx.close()


def test_failed_allocation_returns_oom_and_leaks_nothing():
    """The k-th device allocation of pm_init (or of a later lazily allocating call) fails
    as if cudaMalloc had: the call returns PM_ERR_OOM, the partly built context frees
    everything (live bytes and free device memory back to where they were), and the next
    call succeeds."""
    torch = torch_cuda()
    ensure_built()
    from paper_2211_09815_gb300 import pm
    lib = pm.load_library()
    box, nm, npc = 64.0, 64, 32
    cfg = pm.PMConfig(box, nm, npc, 2, 1 / 64, 1.0, 0, 0, 0, 1, 1)
    th = (ctypes.c_double * 5)(*inputs.THETA_FIDUCIAL)
    om = torch.from_numpy(inputs.white_noise(npc, 1)).cuda()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    live0 = lib.pm_debug_live_bytes()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in (0, 1, 5, 12, 30):
        h = ctypes.c_void_p()
        lib.pm_debug_fail_alloc(k)
        status = lib.pm_init(ctypes.byref(h), ctypes.byref(cfg), th, ctypes.c_void_p(om.data_ptr()), st)
        lib.pm_debug_fail_alloc(-1)
        if status == 0:
            lib.pm_destroy(h)   # k beyond the allocations of pm_init
        else:
            assert status == PM_ERR_OOM
            failures += 1
        torch.cuda.synchronize()
        assert lib.pm_debug_live_bytes() == live0
    assert failures >= 4
    assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)
    # a lazily allocated buffer: the first pm_gradient allocates the target and gradients
    ctx, *_ = make_ctx(box, nm, npc, 2)
    live1 = lib.pm_debug_live_bytes()
    tgt = torch.zeros(nm ** 3, device="cuda")
    lib.pm_debug_fail_alloc(0)
    status = lib.pm_gradient(ctx._h, None, ctypes.c_void_p(tgt.data_ptr()), None, None, None)
    lib.pm_debug_fail_alloc(-1)
    assert status == PM_ERR_OOM
    assert lib.pm_debug_live_bytes() == live1
    gw = torch.empty(npc ** 3, device="cuda")
    ctx.gradient(tgt, grad_omega=gw)
    assert bool(torch.isfinite(gw).all())
    ctx.close()
    assert lib.pm_debug_live_bytes() == live0
