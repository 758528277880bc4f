"""The C-ABI library builds, loads and exports every entry point that include/pm.h
declares (no compute calls: no GPU needed)."""
import os
import re

from paper_2211_09815_gb300 import build, pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|long long)\s+(pm_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("pm_init", "pm_forward", "pm_adjoint", "pm_destroy", "pm_status_string", "pm_loss_mse"):
        assert required in names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = pm.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(_declared()) <= set(pm.SYMBOLS) | {"pm_status_string"}
    assert lib.pm_status_string(0) == b"ok"
    assert lib.pm_status_string(1) == b"invalid argument"


def test_invalid_configs_are_rejected_on_the_host():
    """Validation happens before any CUDA call, so it runs without a GPU."""
    import ctypes
    lib = pm.load_library()
    h = ctypes.c_void_p()
    th = (ctypes.c_double * 5)(2.1e-9, 0.965, 0.31, 0.049, 0.68)
    dummy = ctypes.c_void_p(16)
    bad = [
        pm.PMConfig(100.0, 48, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1),    # mesh not a power of two
        pm.PMConfig(100.0, 32, 64, 10, 1 / 64, 1.0, 0, 0, 0, 1),    # mesh not a multiple of n_ptcl
        pm.PMConfig(100.0, 2048, 64, 10, 1 / 64, 1.0, 0, 0, 0, 1),  # mesh too large
        pm.PMConfig(-1.0, 32, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1),     # box
        pm.PMConfig(100.0, 32, 16, 0, 1 / 64, 1.0, 0, 0, 0, 1),     # steps
        pm.PMConfig(100.0, 32, 16, 10, 1.0, 0.5, 0, 0, 0, 1),       # a1 < a0
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 7, 0, 0, 1),    # precision
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1, 3), # LPT order
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1, 1, 2),   # fixed_state flag
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 0, 8, 0, 1, 1, 1),   # fixed state with checkpoints
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1, 1, 0, 2),   # half_force flag
        pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 1, 0, 0, 1, 1, 0, 1),   # FP16 force mesh with FP64
    ]
    for cfg in bad:
        assert lib.pm_init(ctypes.byref(h), ctypes.byref(cfg), th, dummy, None) == 1
    nan = (ctypes.c_double * 5)(float("nan"), 0.965, 0.31, 0.049, 0.68)
    ok = pm.PMConfig(100.0, 32, 16, 10, 1 / 64, 1.0, 0, 0, 0, 1)
    assert lib.pm_init(ctypes.byref(h), ctypes.byref(ok), nan, dummy, None) == 4
    assert lib.pm_forward(None, None, None, None) == 1


def test_new_entry_points_reject_null_arguments_on_the_host():
    """pm_op_ic, pm_loss_power and pm_set_snapshots check their pointers before any CUDA
    call."""
    import ctypes
    lib = pm.load_library()
    d = (ctypes.c_double * 4)()
    assert lib.pm_op_ic(None, None, None) == 1
    assert lib.pm_loss_power(None, None, d, d, None, ctypes.c_void_p(16)) == 1
    assert lib.pm_set_snapshots(None, 0, None, None, None, None, None) == 1


def test_noalloc_rejects_bad_arguments_on_the_host():
    """pm_density_noalloc checks its arguments as pm_init does (finite box, power-of-two
    sizes, 8 <= n_mesh, n_ptcl | n_mesh) before any CUDA call."""
    import ctypes
    lib = pm.load_library()
    d = ctypes.c_void_p(256)
    assert lib.pm_density_noalloc(float("nan"), 32, 16, d, d, None) == 1
    assert lib.pm_density_noalloc(float("inf"), 32, 16, d, d, None) == 1
    assert lib.pm_density_noalloc(-1.0, 32, 16, d, d, None) == 1
    assert lib.pm_density_noalloc(100.0, 4, 4, d, d, None) == 1     # below 8 cells per side
    assert lib.pm_density_noalloc(100.0, 48, 16, d, d, None) == 1    # not a power of two
    assert lib.pm_density_noalloc(100.0, 32, 64, d, d, None) == 1    # n_ptcl does not divide n_mesh
    assert lib.pm_density_noalloc(100.0, 32, 16, None, d, None) == 1


def test_hooks_and_check_reject_null_contexts():
    lib = pm.load_library()
    assert lib.pm_check(None) == 1
    assert lib.pm_debug_first_wait(None, 0) == 1
    assert lib.pm_debug_fail_alloc(-1) == 0
    assert lib.pm_debug_live_bytes() == 0


def test_tensor_device_is_checked_before_the_call():
    """A CUDA tensor on another device than the library launches on is refused on the host
    (a stand-in tensor object: no GPU is needed)."""
    import types
    import pytest
    fake = types.SimpleNamespace(is_cuda=True, device=types.SimpleNamespace(index=1),
                                 is_contiguous=lambda: True, dtype=None, numel=lambda: 8, data_ptr=lambda: 256)
    with pytest.raises(ValueError, match="cuda:1"):
        pm._ptr(fake, device=0)
    assert pm._ptr(fake, device=1).value == 256
