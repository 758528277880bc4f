"""Thin ctypes binding of libpmgb (include/pm.h): argument marshalling only.

Every computation runs in the CUDA library; this module only converts torch tensors to
device pointers and checks shapes and dtypes.  Importing it does not need a GPU; the
first call that needs the library raises ``PMLibraryError`` if ``libpmgb.so`` has not
been built (``python -m paper_2211_09815_gb300.build``) -- there is no fallback.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpmgb.so")

PM_F32, PM_F64 = 0, 1
STATUS = {0: "PM_OK", 1: "PM_ERR_ARG", 2: "PM_ERR_OOM", 3: "PM_ERR_CUDA", 4: "PM_ERR_NONFINITE",
          5: "PM_ERR_OVERFLOW", 6: "PM_ERR_TIMEOUT", 7: "PM_ERR_STATE"}
SYMBOLS = ("pm_init", "pm_forward", "pm_loss_mse", "pm_adjoint", "pm_destroy", "pm_status_string",
           "pm_last_cuda_error", "pm_scratch_bytes", "pm_op_density", "pm_op_force", "pm_op_force_vjp",
           "pm_op_fft", "pm_op_za", "pm_set_inputs", "pm_gradient", "pm_profile", "pm_profile_read",
           "pm_density_noalloc", "pm_power_spectrum", "pm_gradient_graph", "pm_get_tuning", "pm_set_tuning",
           "pm_autotune", "pm_op_ic", "pm_loss_power", "pm_set_snapshots", "pm_check", "pm_debug_fail_alloc",
           "pm_debug_live_bytes", "pm_debug_first_wait", "pm_set_snapshot_momenta", "pm_set_interp_snapshots",
           "pm_get_fixed_state")
NOALLOC_MAX_CELLS = 128 ** 3
PROF_NAMES = ("scatter", "fft_x_r2c", "fft_cols", "fused_z_force", "fused_z_adjoint", "fft_x_c2r",
              "gather_fwd", "gather_adj", "other")


class PMLibraryError(RuntimeError):
    pass


class PMTuning(ctypes.Structure):
    """Launch shapes of the tunable passes (include/pm.h pm_tuning)."""
    _fields_ = [("tile_log2_density", ctypes.c_int * 3), ("tile_log2_adjoint", ctypes.c_int * 3),
                ("threads_density", ctypes.c_int), ("threads_adjoint", ctypes.c_int), ("tma_columns", ctypes.c_int),
                ("fused_x", ctypes.c_int)]

    def as_dict(self):
        return {"tile_log2_density": list(self.tile_log2_density), "tile_log2_adjoint": list(self.tile_log2_adjoint),
                "threads_density": self.threads_density, "threads_adjoint": self.threads_adjoint,
                "tma_columns": self.tma_columns, "fused_x": self.fused_x}


class PMError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {detail}".strip())


class PMConfig(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double), ("n_mesh", ctypes.c_int), ("n_ptcl", ctypes.c_int),
                ("n_steps", ctypes.c_int), ("a0", ctypes.c_double), ("a1", ctypes.c_double),
                ("precision", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("deconv", ctypes.c_int),
                ("batch", ctypes.c_int), ("lpt_order", ctypes.c_int), ("fixed_state", ctypes.c_int),
                ("half_force", ctypes.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libpmgb.so and declare the ABI; raises PMLibraryError if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise PMLibraryError(f"{path} not built; run python -m paper_2211_09815_gb300.build")
    lib = ctypes.CDLL(path)
    vp, dp, i = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.pm_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PMConfig), dp, vp, vp]
    lib.pm_forward.argtypes = [vp, vp, vp, vp]
    lib.pm_loss_mse.argtypes = [vp, vp, vp, vp]
    lib.pm_adjoint.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.pm_destroy.argtypes = [vp]
    lib.pm_status_string.argtypes = [i]
    lib.pm_status_string.restype = ctypes.c_char_p
    lib.pm_last_cuda_error.restype = ctypes.c_char_p
    lib.pm_scratch_bytes.argtypes = [vp]
    lib.pm_scratch_bytes.restype = ctypes.c_longlong
    lib.pm_op_density.argtypes = [vp, vp, vp]
    lib.pm_op_force.argtypes = [vp, vp, vp]
    lib.pm_op_force_vjp.argtypes = [vp, vp, vp, vp, vp]
    lib.pm_op_fft.argtypes = [vp, i, vp, vp]
    lib.pm_op_za.argtypes = [vp, vp]
    lib.pm_op_ic.argtypes = [vp, vp, vp]
    lib.pm_loss_power.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.pm_set_snapshots.argtypes = [vp, i, ctypes.POINTER(ctypes.c_int), vp, vp, vp, vp]
    lib.pm_set_inputs.argtypes = [vp, dp, vp]
    lib.pm_gradient.argtypes = [vp, vp, vp, vp, vp, vp]
    lib.pm_profile.argtypes = [vp, i]
    lib.pm_profile_read.argtypes = [vp, vp, vp]
    lib.pm_density_noalloc.argtypes = [ctypes.c_double, i, i, vp, vp, vp]
    lib.pm_power_spectrum.argtypes = [vp, vp, vp, vp, vp]
    lib.pm_gradient_graph.argtypes = [vp, vp, vp, vp, vp]
    lib.pm_get_tuning.argtypes = [vp, ctypes.POINTER(PMTuning)]
    lib.pm_set_tuning.argtypes = [vp, ctypes.POINTER(PMTuning)]
    lib.pm_autotune.argtypes = [vp, i, ctypes.POINTER(PMTuning), vp]
    lib.pm_check.argtypes = [vp]
    lib.pm_set_snapshot_momenta.argtypes = [vp, vp, vp]
    lib.pm_get_fixed_state.argtypes = [vp, vp, vp]
    lib.pm_set_interp_snapshots.argtypes = [vp, i, dp, vp, vp, vp, vp]
    lib.pm_debug_fail_alloc.argtypes = [ctypes.c_longlong]
    lib.pm_debug_live_bytes.argtypes = []
    lib.pm_debug_live_bytes.restype = ctypes.c_longlong
    lib.pm_debug_first_wait.argtypes = [vp, i]
    for name in SYMBOLS:
        getattr(lib, name).restype = getattr(lib, name).restype or ctypes.c_int
    _lib = lib
    return lib


def _check(status, where):
    if status != 0:
        lib = load_library()
        raise PMError(status, where, lib.pm_last_cuda_error().decode() if status == 3 else "")


def _ptr(t, dtype=None, numel=None, name="tensor", device=None):
    """Device pointer of a contiguous CUDA tensor after checking dtype, size and device
    (``device``: the CUDA device index the library launches on; default: the current one)."""
    if t is None:
        return None
    import torch
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    dev = torch.cuda.current_device() if device is None else device
    if t.device.index != dev:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the library launches on cuda:{dev}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


def density_noalloc(box, n_mesh, n_ptcl, disp, dens_out, stream=None):
    """CIC overdensity with no device allocation (pm_density_noalloc), for callers that
    cannot call cudaMalloc; float32 only, n_mesh**3 <= NOALLOC_MAX_CELLS.  The library
    reuses one fixed device array for every call: do not run two calls concurrently on
    one GPU."""
    import torch
    if n_mesh ** 3 > NOALLOC_MAX_CELLS:
        raise ValueError(f"n_mesh**3 = {n_mesh ** 3} exceeds the allocation-free limit {NOALLOC_MAX_CELLS}")
    st = stream if stream is not None else torch.cuda.current_stream()
    dev = st.device.index
    if dev != torch.cuda.current_device():
        raise ValueError(f"the stream is on cuda:{dev}; make that device current first")
    _check(load_library().pm_density_noalloc(float(box), int(n_mesh), int(n_ptcl),
                                             _ptr(disp, torch.float32, 3 * n_ptcl ** 3, "disp", dev),
                                             _ptr(dens_out, torch.float32, n_mesh ** 3, "dens_out", dev),
                                             ctypes.c_void_p(st.cuda_stream)), "pm_density_noalloc")


class PMContext:
    """One simulation context (owns the library's device scratch).

    omega: CUDA tensor [batch, n_ptcl, n_ptcl, n_ptcl] (float32 or float64 per precision);
    theta: host sequence of shape [batch, 5] (A_s, n_s, Omega_m, Omega_b, h);
    lpt_order: 1 for Zel'dovich initial conditions, 2 for 2LPT.
    fixed_state: the exactly reversible 64-bit integer particle state.
    half_force: FP16 force meshes between the C2R x passes and the gathers (FP32 only).
    check_errors: after every call that launches work, synchronise the stream and raise
    PMError(PM_ERR_TIMEOUT) if a bounded device wait gave up (pm_check).
    ``state_version`` counts the calls that replace the context's forward state.
    """

    def __init__(self, box, n_mesh, n_ptcl, n_steps, theta, omega, a0=1.0 / 64, a1=1.0,
                 precision=PM_F32, ckpt_every=0, deconv=False, batch=1, stream=None, lpt_order=1,
                 check_errors=True, fixed_state=False, half_force=False):
        import torch
        lib = load_library()
        self.check_errors = check_errors
        self.state_version = 0
        self.device = torch.cuda.current_device()
        self.cfg = PMConfig(box, n_mesh, n_ptcl, n_steps, a0, a1, precision, ckpt_every, int(deconv), batch,
                            int(lpt_order), int(fixed_state), int(half_force))
        self.dtype = torch.float32 if precision == PM_F32 else torch.float64
        self.batch, self.n_mesh, self.n_ptcl = batch, n_mesh, n_ptcl
        self.N, self.M = n_ptcl ** 3, n_mesh ** 3
        th = [float(v) for row in (theta if hasattr(theta[0], "__len__") else [theta]) for v in row]
        if len(th) != 5 * batch:
            raise ValueError("theta must have batch x 5 values")
        arr = (ctypes.c_double * len(th))(*th)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if self.stream.device.index != self.device:
            raise ValueError("the stream must belong to the current device")
        self._h = ctypes.c_void_p()
        _check(lib.pm_init(ctypes.byref(self._h), ctypes.byref(self.cfg), arr,
                           self._p(omega, batch * self.N, "omega"),
                           ctypes.c_void_p(self.stream.cuda_stream)), "pm_init")

    def close(self):
        if self._h:
            load_library().pm_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _p(self, t, numel=None, name="tensor", dtype="ctx"):
        return _ptr(t, self.dtype if dtype == "ctx" else dtype, numel, name, self.device)

    def _run(self, status, where, replaces_state=True):
        """Raise on an error status; then, with check_errors, pm_check (synchronises)."""
        if replaces_state:
            self.state_version += 1
        _check(status, where)
        if self.check_errors:
            _check(load_library().pm_check(self._h), where + " (pm_check)")

    def check(self):
        """pm_check: synchronise and raise PMError(PM_ERR_TIMEOUT) if a device wait gave up."""
        _check(load_library().pm_check(self._h), "pm_check")

    def _new(self, *shape, dtype=None):
        import torch
        return torch.empty(*shape, device="cuda", dtype=dtype or self.dtype)

    def forward(self, disp=None, mom=None, dens=None):
        v = 3 * self.batch * self.N
        self._run(load_library().pm_forward(self._h, self._p(disp, v, "disp"), self._p(mom, v, "mom"),
                                            self._p(dens, self.batch * self.M, "dens")), "pm_forward")

    def loss_mse(self, target, djdd, loss=None):
        """loss: optional host float64 tensor [batch] or CUDA float64 tensor."""
        import torch
        out = loss if loss is not None else torch.zeros(self.batch, dtype=torch.float64)
        _check(load_library().pm_loss_mse(self._h, self._p(target, self.batch * self.M, "target"),
                                          ctypes.c_void_p(out.data_ptr()),
                                          self._p(djdd, self.batch * self.M, "djdd")), "pm_loss_mse")
        return out

    def adjoint(self, djdd=None, djdx=None, djdp=None, grad_omega=None, grad_theta=None):
        v = 3 * self.batch * self.N
        gt = ctypes.c_void_p(grad_theta.data_ptr()) if grad_theta is not None else None
        self._run(load_library().pm_adjoint(self._h, self._p(djdd, self.batch * self.M, "djdd"),
                                            self._p(djdx, v, "djdx"), self._p(djdp, v, "djdp"),
                                            self._p(grad_omega, self.batch * self.N, "grad_omega"), gt),
                  "pm_adjoint")

    def op_density(self, disp, dens):
        self._run(load_library().pm_op_density(self._h, self._p(disp, 3 * self.batch * self.N, "disp"),
                                               self._p(dens, self.batch * self.M, "dens")), "pm_op_density")

    def op_force(self, disp, acc):
        v = 3 * self.batch * self.N
        self._run(load_library().pm_op_force(self._h, self._p(disp, v, "disp"), self._p(acc, v, "acc")),
                  "pm_op_force")

    def op_force_vjp(self, disp, pi, acc, alpha):
        v = 3 * self.batch * self.N
        self._run(load_library().pm_op_force_vjp(self._h, self._p(disp, v, "disp"), self._p(pi, v, "pi"),
                                                 self._p(acc, v, "acc"), self._p(alpha, v, "alpha")),
                  "pm_op_force_vjp")

    def op_fft(self, direction, inp, out):
        self._run(load_library().pm_op_fft(self._h, int(direction), self._p(inp, name="inp", dtype=None),
                                           self._p(out, name="out", dtype=None)), "pm_op_fft")

    def op_za(self, s1):
        self._run(load_library().pm_op_za(self._h, self._p(s1, 3 * self.batch * self.N, "s1")), "pm_op_za")

    def set_snapshots(self, steps, disp=None, dens=None, ddisp=None, ddens=None):
        """Observe the states after the given steps (ascending, 0..n_steps): each forward
        writes s_j into disp[q] and delta_j into dens[q]; each adjoint adds the cotangents
        ddisp[q] (dJ/dx_j) and ddens[q] (dJ/d delta_j).  Buffers: CUDA tensors of
        len(steps) x batch x (3 N or M) elements, kept referenced here while in use."""
        steps = [int(j) for j in steps]
        ns = len(steps)
        v, m = ns * 3 * self.batch * self.N, ns * self.batch * self.M
        arr = (ctypes.c_int * max(ns, 1))(*steps)
        _check(load_library().pm_set_snapshots(self._h, ns, arr, self._p(disp, v, "disp"),
                                               self._p(dens, m, "dens"), self._p(ddisp, v, "ddisp"),
                                               self._p(ddens, m, "ddens")), "pm_set_snapshots")
        self._snapshot_buffers = (disp, dens, ddisp, ddens) if ns else None
        self._snapshot_steps = steps
        self._snapshot_momenta = None

    def set_snapshot_momenta(self, mom=None, dmom=None):
        """Momenta p_j of the snapshot steps: each forward writes them into mom[q], each
        adjoint adds the cotangents dmom[q] (CUDA tensors of len(steps) x batch x 3 N)."""
        ns = len(self._snapshot_steps)
        v = ns * 3 * self.batch * self.N
        _check(load_library().pm_set_snapshot_momenta(self._h, self._p(mom, v, "mom"), self._p(dmom, v, "dmom")),
               "pm_set_snapshot_momenta")
        self._snapshot_momenta = (mom, dmom)

    def set_interp_snapshots(self, a_values, disp=None, dens=None, ddisp=None, ddens=None):
        """Positions at scale factors between steps (ascending, in (a0, a1]): each forward
        writes s(a_q) into disp[q] and delta(a_q) into dens[q]; each adjoint adds the
        cotangents ddisp[q], ddens[q].  Buffers: CUDA tensors of len(a_values) x batch x
        (3 N or M) elements, kept referenced here while in use."""
        import numpy as np
        a = np.ascontiguousarray(np.asarray(a_values, dtype=np.float64).ravel())
        na = a.size
        v, m = na * 3 * self.batch * self.N, na * self.batch * self.M
        _check(load_library().pm_set_interp_snapshots(
            self._h, na, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self._p(disp, v, "disp"),
            self._p(dens, m, "dens"), self._p(ddisp, v, "ddisp"), self._p(ddens, m, "ddens")),
            "pm_set_interp_snapshots")
        self._interp_buffers = (disp, dens, ddisp, ddens) if na else None

    def get_fixed_state(self, disp_fixed=None, mom_fixed=None):
        """The 64-bit fixed-point state (contexts with fixed_state=True) into int64 CUDA
        tensors of batch x 3 N elements."""
        import torch
        v = 3 * self.batch * self.N
        self._run(load_library().pm_get_fixed_state(self._h, self._p(disp_fixed, v, "disp_fixed", torch.int64),
                                                    self._p(mom_fixed, v, "mom_fixed", torch.int64)),
                  "pm_get_fixed_state", False)

    def op_ic(self, s0=None, p0=None):
        """Initial state (s0, p0) at a0 of the context's LPT order."""
        v = 3 * self.batch * self.N
        self._run(load_library().pm_op_ic(self._h, self._p(s0, v, "s0"), self._p(p0, v, "p0")), "pm_op_ic")

    def set_inputs(self, theta=None, omega=None):
        """theta: host [batch][5] or None; omega: host (pinned) or CUDA tensor or None."""
        lib = load_library()
        arr = None
        if theta is not None:
            th = [float(v) for row in (theta if hasattr(theta[0], "__len__") else [theta]) for v in row]
            arr = (ctypes.c_double * len(th))(*th)
        if omega is not None and omega.is_cuda and omega.device.index != self.device:
            raise ValueError(f"omega is on cuda:{omega.device.index}, the context on cuda:{self.device}")
        om = ctypes.c_void_p(omega.data_ptr()) if omega is not None else None
        self._run(lib.pm_set_inputs(self._h, arr, om), "pm_set_inputs")

    def gradient(self, target, omega=None, loss=None, grad_omega=None, grad_theta=None):
        """All arguments are torch tensors on the host (pinned) or the device."""
        def p(t):
            if t is not None and t.is_cuda and t.device.index != self.device:
                raise ValueError(f"a tensor is on cuda:{t.device.index}, the context on cuda:{self.device}")
            return ctypes.c_void_p(t.data_ptr()) if t is not None else None
        self._run(load_library().pm_gradient(self._h, p(omega), p(target), p(loss), p(grad_omega), p(grad_theta)),
                  "pm_gradient")

    def gradient_graph(self, target, loss=None, grad_omega=None, grad_theta=None):
        """pm_gradient_graph: device tensors only; needs a non-default stream."""
        def p(t, name):
            return self._p(t, name=name, dtype=None)
        self._run(load_library().pm_gradient_graph(self._h, p(target, "target"), p(loss, "loss"),
                                                   p(grad_omega, "grad_omega"), p(grad_theta, "grad_theta")),
                  "pm_gradient_graph")

    def power_spectrum(self, dens=None):
        """(kmean [n/2], P [batch, n/2], nmodes [n/2]) as float64 numpy arrays."""
        import numpy as np
        nb = self.n_mesh // 2
        pk = np.zeros((self.batch, nb))
        km = np.zeros(nb)
        nm = np.zeros(nb)
        f = ctypes.POINTER(ctypes.c_double)
        _check(load_library().pm_power_spectrum(self._h, self._p(dens, self.batch * self.M, "dens"),
                                                pk.ctypes.data_as(f), km.ctypes.data_as(f), nm.ctypes.data_as(f)),
               "pm_power_spectrum")
        return km, pk, nm

    def loss_power(self, pk_target, weights, djdd, dens=None):
        """Objective sum_b w_b (P_b - T_b)^2 on the shell power of ``dens`` (the last forward
        density when None) and its cotangent into ``djdd``; pk_target, weights: host
        arrays [batch, n_mesh/2].  Returns the per-instance loss (float64 numpy)."""
        import numpy as np
        nb = self.n_mesh // 2
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(pk_target, dtype=np.float64), (self.batch, nb)))
        w = np.ascontiguousarray(np.broadcast_to(np.asarray(weights, dtype=np.float64), (self.batch, nb)))
        loss = np.zeros(self.batch)
        f = ctypes.POINTER(ctypes.c_double)
        _check(load_library().pm_loss_power(self._h, self._p(dens, self.batch * self.M, "dens"),
                                            t.ctypes.data_as(f), w.ctypes.data_as(f), loss.ctypes.data_as(f),
                                            self._p(djdd, self.batch * self.M, "djdd")), "pm_loss_power")
        return loss

    def profile(self, enable=True):
        _check(load_library().pm_profile(self._h, int(enable)), "pm_profile")

    def profile_read(self):
        """{category: (milliseconds, kernel launches)} accumulated since the last read."""
        ms = (ctypes.c_double * len(PROF_NAMES))()
        n = (ctypes.c_longlong * len(PROF_NAMES))()
        _check(load_library().pm_profile_read(self._h, ms, n), "pm_profile_read")
        return {name: (ms[i], n[i]) for i, name in enumerate(PROF_NAMES)}

    def get_tuning(self):
        t = PMTuning()
        _check(load_library().pm_get_tuning(self._h, ctypes.byref(t)), "pm_get_tuning")
        return t.as_dict()

    def set_tuning(self, tuning):
        """tuning: dict with the fields of PMTuning (missing fields keep their value)."""
        t = PMTuning()
        _check(load_library().pm_get_tuning(self._h, ctypes.byref(t)), "pm_get_tuning")
        for k, v in tuning.items():
            if k.startswith("tile_log2"):
                getattr(t, k)[:] = list(v)
            else:
                setattr(t, k, int(v))
        _check(load_library().pm_set_tuning(self._h, ctypes.byref(t)), "pm_set_tuning")

    def autotune(self, reps=3):
        """Time the candidate launch shapes on the current state and keep the fastest;
        returns (chosen tuning dict, [best forward deposit, adjoint deposit, y pass] ms)."""
        t = PMTuning()
        ms = (ctypes.c_double * 3)()
        self._run(load_library().pm_autotune(self._h, int(reps), ctypes.byref(t), ms), "pm_autotune", False)
        return t.as_dict(), list(ms)

    @property
    def scratch_bytes(self):
        return load_library().pm_scratch_bytes(self._h)
