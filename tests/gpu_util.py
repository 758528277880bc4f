"""Helpers for the GPU parity tests: build/load the library, run oracle and CUDA side by
side on the same seeded inputs."""
import numpy as np

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def ensure_built():
    from paper_2211_09815_gb300 import build
    build.build()


def make_ctx(box, n_mesh, n_ptcl, n_steps, theta=inputs.THETA_FIDUCIAL, seed=1, precision=0, batch=1,
             ckpt_every=0, deconv=False, a0=1 / 64, a1=1.0, omega=None, lpt_order=1):
    torch = torch_cuda()
    ensure_built()
    from paper_2211_09815_gb300 import pm
    dt = torch.float32 if precision == 0 else torch.float64
    if omega is None:
        omega = np.stack([inputs.white_noise(n_ptcl, seed + b) for b in range(batch)])
    om = torch.from_numpy(np.ascontiguousarray(omega)).to(device="cuda", dtype=dt)
    th = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    if th.shape[0] == 1 and batch > 1:
        th = np.repeat(th, batch, axis=0)
    ctx = pm.PMContext(box, n_mesh, n_ptcl, n_steps, th.tolist(), om, a0=a0, a1=a1, precision=precision,
                       ckpt_every=ckpt_every, deconv=deconv, batch=batch, lpt_order=lpt_order)
    return ctx, om, omega, th


def oracle_cfg(box, n_mesh, n_ptcl, n_steps, deconv=False, a0=1 / 64, a1=1.0, lpt_order=1):
    return opm.PMConfig(box=box, n_mesh=n_mesh, n_ptcl=n_ptcl, n_steps=n_steps, deconv=deconv, a0=a0, a1=a1,
                        lpt_order=lpt_order)


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def cosine(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))


def same_cells_fp32(disp32, cfg):
    """Particles whose CIC cell the FP32 kernel arithmetic, floor(fma(s, n/L, 1/2)) added to
    the lattice index, and the oracle's FP64 floor(x / l) agree on along every axis.  The
    cell is an integer decided by floating point: a particle within FP32 rounding of a cell
    face lands on either side, and there the weight gradient of Eq. 10 (floor convention)
    jumps, so quantities built on it (alpha, dJ/dx) are compared on the other particles."""
    n, npc = cfg.n_mesh, cfg.n_ptcl
    j = np.indices((npc,) * 3).reshape(3, -1)
    inv_l32 = np.float32(n / cfg.box)
    # exact product of two FP32 values plus 1/2 in FP64, then one rounding to FP32: the fma
    v32 = (np.asarray(disp32, dtype=np.float32).astype(np.float64) * np.float64(inv_l32) + 0.5).astype(np.float32)
    c32 = (j * (n // npc) + np.floor(v32).astype(np.int64)) % n
    x = opm.lattice(cfg) + np.asarray(disp32, dtype=np.float32).astype(np.float64)
    c64 = np.floor(x / cfg.cell).astype(np.int64) % n
    return np.all(c32 == c64, axis=0)
