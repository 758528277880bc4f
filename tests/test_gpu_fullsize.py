"""Parity at the full size of the timed workload: 512^3 particles on a 1024^3 mesh in a
1 Gpc/h box, in the launch shapes the benchmark times (autotuned).

The FP64 oracle cannot deposit or transform a 1024^3 mesh in test time, so the density is
compared on sampled cells (direct CIC summation, `oracle.pm.density_at`), and the
transforms and the force through properties that hold at any size: mass conservation,
FFT round trip and Parseval, zero net force.  The displacement field is seeded and
synthetic: Gaussian displacements of 3 cells, and three blocks of 32^3 particles collapsed
onto their block centres, so that some mesh tiles receive over 3 x 10^4 particles.
"""
import numpy as np
import pytest

from oracle import pm as opm
from paper_2211_09815_gb300 import inputs

from gpu_util import make_ctx, oracle_cfg, torch_cuda

pytestmark = pytest.mark.gpu

BOX, NM, NP = 1000.0, 1024, 512


def _collapse_blocks():
    """Three seeded blocks of 32^3 Lagrangian particles (64^3 cells) collapsed onto their
    block centres: 32768 particles within about a cell, more than 2^16 particle visits in
    the mesh tiles there."""
    nb = NP // 32
    pick = (inputs.uniform01(49, 3) * nb ** 3).astype(np.int64)
    return [np.array([b // (nb * nb), (b // nb) % nb, b % nb]) for b in pick]


@pytest.fixture(scope="module")
def big():
    torch = torch_cuda()
    ctx, *_ = make_ctx(BOX, NM, NP, 1)
    ctx.autotune()
    N = NP ** 3
    cell = BOX / NM
    disp = np.empty((3, N), dtype=np.float32)
    for c in range(3):
        disp[c] = 3.0 * cell * inputs.white_noise(NP, 41 + c).ravel()
    cfg = oracle_cfg(BOX, NM, NP, 1)
    q = opm.lattice(cfg)
    j = np.indices((NP,) * 3).reshape(3, -1)
    centres = []
    for k, blk in enumerate(_collapse_blocks()):
        inside = np.all(j // 32 == blk[:, None], axis=0)
        centre = (blk * 32 + 16) * (BOX / NP)
        centres.append(centre)
        noise = 0.3 * cell * np.stack([inputs.white_noise(32, 60 + 3 * k + c).ravel() for c in range(3)])
        disp[:, inside] = (centre[:, None] - q[:, inside] + noise).astype(np.float32)
    d = torch.from_numpy(disp).to("cuda").contiguous()
    yield ctx, d, disp, q, cfg, centres
    ctx.close()


def test_fullsize_density_on_sampled_cells_and_mass(big):
    torch = torch_cuda()
    ctx, d, disp, q, cfg, centres = big
    dens = torch.empty(NM ** 3, device="cuda")
    ctx.op_density(d, dens)
    rng = np.random.default_rng(3)
    cells = list(rng.choice(NM ** 3, size=512, replace=False))
    cell = BOX / NM
    for centre in centres:   # the cells around each collapse point
        c0 = np.floor(centre / cell).astype(np.int64)
        for off in np.ndindex(4, 4, 4):
            g = (c0 + np.array(off) - 2) % NM
            cells.append((g[0] * NM + g[1]) * NM + g[2])
    cells = np.unique(np.array(cells, dtype=np.int64))
    got = dens[torch.from_numpy(cells).cuda()].cpu().numpy().astype(np.float64)
    ref = opm.density_at(q + disp.astype(np.float64), cfg, cells)
    # exact fixed-point sums of FP32 weights: the weights' FP32 rounding (fractions of
    # displacements up to ~50 cells) bounds the difference
    assert np.all(np.abs(got - ref) <= 2e-5 * np.abs(ref + 1.0) + 1e-5)
    assert ref.max() > 1e3   # the collapse points were sampled
    # mass conservation over the whole mesh
    tot = float((dens.double() + 1.0).sum())
    assert abs(tot - NM ** 3) <= 1e-6 * NM ** 3


def test_fullsize_fft_round_trip_and_parseval(big):
    torch = torch_cuda()
    ctx = big[0]
    gen = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(NM, NM, NM, device="cuda", generator=gen)
    spec = torch.empty(NM, NM, NM // 2 + 1, 2, device="cuda")
    ctx.op_fft(-1, x, spec)
    p = spec.double().pow(2).sum(-1)
    w = torch.full((NM // 2 + 1,), 2.0, device="cuda", dtype=torch.float64)
    w[0] = 1.0
    w[-1] = 1.0
    parseval = float((p * w).sum()) / NM ** 3
    assert abs(parseval / float(x.double().pow(2).sum()) - 1.0) < 1e-5
    del p
    back = torch.empty_like(x)
    ctx.op_fft(+1, spec, back)
    err = float((back / NM ** 3 - x).abs().max() / x.abs().max())
    assert err < 2e-6 * np.log2(NM ** 3)


def test_fullsize_zero_net_force(big):
    torch = torch_cuda()
    ctx, d = big[0], big[1]
    acc = torch.empty(3 * NP ** 3, device="cuda")
    ctx.op_force(d, acc)
    a = acc.view(3, -1).double()
    net = a.sum(dim=1).abs()
    scale = a.abs().sum(dim=1)
    assert bool(torch.all(net <= 1e-4 * scale))


def _exact_dft_modes(x_dev, kz, ky, kx, chunk=32):
    """The unnormalised forward DFT X[kz, ky, kx] = sum x[z, y, x] exp(-2 pi i (kz z + ky y
    + kx x) / n) of a real n^3 mesh at the outer product of the sampled frequency sets,
    written out as three separable contractions in float64 on the host (the mesh is
    streamed from the device in z slabs).  Phases use the exact integer residue of k x
    modulo n."""
    n = x_dev.shape[0]
    idx = np.arange(n)

    def phases(ks):
        m = (np.outer(idx, np.asarray(ks)) % n).astype(np.float64)
        return np.exp(-2j * np.pi * m / n)          # [n, K]

    ex, ey, ez = phases(kx), phases(ky), phases(kz)
    out = np.zeros((len(kz), len(ky), len(kx)), dtype=np.complex128)
    for z0 in range(0, n, chunk):
        xc = x_dev[z0:z0 + chunk].cpu().numpy().astype(np.float64).reshape(-1, n)
        a = (xc @ ex.real + 1j * (xc @ ex.imag)).reshape(chunk, n, len(kx))    # sum over x
        b = np.einsum("zyk,yl->zlk", a, ey)                                     # sum over y
        out += np.einsum("zlk,zm->mlk", b, ez[z0:z0 + chunk])                   # sum over z
    return out


def test_fullsize_fft_r2c_matches_exact_dft_on_sampled_modes(big):
    """The 1024^3 R2C in the instances the benchmark times (x pass of 512 complex points,
    TMA-staged y and z column passes of 1024) against the exact DFT, element by element on
    12 x 12 x 12 sampled modes: the zero and Nyquist planes of every axis (the x Nyquist
    plane is the separately stored side plane), their neighbours and seeded random
    frequencies.  Tolerance as for the smaller transforms, 2e-6 log2(n^3) of the largest
    sampled amplitude."""
    torch = torch_cuda()
    ctx = big[0]
    gen = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(NM, NM, NM, device="cuda", generator=gen)
    spec = torch.empty(NM, NM, NM // 2 + 1, 2, device="cuda")
    ctx.op_fft(-1, x, spec)
    rng = np.random.default_rng(11)
    full = [0, 1, NM // 2 - 1, NM // 2, NM // 2 + 1, NM - 1]
    kz = np.array(full + list(rng.choice(np.arange(2, NM - 2), 6, replace=False)))
    ky = np.array(full + list(rng.choice(np.arange(2, NM - 2), 6, replace=False)))
    kx = np.array([0, 1, 2, NM // 2 - 1, NM // 2] + list(rng.choice(np.arange(3, NM // 2 - 1), 7, replace=False)))
    ref = _exact_dft_modes(x, kz, ky, kx)
    sel = spec[torch.from_numpy(kz).cuda()][:, torch.from_numpy(ky).cuda()][:, :, torch.from_numpy(kx).cuda()]
    got = sel.double().cpu().numpy()
    got = got[..., 0] + 1j * got[..., 1]
    tol = 2e-6 * np.log2(NM ** 3)
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))
