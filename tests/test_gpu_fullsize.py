"""Parity at the full sizes of the named workloads, in the launch configuration
the benchmark times.

The oracle cannot run 128^3 x 2000 or 512^3 lattices in seconds, so these tests
(a) check properties that hold at any size over the full run (mass
conservation, no non-finite values), and (b) compare short continuations: the
GPU state at a late time is read back, and the oracle advances it (the whole
128^3 lattice, or a sub-block whose light cone stays inside it) by a few steps;
the GPU's own continuation must agree element by element.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def olb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11752_gb300 import build, olb as _olb
    build.build()
    _olb.load()
    return _olb


def _cavity(olb, torch, dtype, scheme, n=128):
    m = I.cavity(n)
    lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype=dtype, scheme=scheme)
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 0)
    lat.set_wall_velocity(I.LID, (0.05, 0.0, 0.0))
    tau = I.cavity_tau(n, 400.0, 0.05)
    lat.set_bgk(tau)
    lat.init_equilibrium()
    lat.perturb(torch.from_numpy(I.population_noise(1, 19, m, 1e-6).reshape(-1)).cuda())
    return lat, m, tau


@pytest.mark.parametrize("dtype,scheme,tol", [("f32", "pull", 1e-5), ("f32", "aa", 1e-5),
                                              ("f64", "pull", 1e-12)])
def test_cavity128_full_run(oracle, olb, dtype, scheme, tol):
    import torch

    lat, m, tau = _cavity(olb, torch, dtype, scheme)
    d0 = lat.diagnostics()
    stats = lat.step_stats(2000)
    d1 = lat.diagnostics()
    assert stats[6] == 0 and d1[6] == 0
    # mass: exact in exact arithmetic (halfway walls, lid with matching edge links)
    assert abs(d1[0] - d0[0]) <= (1e-12 if dtype == "f64" else 2e-6) * d0[0]
    assert 0.01 < d1[5] < 0.06  # the lid drives a flow slower than the lid
    # continuation: oracle advances the GPU state by 2 steps on the whole lattice
    f = np.ascontiguousarray(lat.get_populations().cpu().numpy())
    wu = np.zeros((256, 3))
    wu[I.LID] = (0.05, 0, 0)
    ref = oracle.Lattice(oracle.D3Q19, m, tau, periodic=0, wall_u=wu)
    ref.step(f, 2)
    lat.step(2)
    fg = lat.get_populations().cpu().numpy()
    assert rel_err(fg, f, m == I.FLUID) <= tol
    lat.close()


def _block(t, lo, size, dims):
    """Sub-block [lo, lo + size) of a [q, nz, ny, nx] CUDA tensor, wrapping periodic
    dims (index lists taken modulo the extent)."""
    import torch

    out = t
    for axis, (start, n, ext) in enumerate(zip(lo, size, dims)):
        idx = torch.arange(start, start + n, device=t.device) % ext
        out = out.index_select(axis + 1, idx)
    return out.cpu().numpy()


@pytest.mark.parametrize("dtype,tol", [("f32", 1e-5), ("f16", 2e-3)])
def test_tgv512_block_continuation(oracle, olb, dtype, tol):
    """512^3 periodic vortex: after 30 steps, a 24^3 block straddling the periodic
    corner is advanced 4 steps by the oracle; its inner 16^3 cells (outside the
    reach of the block's artificial edges) must match the GPU continuation."""
    import torch

    n, k, b = 512, 4, 24
    lat = olb.Lattice(olb.D3Q19, (n, n, n), dtype=dtype, scheme="pull")
    lat.set_material(torch.ones(n ** 3, dtype=torch.uint8, device="cuda"), 7)
    lat.set_bgk(0.6)
    rho, u = I.tgv3d(n, 0.02, xp=torch, device="cuda")
    lat.init_equilibrium(rho.reshape(-1), u.reshape(-1))
    del rho, u
    lat.step(30)
    lo = (n - b // 2, n - b // 2, n - b // 2)
    f0 = np.ascontiguousarray(_block(lat.get_populations(), lo, (b, b, b), (n, n, n)))
    torch.cuda.empty_cache()
    lat.step(k)
    f1 = _block(lat.get_populations(), lo, (b, b, b), (n, n, n))
    lat.close()
    torch.cuda.empty_cache()
    ref = oracle.Lattice(oracle.D3Q19, I.periodic_box(b, b, b), 0.6, periodic=0)
    ref.step(f0, k)
    inner = (slice(None),) + (slice(k, b - k),) * 3
    # errors are measured against the deviation from rest f - w, the part that
    # the shifted storage holds (16 bits: one rounding of it per step)
    w = np.array([1 / 3] + [1 / 18] * 3 + [1 / 36] * 6 + [1 / 18] * 3 + [1 / 36] * 6)[:, None, None, None]
    err = np.max(np.abs(f1[inner] - f0[inner])) / np.max(np.abs(f0[inner] - w))
    assert err <= tol, err


def test_channel_384_block_continuation_f16(oracle, olb):
    """The adjoint-at-scale channel (384 x 192 x 192, porosity, force, walls on
    y and z, periodic x) in FP16 storage: a 20^3 block at a wall corner, straddling
    the periodic x boundary, advanced 3 steps by the oracle."""
    import torch

    nx, ny, nz = 384, 192, 192
    m = I.channel(nx, ny, nz)
    gamma = I.smoothed_porosity(2, m)
    tau = 0.8
    F = (I.channel_force(ny, tau), 0.0, 0.0)
    lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype="f16", scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    lat.set_bgk(tau)
    lat.set_force(F)
    lat.set_porosity(torch.from_numpy(gamma.reshape(-1).copy()).cuda())
    lat.init_equilibrium()
    lat.step(40)
    k, b = 3, 20
    lo = (0, 0, nx - b // 2)  # z, y, x
    f0 = np.ascontiguousarray(_block(lat.get_populations(), lo, (b, b, b), (nz, ny, nx)))
    lat.step(k)
    f1 = _block(lat.get_populations(), lo, (b, b, b), (nz, ny, nx))
    lat.close()
    torch.cuda.empty_cache()
    zi = np.arange(lo[0], lo[0] + b) % nz
    yi = np.arange(lo[1], lo[1] + b) % ny
    xi = np.arange(lo[2], lo[2] + b) % nx
    mb = m[np.ix_(zi, yi, xi)]
    gb = gamma[np.ix_(zi, yi, xi)]
    ref = oracle.Lattice(oracle.D3Q19, mb, tau, periodic=0, force=F, gamma=gb)
    ref.step(f0, k)
    # inner region: k cells from the artificial faces (z = b, y = b, x = 0, x = b)
    inner = (slice(None), slice(0, b - k), slice(0, b - k), slice(k, b - k))
    fl = mb[inner[1:]] == I.FLUID
    w = np.array([1 / 3] + [1 / 18] * 3 + [1 / 36] * 6 + [1 / 18] * 3 + [1 / 36] * 6)[:, None, None, None]
    dev = np.max(np.abs((f0 - w)[inner][:, fl]))
    err = np.max(np.abs(f1[inner][:, fl] - f0[inner][:, fl])) / dev
    assert err <= 2e-3, err


def test_adjoint_channel256_per_cell_against_differences(olb):
    """FP32- and FP64-storage adjoints on the 256 x 128 x 128 porous channel (300
    steps, K = 50) against central differences of FP64 GPU forward runs at 8 seeded
    fluid cells and tau, per cell and with no absolute slack: FP64 within 1e-5 (the resolution of the
    differences at the smallest sampled gradient), FP32
    within 1e-4 relative.  The gradients are 1e-13 .. 1e-11 against a loss of ~4e-6,
    so the step is h = 1e-3 (at 1e-5 the two losses share all but their last few
    digits), and the quotients at h and h/2 are combined by Richardson extrapolation,
    (4 D(h/2) - D(h)) / 3, which removes their h^2 truncation term (about 1e-6
    relative at h = 1e-3)."""
    import torch

    nx, ny, nz = 256, 128, 128
    m = I.channel(nx, ny, nz)
    gamma = I.smoothed_porosity(2, m)
    tau = 0.8
    F = (I.channel_force(ny, tau), 0.0, 0.0)
    steps, K = 300, 50
    obj = (0, nx - 1, 0)
    # FP64: 1e-5, the differences' own resolution at the smallest sampled gradient
    # (rounding noise ~ eps |L| / (h |dL/dgamma|) = 1e-16 * 4e-6 / (5e-4 * 1.6e-13) ~ 5e-6)

    def lattice(dt):
        lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype=dt, scheme="pull")
        lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
        lat.set_force(F)
        return lat

    grads = {}
    for dt in ("f32", "f64"):
        lat = lattice(dt)
        lat.set_bgk(tau)
        lat.set_porosity(torch.from_numpy(gamma.reshape(-1).copy()).cuda())
        lat.init_equilibrium()
        loss, dg, dtau = lat.adjoint_run(steps, K, obj)
        grads[dt] = (dg.cpu().numpy().reshape(-1), dtau)
        lat.close()
        del dg
        torch.cuda.empty_cache()
    ref = lattice("f64")
    plane = torch.from_numpy(m[:, :, nx - 1] == I.FLUID).cuda()

    def run(gam, t):
        ref.set_bgk(t)
        ref.set_porosity(torch.from_numpy(gam.reshape(-1).copy()).cuda())
        ref.init_equilibrium()
        ref.step(steps)
        _, u = ref.moments()
        return float(u[0, :, :, nx - 1][plane].mean())

    def quotient(c, h):
        gp = gamma.copy().reshape(-1)
        gm = gp.copy()
        gp[c] += h
        gm[c] -= h
        return (run(gp, tau) - run(gm, tau)) / (2 * h)

    h = 1e-3
    # cells the outlet plane's adjoint reaches within 300 steps (elsewhere the
    # gradient is below 1e-25 and a difference quotient of FP64 runs gives 0)
    near = m.copy()
    near[:, :, 40:nx - 60] = 0
    cells = I.random_fluid_cells(3, near, 8)
    fd = [(4 * quotient(c, h / 2) - quotient(c, h)) / 3 for c in cells]
    for c, d in zip(cells, fd):
        assert abs(grads["f64"][0][c] - d) <= 1e-5 * abs(d), (c, d, grads["f64"][0][c])
        assert abs(grads["f32"][0][c] - d) <= 1e-4 * abs(d), (c, d, grads["f32"][0][c])
    ht = 1e-6
    d = (run(gamma, tau + ht) - run(gamma, tau - ht)) / (2 * ht)
    assert abs(grads["f64"][1] - d) <= 1e-6 * abs(d)
    assert abs(grads["f32"][1] - d) <= 1e-4 * abs(d)
    ref.close()
