"""GPU parity of the advection-diffusion lattice (olb_ade_*, D2Q5 / D3Q7 BGK with
the first-order equilibrium) against the oracle's: the scalar C within 1e-13
(FP64) and 1e-5 (FP32) relative after 60 steps, uniform and per-cell velocity,
sizes that are not multiples of the thread block; conservation; argument errors."""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

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


def _velocity(desc, shape, field):
    nz, ny, nx = shape
    if not field:
        return np.array([0.05, -0.03, 0.02 if desc == 3 else 0.0])
    v = 0.1 * (I.uniform(21, (3, nz, ny, nx)) - 0.5)
    if desc == 2:
        v[2] = 0.0
    return np.ascontiguousarray(v)


@pytest.mark.parametrize("desc,dims", [(2, (37, 29, 1)), (3, (21, 17, 13))])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
@pytest.mark.parametrize("field", [False, True])
def test_ade_matches_oracle(oracle, olb, desc, dims, dtype, tol, field):
    import torch

    nx, ny, nz = dims
    shape = (nz, ny, nx)
    tau, steps = 0.74, 60
    C0 = np.ascontiguousarray(1.0 + 0.5 * I.uniform(22, shape))
    v = _velocity(desc, shape, field)
    lat_o = oracle.AdeLattice(0 if desc == 2 else 1, shape, tau, v)
    g = lat_o.init(C0)
    lat_o.step(g, steps)
    Co = lat_o.density(g)
    a = olb.AdeLattice(desc, dims, dtype)
    a.set_tau(tau)
    if field:
        a.set_velocity(field=torch.from_numpy(v).cuda())
    else:
        a.set_velocity(v)
    a.init(torch.from_numpy(C0).cuda())
    a.step(steps)
    Cg = a.density().cpu().numpy()
    a.close()
    assert np.max(np.abs(Cg - Co)) <= tol * np.max(np.abs(Co))


def test_ade_host_arrays_and_conservation(olb):
    dims = (16, 12, 10)
    shape = (10, 12, 16)
    a = olb.AdeLattice(3, dims, "f64")
    a.set_tau(0.9)
    a.set_velocity((0.04, 0.01, -0.02))
    C0 = np.ascontiguousarray(1.0 + I.uniform(23, shape))
    a.init(C0)
    a.step(101)
    out = np.zeros(shape)
    a.density(out)
    assert abs(out.sum() - C0.sum()) <= 1e-13 * C0.sum()
    a.close()


def test_ade_rejects_bad_arguments(olb):
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(0, (8, 8, 1))          # a fluid descriptor
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(2, (8, 8, 2))          # D2Q5 with nz > 1
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(3, (8, 8, 8), "f16")   # 16-bit storage is not offered here
    a = olb.AdeLattice(3, (8, 8, 8))
    with pytest.raises(olb.OlbError):
        a.set_tau(0.5)
    with pytest.raises(olb.OlbError):
        a.set_velocity()
    a.close()


# ---------------------------------------------------------------------------------
# Boundaries: no-flux walls (bounce-back), Dirichlet cells (anti-bounce-back),
# non-periodic domain edges; and the velocity taken from a fluid lattice.
# ---------------------------------------------------------------------------------
def _mixed_material(desc, shape, seed):
    """Bulk cells with scattered no-flux (0) and Dirichlet (2, 3, 4) cells."""
    r = I.uniform(seed, shape)
    m = np.ones(shape, np.uint8)
    m[r < 0.06] = 0
    m[(r >= 0.06) & (r < 0.09)] = 2
    m[(r >= 0.09) & (r < 0.11)] = 3
    m[(r >= 0.11) & (r < 0.12)] = 4
    return m


@pytest.mark.parametrize("desc,dims,periodic", [(2, (37, 29, 1), 1), (3, (21, 17, 13), 5), (3, (16, 15, 12), 0)])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
def test_ade_boundaries_match_oracle(oracle, olb, desc, dims, periodic, dtype, tol):
    import torch

    nx, ny, nz = dims
    shape = (nz, ny, nx)
    tau, steps = 0.71, 70
    m = _mixed_material(desc, shape, 41)
    wall = np.zeros(256)
    wall[2], wall[3], wall[4] = 0.5, 2.0, 1.3
    v = _velocity(desc, shape, True)
    C0 = np.ascontiguousarray(np.where(m == 1, 1.0 + 0.5 * I.uniform(42, shape), 0.25))
    lat_o = oracle.AdeLattice(0 if desc == 2 else 1, shape, tau, v, material=m, wall_C=wall, periodic=periodic)
    g = lat_o.init(C0)
    lat_o.step(g, steps)
    Co = lat_o.density(g)
    a = olb.AdeLattice(desc, dims, dtype)
    a.set_tau(tau)
    a.set_velocity(field=torch.from_numpy(v).cuda())
    a.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), periodic, wall)
    a.init(torch.from_numpy(C0).cuda())
    a.step(steps)
    Cg = a.density().cpu().numpy()
    a.close()
    assert np.max(np.abs(Cg - Co)) <= tol * np.max(np.abs(Co))


@pytest.mark.parametrize("desc", [2, 3])
def test_ade_dirichlet_plates_exact_linear_profile(olb, desc):
    """Steady diffusion between two Dirichlet plates (C = 1 and 2): the straight
    line through the halfway walls, y = 1/2 and y = ny - 3/2, to round-off."""
    ny, n_par = 12, 4
    dims = (n_par, ny, 1) if desc == 2 else (n_par, ny, n_par)
    shape = dims[::-1]
    m = np.ones(shape, np.uint8)
    m[:, 0, :] = 2
    m[:, -1, :] = 3
    wall = np.zeros(256)
    wall[2], wall[3] = 1.0, 2.0
    a = olb.AdeLattice(desc, dims, "f64")
    a.set_tau(0.9)
    a.set_velocity((0.03, 0.0, 0.0))
    a.set_material(m, 1 if desc == 2 else 5, wall)
    a.init(np.ascontiguousarray(np.where(m == 1, 1.5, 0.0)))
    prev = None
    for _ in range(400):
        a.step(200)
        C = a.density().cpu().numpy()[0, 1:-1, 0]
        if prev is not None and np.max(np.abs(C - prev)) < 1e-15:
            break
        prev = C
    a.close()
    y = np.arange(1, ny - 1, dtype=float)
    assert np.max(np.abs(C - (1.0 + (y - 0.5) / (ny - 2)))) <= 1e-12


def test_ade_velocity_from_a_fluid_lattice(olb):
    """Coupled run: the scalar advected by the fluid's own velocity, taken on the
    device, equals the run fed the same velocity through olb_moments."""
    import torch

    n = 24
    fl = olb.Lattice(olb.D3Q19, (n, n, n), dtype="f64", scheme="pull")
    fl.set_material(torch.ones(n ** 3, dtype=torch.uint8, device="cuda"), 7)
    fl.set_bgk(0.7)
    rho, u = I.tgv3d(n, 0.03)
    fl.init_equilibrium(torch.from_numpy(rho.reshape(-1)).cuda(), torch.from_numpy(u.reshape(-1)).cuda())
    C0 = torch.from_numpy(1.0 + I.uniform(43, (n, n, n))).cuda()
    a = olb.AdeLattice(3, (n, n, n), "f64")
    b = olb.AdeLattice(3, (n, n, n), "f64")
    for lat in (a, b):
        lat.set_tau(0.8)
        lat.set_velocity((0.0, 0.0, 0.0))
        lat.init(C0)
    for _ in range(15):
        fl.step(1)
        a.set_velocity_from(fl)
        a.step(1)
        _, uu = fl.moments()
        b.set_velocity(field=uu.contiguous())
        b.step(1)
    assert torch.equal(a.density(), b.density())
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(3, (n, n, n + 1)).set_velocity_from(fl)
    a.close()
    b.close()
    fl.close()
