"""Pins of the oracle's plane-mean objective (the discrete plane mode of the flux
functors, section "Discrete Flux Functor") and of its statistics max |u| and
sum |u|^2/2 (lesson "Extract Data From a Simulation"), against values that the
flow or the prescribed input fixes independently of the oracle's own reductions.

* Steady Couette flow between halfway walls is linear, u_x = U (y - 1/2)/(ny - 2)
  (pinned in the flow tests), so the mean of u_x over the fluid cells of any
  x- or z-plane is exactly U/2, and over a y-plane U (y - 1/2)/(ny - 2).  A plane
  average that also counted the wall cells of the plane, or that took the plane
  along another axis, gives a different number.
* Darcy flow through a uniform porous medium has u = K F / nu exactly, with the
  guide's permeability (pinned in the flow tests), and that value contains the
  F/2 shift of u = (j + F/2)/rho: without the shift the mean is off by F/2.
* A state built as f = f^eq(rho, u) has first moment rho u (pinned cell by cell),
  so every reduction over it has a closed form in the prescribed rho and u.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


def _steady(oracle, lat, f, probe, window=10, every=200, max_steps=40000):
    """Step until the probed value stops changing (sigma < 1e-13 of the mean over
    `window` samples, the ValueTracer criterion of the lesson "Convergence Check")."""
    vals = []
    for _ in range(max_steps // every):
        lat.step(f, every)
        vals = (vals + [probe(f)])[-window:]
        if len(vals) == window and np.std(vals) < 1e-13 * abs(np.mean(vals)):
            return f
    raise AssertionError("no steady state")


def _couette(oracle, d, tau, ny, U, nx=3):
    nz = 1 if d == 0 else 2
    m = I.plates(nx, ny, nz, top=I.LID)
    wu = np.zeros((256, 3))
    wu[I.LID] = (U, 0, 0)
    lat = oracle.Lattice(d, m, tau, periodic=1 | (4 if d == 1 else 0), wall_u=wu)
    f = lat.init_equilibrium(*I.rest(m.shape))
    _steady(oracle, lat, f, lambda f: lat.moments(f)[1][0, 0, ny // 2, 0])
    return lat, f, m


@pytest.mark.parametrize("d,tau", [(0, 0.8), (1, 0.6)])
def test_plane_mean_of_couette_flow(oracle, d, tau):
    ny, U = 10, 0.01
    lat, f, m = _couette(oracle, d, tau, ny, U)
    H = ny - 2
    # x-planes: every (y, z) of the plane, walls included; fluid cells average to U/2
    for ix in (0, 2):
        assert abs(lat.loss(f, (0, ix, 0, 0)) - U / 2) < 1e-11 * U
        assert abs(lat.loss(f, (0, ix, 1, 0))) < 1e-15  # u_y vanishes
    # y-planes: one fluid row each, mean = the linear profile at that row
    for iy in (1, 4, ny - 2):
        assert abs(lat.loss(f, (1, iy, 0, 0)) - U * (iy - 0.5) / H) < 1e-11 * U
    if d == 1:
        for iz in (0, 1):
            assert abs(lat.loss(f, (2, iz, 0, 0)) - U / 2) < 1e-11 * U


@pytest.mark.parametrize("d", [0, 1])
def test_plane_mean_of_darcy_flow_includes_the_force_shift(oracle, d):
    tau, d_por, F = 0.8, 0.9, 1e-5
    shape = (1, 3, 4) if d == 0 else (2, 3, 4)
    m = I.periodic_box(shape[2], shape[1], shape[0])
    lat = oracle.Lattice(d, m, tau, periodic=7 if d == 1 else 3, force=(F, 0, 0),
                         gamma=np.full(m.shape, d_por))
    f = lat.init_equilibrium(*I.rest(m.shape))
    lat.step(f, 4000)
    nu = I.viscosity(tau)
    K = nu * tau / (1.0 - d_por)
    exact = K * F / nu  # rho stays 1 in the uniform periodic flow
    for axis, index in ((0, 1), (1, 2)) + (((2, 1),) if d == 1 else ()):
        assert abs(lat.loss(f, (axis, index, 0, 0)) - exact) < 1e-10 * exact
        assert abs(lat.loss(f, (axis, index, 1, 0))) < 1e-11 * exact


def _prescribed(d, shape, seed):
    """Seeded rho in [0.9, 1.1] and |u| < 0.01 on every cell."""
    rho = 0.9 + 0.2 * I.uniform(seed, shape)
    u = 0.02 * (I.uniform(seed + 1, (3,) + shape) - 0.5) / np.sqrt(3.0)
    if d == 0:
        u[2] = 0.0
    return rho, u


@pytest.mark.parametrize("d", [0, 1])
def test_plane_mean_of_an_equilibrium_state_counts_fluid_cells_only(oracle, d):
    """Walls inside the plane (a solid block and the channel walls) carry their own
    prescribed velocities in f; only the plane's fluid cells enter the mean, and
    u = (rho u_in + F/2)/rho there."""
    shape = (1, 7, 6) if d == 0 else (5, 7, 6)
    nz, ny, nx = shape
    m = I.channel(nx, ny, nz)
    m[:, 2:4, 1:3] = I.WALL
    F = np.array([3e-4, -2e-4, 1e-4 if d == 1 else 0.0])
    lat = oracle.Lattice(d, m, 0.7, periodic=1, force=F)
    rho, u = _prescribed(d, shape, 11)
    f = lat.init_equilibrium(rho, u)
    fl = m == I.FLUID
    ur = u + F[:, None, None, None] / (2.0 * rho)
    for axis, index in ((0, 2), (0, 5), (1, 2), (1, 5)) + (((2, 1), (2, 3)) if d == 1 else ()):
        sel = np.zeros(shape, bool)
        sl = [slice(None)] * 3
        sl[2 - axis] = index
        sel[tuple(sl)] = True
        cells = sel & fl
        for comp in range(2 if d == 0 else 3):
            exact = ur[comp][cells].mean()
            assert abs(lat.loss(f, (axis, index, comp, 0)) - exact) < 1e-15


@pytest.mark.parametrize("d", [0, 1])
def test_max_speed_and_energy_of_a_prescribed_field(oracle, d):
    """max |u| is the largest speed |u| = |j + F/2| / rho over fluid cells: not the
    largest |j|, not the largest single component, and never a wall cell's."""
    shape = (1, 8, 9) if d == 0 else (6, 8, 9)
    m = I.cavity_box(shape[2], shape[1], shape[0])
    F = np.array([1e-5, 2e-5, -1e-5 if d == 1 else 0.0])
    wu = np.zeros((256, 3))
    lat = oracle.Lattice(d, m, 0.7, periodic=0, force=F, wall_u=wu)
    rho, u = _prescribed(d, shape, 21)
    z = 0 if d == 0 else 2
    # A: the fastest cell (|u| = 0.0781 by its three, or two, components)
    rho[z, 3, 3] = 1.0
    u[:, z, 3, 3] = (0.03, -0.04, 0.06) if d == 1 else (0.05, -0.06, 0.0)
    # B: largest momentum |j| = 1.2 * 0.07 = 0.084 > 0.0781, but |u| = 0.07
    rho[z, 4, 5] = 1.2
    u[:, z, 4, 5] = (0.07, 0.0, 0.0)
    # C: largest single component |u_y| (2D) or |u_z| (3D) = 0.075 < 0.0781
    u[:, z, 2, 6] = (0.0, 0.0, -0.075) if d == 1 else (0.0, -0.075, 0.0)
    # a wall cell with a prescribed (and ignored) velocity far above all of them
    assert m[z, 0, 4] != I.FLUID
    u[:, z, 0, 4] = (0.2, 0.0, 0.0)
    f = lat.init_equilibrium(rho, u)
    out = lat.diagnostics(f)
    fl = m == I.FLUID
    ur = u + F[:, None, None, None] / (2.0 * rho)
    speed = np.sqrt((ur ** 2).sum(axis=0))
    assert abs(out[5] - speed[fl].max()) < 1e-15
    assert abs(out[5] - 0.0781) < 2e-4
    assert abs(out[4] - 0.5 * (speed[fl] ** 2).sum()) < 1e-14 * out[4]
    assert abs(out[0] - rho[fl].sum()) < 1e-13 * out[0]
    for a in range(3):
        assert abs(out[1 + a] - (rho * u[a])[fl].sum()) < 1e-15 * fl.sum()
    assert out[6] == 0
