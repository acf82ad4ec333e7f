"""Pins of the oracle's advection-diffusion BGK (section "Advection--Diffusion
Equation": first-order equilibrium g^eq_i = w_i C (1 + c_i.v/cs2) on D2Q5 / D3Q7,
diffusivity mu = cs2 (tau - 1/2)).

* Tables: sum w = 1, sum w c = 0, sum w c_a c_b = cs2 delta_ab, opposites.
* Equilibrium moments: sum g^eq = C, sum c g^eq = C v.
* The scalar is conserved; a uniform field is a fixed point.
* Second-order convergence to the closed-form solutions of the guide's examples
  advectionDiffusion1d (with its parameter table), advectionDiffusion2d and the
  smooth case of advectionDiffusion3d.
"""
import math

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


@pytest.mark.parametrize("d", [0, 1])
def test_ade_tables(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.ade_descriptor(d)
    assert (dim, q) == ((2, 5) if d == 0 else (3, 7))
    assert not c[0].any() and w[0] > 0
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(w @ c).max() < 1e-15
    second = np.einsum("i,ia,ib->ab", w, c, c)
    eye = np.diag([1.0] * dim + [0.0] * (3 - dim))
    assert np.abs(second - cs2 * eye).max() < 1e-15
    for i in range(q):
        assert (c[opp[i]] == -c[i]).all()
    # face velocities: the first non-zero component is -1 for i = 1 .. (q-1)/2
    for i in range(1, (q - 1) // 2 + 1):
        assert c[i][np.nonzero(c[i])[0][0]] == -1 and opp[i] == i + (q - 1) // 2


@pytest.mark.parametrize("d", [0, 1])
def test_ade_equilibrium_moments(oracle, d):
    dim, q, c, _, _, _ = oracle.ade_descriptor(d)
    shape = (1, 3, 4) if d == 0 else (2, 3, 4)
    C = 0.5 + I.uniform(11, shape)
    v = 0.2 * (I.uniform(12, (3,) + shape) - 0.5)
    if d == 0:
        v[2] = 0.0
    lat = oracle.AdeLattice(d, shape, 0.9, v)
    g = lat.init(C)
    assert np.abs(g.sum(axis=0) - C).max() <= 1e-15 * C.max()
    flux = np.einsum("ia,i...->a...", c.astype(float), g)
    assert np.abs(flux - C * v).max() <= 1e-16


@pytest.mark.parametrize("d", [0, 1])
def test_ade_conserves_the_scalar_and_keeps_a_uniform_field(oracle, d):
    shape = (1, 9, 11) if d == 0 else (5, 6, 7)
    v = (0.05, -0.03, 0.02 if d == 1 else 0.0)
    lat = oracle.AdeLattice(d, shape, 0.7, v)
    C = 1.0 + I.uniform(13, shape)
    g = lat.init(C)
    total = g.sum()
    lat.step(g, 120)
    assert abs(g.sum() - total) <= 1e-13 * total
    u = lat.init(np.full(shape, 1.3))
    ref = u.copy()
    lat.step(u, 50)
    assert np.abs(u - ref).max() <= 1e-15


def _sine_run(oracle, d, n, tau, mu, u, T, dims_sin):
    """Periodic [-1, 1]^dims with n cells per side (x_i = -1 + i dx), diffusive scaling
    dt = mu_L dx^2 / mu, C = 1 + prod_a sin(pi (x_a - u_a t)) on the first `dims_sin`
    axes; returns the relative L2 error of C - 1 at the step nearest to time T."""
    _, _, _, _, _, cs2 = oracle.ade_descriptor(d)
    mu_l = cs2 * (tau - 0.5)
    dx = 2.0 / n
    dt = mu_l * dx * dx / mu
    ul = [ua * dt / dx for ua in u]
    steps = int(round(T / dt))
    t = steps * dt
    shape = (1, 1 if dims_sin < 2 else n, n) if d == 0 else (n, n, n)
    x = -1.0 + dx * np.arange(n)

    def field(time):
        prof = np.ones(shape)
        axes = [(2, 0), (1, 1), (0, 2)][:dims_sin]  # (array axis, velocity component)
        for ax, comp in axes:
            s = np.sin(math.pi * (x - u[comp] * time))
            prof = prof * s.reshape([n if k == ax else 1 for k in range(3)])
        return prof

    lat = oracle.AdeLattice(d, shape, tau, (ul[0], ul[1], ul[2]))
    g = lat.init(1.0 + field(0.0))
    lat.step(g, steps)
    exact = field(t) * math.exp(-dims_sin * mu * math.pi ** 2 * t)
    num = lat.density(g) - 1.0
    return float(np.linalg.norm(num - exact) / np.linalg.norm(exact))


def _eoc(errs):
    return [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(len(errs) - 1)]


def test_advection_diffusion_1d_with_the_guides_parameters(oracle):
    """advectionDiffusion1d: mu = 1.5, Pe = 40/3 on [-1, 1] (u = 10), dt = dx^2, and the
    table's resolutions N = 50, 100, 200 with u_L = 0.4, 0.2, 0.1 (tau = 1/2 + mu/cs2 = 5
    on D2Q5); chi* = sin(pi (x - u t)) exp(-mu pi^2 t), here at t = 0.05.  N = 50 with
    u_L = 0.4 is not yet asymptotic (46% error): the order there is 1.79, and 1.98 on the
    finer pair."""
    errs = []
    for n, u_l in ((50, 0.4), (100, 0.2), (200, 0.1)):
        dx = 2.0 / n
        assert abs(10.0 * dx - u_l) < 1e-15  # u_L = u dt / dx with dt = dx^2
        errs.append(_sine_run(oracle, 0, n, 5.0, 1.5, (10.0, 0.0, 0.0), 0.05, 1))
    eoc = _eoc(errs)
    assert 1.7 <= eoc[0] <= 2.2 and 1.9 <= eoc[1] <= 2.1, (errs, eoc)


def test_advection_diffusion_2d_second_order(oracle):
    """advectionDiffusion2d: mu = 0.05, u = (0.5, 0.25), until the pulse has decayed to
    about half."""
    errs = [_sine_run(oracle, 0, n, 0.8, 0.05, (0.5, 0.25, 0.0), 0.7, 2) for n in (32, 64, 128)]
    eoc = _eoc(errs)
    assert all(1.8 <= e <= 2.2 for e in eoc), (errs, eoc)


def test_advection_diffusion_3d_second_order(oracle):
    """advectionDiffusion3d, smooth case: chi* = prod sin(pi (x_a - u_a t)) exp(-3 mu pi^2 t)."""
    errs = [_sine_run(oracle, 1, n, 0.8, 0.05, (0.5, 0.25, -0.3), 0.3, 3) for n in (12, 24, 48)]
    eoc = _eoc(errs)
    assert all(1.8 <= e <= 2.3 for e in eoc), (errs, eoc)


# ---------------------------------------------------------------------------------
# Boundaries: no-flux walls (bounce-back) and Dirichlet cells (the guide's constant-
# temperature boundary, read as anti-bounce-back g_opp(i)(x) = -g*_i(x) + 2 w_i C_w).
# ---------------------------------------------------------------------------------
def _plates(d, n_par, ny, lo=2, hi=3):
    shape = (1, ny, n_par) if d == 0 else (n_par, ny, n_par)
    m = np.ones(shape, np.uint8)
    m[:, 0, :] = lo
    m[:, -1, :] = hi
    return m


@pytest.mark.parametrize("d,tau,v", [(0, 0.6, 0.0), (0, 1.0, 0.05), (0, 2.0, 0.0), (1, 0.8, 0.04)])
def test_dirichlet_plates_give_the_exact_linear_profile(oracle, d, tau, v):
    """Steady diffusion between two Dirichlet plates: C is the straight line through
    C_lo and C_hi at the halfway walls y = 1/2 and y = ny - 3/2, whatever tau and a
    velocity along the plates."""
    ny = 12
    m = _plates(d, 4, ny)
    wall = np.zeros(256)
    wall[2], wall[3] = 1.0, 2.0
    lat = oracle.AdeLattice(d, m.shape, tau, (v, 0.0, 0.0), material=m, wall_C=wall,
                            periodic=1 if d == 0 else 5)
    g = lat.init(np.where(m == 1, 1.5, 0.0))
    prev = None
    for _ in range(400):
        lat.step(g, 200)
        C = lat.density(g)[0, 1:-1, 0]
        if prev is not None and np.max(np.abs(C - prev)) < 1e-15:
            break
        prev = C
    y = np.arange(1, ny - 1, dtype=float)
    exact = 1.0 + (y - 0.5) / (ny - 2)
    assert np.max(np.abs(C - exact)) <= 1e-12


@pytest.mark.parametrize("d", [0, 1])
def test_no_flux_walls_conserve_the_scalar(oracle, d):
    shape = (1, 9, 11) if d == 0 else (6, 7, 8)
    m = np.zeros(shape, np.uint8)
    if d == 0:
        m[0, 1:-1, 1:-1] = 1
    else:
        m[1:-1, 1:-1, 1:-1] = 1
    lat = oracle.AdeLattice(d, shape, 0.7, (0.05, -0.02, 0.03 if d == 1 else 0.0), material=m, periodic=0)
    C = np.where(m == 1, 1.0 + I.uniform(31, shape), 0.0)
    g = lat.init(C)
    bulk = m == 1
    total = g[:, bulk].sum()
    lat.step(g, 150)
    assert abs(g[:, bulk].sum() - total) <= 1e-13 * total


def test_domain_edges_act_as_no_flux_walls(oracle):
    """A non-periodic edge and an explicit layer of no-flux cells give the same bulk."""
    C = 1.0 + I.uniform(32, (1, 8, 10))
    a = oracle.AdeLattice(0, (1, 8, 10), 0.8, (0.03, 0.02, 0.0), periodic=0)
    ga = a.init(C)
    a.step(ga, 60)
    m = np.zeros((1, 10, 12), np.uint8)
    m[0, 1:-1, 1:-1] = 1
    Cb = np.zeros((1, 10, 12))
    Cb[0, 1:-1, 1:-1] = C[0]
    b = oracle.AdeLattice(0, (1, 10, 12), 0.8, (0.03, 0.02, 0.0), material=m, periodic=0)
    gb = b.init(Cb)
    b.step(gb, 60)
    assert np.array_equal(a.density(ga)[0], b.density(gb)[0, 1:-1, 1:-1])
