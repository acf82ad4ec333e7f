"""Pins of the oracle's TRT collision (collision::TRT of the guide's dynamics
tuples, section "Dynamics"; the guide names the operator without printing it, and
it is read as the two-relaxation-time operator with omega+ = 1/tau on the even
part and omega- set by the magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2)).

* With omega- = omega+ (Lambda = (tau - 1/2)^2) it is the BGK operator.
* A collision conserves mass, and momentum up to the Guo source F.
* The viscosity comes from omega+ alone: the Taylor-Green vortex decays at
  exp(-2 nu k^2 t), nu = (tau - 1/2)/3, whatever Lambda.
* Force-driven Poiseuille flow between halfway bounce-back walls is the exact
  parabola with its zeros on the walls for Lambda = 3/16 at every tau (the known
  property of the TRT operator); BGK has that only at tau = 1/2 + sqrt(3/16).
* Its discrete adjoint (explicit Jacobian) against dual numbers and central
  differences.
"""
import math

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


@pytest.mark.parametrize("d", [0, 1])
def test_trt_with_equal_rates_is_bgk(oracle, d):
    q = 9 if d == 0 else 19
    for k, tau in enumerate((0.53, 0.8, 1.7)):
        magic = (tau - 0.5) ** 2
        for c in range(5):
            rho = 0.9 + 0.2 * I.uniform(100 + k * 10 + c, (1,))[0]
            u = 0.1 * (I.uniform(200 + k * 10 + c, (3,)) - 0.5)
            if d == 0:
                u[2] = 0
            f = oracle.equilibrium(d, rho, u) + 1e-3 * (I.uniform(300 + k * 10 + c, (q,)) - 0.5)
            F = (1e-4, -2e-4, 3e-5 if d == 1 else 0.0)
            a = oracle.collide_cell(d, f, tau, gamma=0.7, F=F)
            b = oracle.collide_cell_trt(d, f, tau, magic, gamma=0.7, F=F)
            assert np.max(np.abs(a - b)) <= 1e-15 * np.max(np.abs(a))


def test_trt_lattice_with_equal_rates_matches_bgk(oracle):
    tau = 0.62
    m = I.cavity_box(9, 8, 7)
    wu = np.zeros((256, 3))
    wu[I.LID] = (0.05, 0.0, 0.02)
    runs = []
    for coll, magic in ((oracle.BGK, 0.25), (oracle.TRT, (tau - 0.5) ** 2)):
        lat = oracle.Lattice(1, m, tau, wall_u=wu, force=(1e-5, 0, 0), gamma=I.smoothed_porosity(3, m),
                             collision=coll, magic=magic)
        f = lat.init_equilibrium(*I.rest(m.shape)) + I.population_noise(4, 19, m, 1e-4)
        lat.step(f, 40)
        runs.append(f)
    fl = m == I.FLUID
    assert np.max(np.abs(runs[0] - runs[1])[:, fl]) <= 1e-13 * np.max(np.abs(runs[0]))


@pytest.mark.parametrize("d", [0, 1])
def test_trt_conserves_mass_and_momentum(oracle, d):
    _, q, c, _, _, _ = oracle.descriptor(d)
    for k in range(6):
        rho = 0.9 + 0.2 * I.uniform(400 + k, (1,))[0]
        u = 0.1 * (I.uniform(500 + k, (3,)) - 0.5)
        if d == 0:
            u[2] = 0
        f = oracle.equilibrium(d, rho, u) + 1e-2 * (I.uniform(600 + k, (q,)) - 0.5)
        F = np.array([2e-4, -1e-4, 5e-5 if d == 1 else 0.0])
        fs = oracle.collide_cell_trt(d, f, 0.7 + 0.2 * k, 1.0 / (3 + k), F=F)
        assert abs(fs.sum() - f.sum()) <= 1e-15 * f.sum()
        assert np.max(np.abs(c.T @ fs - (c.T @ f + F))) <= 1e-15


@pytest.mark.parametrize("magic", [1.0 / 12.0, 3.0 / 16.0, 1.0])
def test_trt_viscosity_from_the_even_rate(oracle, magic):
    """Under diffusive scaling (tau fixed, u0 ~ 1/N, steps ~ N^2) the amplitude
    converges at second order to exp(-2 nu k^2 t) with nu = (tau - 1/2)/3 for every
    Lambda; Lambda only changes the error constant."""
    tau = 0.8
    errs = []
    for n in (16, 32, 64):
        s = n / 16
        m = I.periodic_box(n, n, 1)
        lat = oracle.Lattice(0, m, tau, periodic=7, collision=oracle.TRT, magic=magic)
        u0, steps = 0.08 / s, int(64 * s * s)
        f = lat.init_equilibrium(*I.tgv2d(n, u0))
        lat.step(f, steps)
        _, u = lat.moments(f)
        ua = I.tgv2d_velocity(n, u0, I.viscosity(tau), steps)
        amp = float((u[:2] * ua[:2]).sum() / (ua[:2] ** 2).sum())
        errs.append(abs(amp - 1.0))
    eoc = [math.log(errs[i] / errs[i + 1]) / math.log(2.0) for i in range(2)]
    assert all(1.8 <= e <= 2.2 for e in eoc), (errs, eoc)


def _steady_profile(oracle, d, tau, ny, F, collision, magic, steps=40000):
    nz = 1 if d == 0 else 2
    m = I.plates(1, ny, nz)
    lat = oracle.Lattice(d, m, tau, periodic=1 | 4, force=(F, 0, 0), collision=collision, magic=magic)
    f = lat.init_equilibrium(*I.rest(m.shape))
    window = []
    for _ in range(steps // 200):
        lat.step(f, 200)
        u = lat.moments(f)[1][0, 0, :, 0]
        window = (window + [u[ny // 2]])[-10:]
        if len(window) == 10 and np.std(window) < 1e-13 * abs(np.mean(window)):
            break
    _, u = lat.moments(f)
    return np.arange(1, ny - 1, dtype=float), u[0, 0, 1:-1, 0]


@pytest.mark.parametrize("d,tau", [(0, 0.6), (0, 1.0), (1, 0.75), (0, 2.0)])
def test_trt_poiseuille_exact_at_magic_3_16(oracle, d, tau):
    ny, F = 12, 1e-6
    nu = I.viscosity(tau)
    y, prof = _steady_profile(oracle, d, tau, ny, F, oracle.TRT, 3.0 / 16.0)
    exact = F / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    assert np.max(np.abs(prof - exact)) <= 1e-9 * exact.max()
    # BGK at the same tau misses the walls (tau != 1/2 + sqrt(3/16))
    if abs(tau - (0.5 + math.sqrt(3.0 / 16.0))) > 0.05:
        yb, pb = _steady_profile(oracle, d, tau, ny, F, oracle.BGK, 0.25)
        assert np.max(np.abs(pb - exact)) > 1e-4 * exact.max()


def test_trt_rejects_a_non_positive_magic_parameter(oracle):
    with pytest.raises(ValueError):
        oracle.collide_cell_trt(0, np.ones(9) / 9, 0.8, 0.0)
    m = I.channel(8, 6, 1)
    lat = oracle.Lattice(0, m, 0.8, periodic=1, collision=oracle.TRT, magic=-1.0)
    with pytest.raises(ValueError):
        lat.step(lat.init_equilibrium(*I.rest(m.shape)), 1)


# ---------------------------------------------------------------------------------
# The discrete adjoint of the TRT map (the explicit Jacobian of the oracle), pinned
# like the BGK one: transpose identity against dual numbers, tangent-linear of the
# whole run, central differences.  d/dtau holds Lambda fixed (omega- follows omega+).
# ---------------------------------------------------------------------------------
def _trt_channel(oracle, d, shape, moving=False, magic=3.0 / 16.0, tau=0.7):
    from test_oracle_adjoint import _porous_channel

    lat, f0 = _porous_channel(oracle, d, shape, tau=tau, moving=moving)
    lat.collision = oracle.TRT
    lat.magic = magic
    return lat, f0


@pytest.mark.parametrize("d,magic", [(0, 3.0 / 16.0), (1, 3.0 / 16.0), (1, 1.0)])
def test_trt_collision_transpose_identity(oracle, d, magic):
    shape = (1, 6, 7) if d == 0 else (4, 5, 6)
    lat, f = _trt_channel(oracle, d, shape, magic=magic)
    q = lat.q
    v = I.uniform(171, (q,) + shape) - 0.5
    vg = I.uniform(172, shape) - 0.5
    vt = 0.3
    w = I.uniform(173, (q,) + shape) - 0.5
    fl = lat.material == I.FLUID
    w[:, ~fl] = 0.0
    Jv = lat.collide_tangent(f, v, dgamma=vg, dtau=vt)
    lam, dg, dt = lat.collide_adjoint(f, w)
    lhs = float((Jv * w).sum())
    rhs = float((v * lam).sum() + (vg * dg).sum() + vt * dt)
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    # the tau part alone (the chain through omega-)
    lhs_t = float((lat.collide_tangent(f, np.zeros_like(v), dtau=1.0) * w).sum())
    assert abs(lhs_t - dt) <= 1e-13 * abs(lhs_t)


@pytest.mark.parametrize("d,moving", [(0, False), (1, False), (0, True), (1, True)])
def test_trt_adjoint_matches_tangent_linear(oracle, d, moving):
    shape = (1, 8, 10) if d == 0 else (5, 6, 8)
    lat, f0 = _trt_channel(oracle, d, shape, moving=moving)
    n = 30
    fl = lat.material == I.FLUID
    f = f0.copy()
    lat.step(f, n)
    _, u = lat.moments(f)
    for obj in ((0, shape[2] - 1, 0), oracle.Misfit(u * 1.01 + 1e-4)):
        loss, dg, dtau = lat.adjoint(f0, n, obj)
        for k, seed in enumerate((191, 192)):
            v = np.where(fl, I.uniform(seed, shape) - 0.5, 0.0)
            s = 0.7 if k == 1 else 0.0
            loss_t, dl = lat.tangent(f0, n, obj, dgamma=v, dtau=s)
            assert loss_t == loss
            pred = float((dg * v).sum() + dtau * s)
            assert abs(pred - dl) <= 1e-11 * abs(dl), (pred, dl)


def test_trt_adjoint_matches_central_differences(oracle):
    shape = (4, 6, 8)
    lat, f0 = _trt_channel(oracle, 1, shape, magic=0.3)
    n = 25
    obj = (0, shape[2] - 1, 0)
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    base = lat.gamma.copy()
    for c in I.random_fluid_cells(5, lat.material, 5):
        vals = []
        for sgn in (1, -1):
            g = base.copy()
            g.reshape(-1)[c] += sgn * 1e-5
            lat.gamma = g
            f = f0.copy()
            lat.step(f, n)
            vals.append(lat.loss(f, obj))
        lat.gamma = base
        fd = (vals[0] - vals[1]) / 2e-5
        assert abs(fd - dg.reshape(-1)[c]) <= 1e-6 * abs(fd) + 1e-14
    vals = []
    for sgn in (1, -1):
        lat.tau = 0.7 + sgn * 1e-6
        f = f0.copy()
        lat.step(f, n)
        vals.append(lat.loss(f, obj))
    lat.tau = 0.7
    fd = (vals[0] - vals[1]) / 2e-6
    assert abs(fd - dtau) <= 1e-6 * abs(fd)
