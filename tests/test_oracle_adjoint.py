"""Pins of the oracle's discrete adjoint (reading: exact adjoint of the discrete
map, since the guide names the adjoint LBM of its OptiCaseDual but does not
print its equations -- section "Derivative Computation").

Three independent references: the transpose identity <J v, w> = <v, J^T w> with
J v from forward-mode dual numbers (the analogue of ADf, same section); the
tangent-linear derivative of the whole run; and central difference quotients
(OptiCaseCDQ) of the objective computed from plain forward runs.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


def _porous_channel(oracle, d, shape, tau=0.8, seed=2, moving=False):
    nz, ny, nx = shape
    m = I.channel(nx, ny, nz)
    wu = np.zeros((256, 3))
    if moving:
        m[:, ny - 1, :] = I.LID
        wu[I.LID] = (0.03, 0.0, 0.01 if d == 1 else 0.0)
    gamma = I.smoothed_porosity(seed, m)
    F = (I.channel_force(ny, tau, 0.03), 0.0, 0.0)
    lat = oracle.Lattice(d, m, tau, periodic=1, force=F, gamma=gamma, wall_u=wu)
    f0 = lat.init_equilibrium(*I.rest(m.shape)) + I.population_noise(seed + 1, lat.q, m, 1e-4)
    return lat, f0


@pytest.mark.parametrize("d", [0, 1])
def test_collision_transpose_identity(oracle, d):
    shape = (1, 6, 7) if d == 0 else (4, 5, 6)
    lat, f = _porous_channel(oracle, d, shape)
    q = lat.q
    v = I.uniform(71, (q,) + shape) - 0.5
    vg = I.uniform(72, shape) - 0.5
    vt = 0.3
    w = I.uniform(73, (q,) + shape) - 0.5
    fl = lat.material == I.FLUID
    w[:, ~fl] = 0.0
    Jv = lat.collide_tangent(f, v, dgamma=vg, dtau=vt)
    lam, dg, dt = lat.collide_adjoint(f, w)
    lhs = float((Jv * w).sum())
    rhs = float((v * lam).sum() + (vg * dg).sum() + vt * dt)
    assert abs(lhs - rhs) <= 1e-14 * max(abs(lhs), 1e-300)


@pytest.mark.parametrize("d", [0, 1])
def test_streaming_transpose_identity(oracle, d):
    shape = (1, 6, 7) if d == 0 else (5, 6, 7)
    nz, ny, nx = shape
    m = I.channel(nx, ny, nz)
    m[:, ny - 1, :] = I.LID
    wu = np.zeros((256, 3))
    wu[I.LID] = (0.04, 0.0, -0.02 if d == 1 else 0.0)
    lat = oracle.Lattice(d, m, 0.7, periodic=1, wall_u=wu)
    q = lat.q
    fl = m == I.FLUID
    v = np.where(fl[None], I.uniform(81, (q,) + shape) - 0.5, 0.0)
    p = np.where(fl[None], I.uniform(82, (q,) + shape) - 0.5, 0.0)
    w = np.where(fl[None], I.uniform(83, (q,) + shape) - 0.5, 0.0)
    zero = np.zeros_like(v)
    # Streaming is affine in (post-collision fs, pre-collision fpre): the linear
    # part in fs is S v = stream(v, 0) - stream(0, 0), the part in fpre is
    # stream(0, p) - stream(0, 0) (moving-wall density term).
    base = lat.stream(zero, zero)
    Sv = lat.stream(v, zero) - base
    Sp = lat.stream(zero, p) - base
    lams, direct = lat.stream_adjoint(w)
    lhs = float((Sv * w)[:, fl].sum())
    rhs = float((v * lams)[:, fl].sum())
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    lhs_p = float((Sp * w)[:, fl].sum())
    rhs_p = float((p.sum(axis=0) * direct)[fl].sum())
    assert abs(lhs_p) > 1e-6
    assert abs(lhs_p - rhs_p) <= 1e-13 * abs(lhs_p)


@pytest.mark.parametrize("d,moving", [(0, False), (1, False), (0, True), (1, True)])
def test_adjoint_matches_tangent_linear(oracle, d, moving):
    shape = (1, 8, 10) if d == 0 else (5, 6, 8)
    lat, f0 = _porous_channel(oracle, d, shape, moving=moving)
    n = 30
    obj = (0, shape[2] - 1, 0)  # mean u_x on the plane x = nx - 1
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    fl = lat.material == I.FLUID
    for k, seed in enumerate((91, 92, 93)):
        v = np.where(fl, I.uniform(seed, shape) - 0.5, 0.0)
        s = 0.7 if k == 1 else 0.0
        loss_t, dl = lat.tangent(f0, n, obj, dgamma=v, dtau=s)
        assert loss_t == loss
        pred = float((dg * v).sum() + dtau * s)
        assert abs(pred - dl) <= 1e-11 * abs(dl), (pred, dl)


def test_adjoint_matches_central_differences(oracle):
    shape = (4, 6, 8)
    lat, f0 = _porous_channel(oracle, 1, shape)
    n = 25
    obj = (0, shape[2] - 1, 0)
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    cells = I.random_fluid_cells(3, lat.material, 6)
    h = 1e-5
    base_gamma = lat.gamma.copy()
    for c in cells:
        vals = []
        for sgn in (1, -1):
            g = base_gamma.copy()
            g.reshape(-1)[c] += sgn * h
            lat.gamma = g
            f = f0.copy()
            lat.step(f, n)
            vals.append(lat.loss(f, obj))
        lat.gamma = base_gamma
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dg.reshape(-1)[c]) <= 1e-6 * abs(fd) + 1e-14
    ht = 1e-6
    vals = []
    for sgn in (1, -1):
        lat.tau = 0.8 + sgn * ht
        f = f0.copy()
        lat.step(f, n)
        vals.append(lat.loss(f, obj))
    lat.tau = 0.8
    fd = (vals[0] - vals[1]) / (2 * ht)
    assert abs(fd - dtau) <= 1e-6 * abs(fd)


def test_adjoint_rejects_empty_objective_plane(oracle):
    lat, f0 = _porous_channel(oracle, 0, (1, 6, 6))
    with pytest.raises(ValueError):
        lat.adjoint(f0, 3, (1, 0, 0))  # plane y = 0 is all wall


# ---------------------------------------------------------------------------------
# Velocity-misfit objective J = 1/2 sum_region |u - u*|^2 (the guide's optimisation
# examples domainIdentification3d and testFlowOpti3d, with dx = 1).
# ---------------------------------------------------------------------------------
def _misfit(oracle, lat, f0, n, seed=5):
    """A target field u* (the final velocity of a run with another porosity, plus a
    smooth offset) and a region (a box of the interior)."""
    nz, ny, nx = lat.shape
    g_alt = np.clip(lat.gamma * (0.8 + 0.4 * I.uniform(seed, lat.shape)), 0.0, 1.0)
    saved = lat.gamma
    lat.gamma = g_alt
    f = f0.copy()
    lat.step(f, n)
    _, u_ref = lat.moments(f)
    lat.gamma = saved
    u_t = u_ref + 1e-3 * (I.uniform(seed + 1, u_ref.shape) - 0.5)
    region = np.zeros(lat.shape, bool)
    region[:, 1:ny - 1, nx // 4: nx - 1] = True
    return oracle.Misfit(u_t, region)


def test_misfit_loss_is_half_the_squared_velocity_error(oracle):
    lat, f0 = _porous_channel(oracle, 1, (4, 6, 8))
    f = f0.copy()
    lat.step(f, 7)
    obj = _misfit(oracle, lat, f0, 7)
    _, u = lat.moments(f)
    sel = obj.region & (lat.material == I.FLUID)
    want = 0.5 * float(((u - obj.u_target) ** 2)[:, sel].sum())
    assert abs(lat.loss(f, obj) - want) <= 1e-14 * want
    # no region: every fluid cell; D2Q9 sums the two components only
    lat2, f2 = _porous_channel(oracle, 0, (1, 6, 9))
    _, u2 = lat2.moments(f2)
    ut = np.zeros((3,) + lat2.shape)
    ut[:2] = 0.01
    ut[2] = 5.0  # ignored in 2D
    fl = lat2.material == I.FLUID
    want2 = 0.5 * float(((u2[:2] - 0.01) ** 2)[:, fl].sum())
    assert abs(lat2.loss(f2, oracle.Misfit(ut)) - want2) <= 1e-14 * want2


@pytest.mark.parametrize("d,moving", [(0, False), (1, False), (0, True), (1, True)])
def test_misfit_adjoint_matches_tangent_linear(oracle, d, moving):
    shape = (1, 8, 10) if d == 0 else (5, 6, 8)
    lat, f0 = _porous_channel(oracle, d, shape, moving=moving)
    n = 30
    obj = _misfit(oracle, lat, f0, n)
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    assert loss > 0
    fl = lat.material == I.FLUID
    for k, seed in enumerate((94, 95, 96)):
        v = np.where(fl, I.uniform(seed, shape) - 0.5, 0.0)
        s = 0.7 if k == 1 else 0.0
        loss_t, dl = lat.tangent(f0, n, obj, dgamma=v, dtau=s)
        assert loss_t == loss
        pred = float((dg * v).sum() + dtau * s)
        assert abs(pred - dl) <= 1e-11 * abs(dl), (pred, dl)


def test_misfit_adjoint_matches_central_differences(oracle):
    shape = (4, 6, 8)
    lat, f0 = _porous_channel(oracle, 1, shape)
    n = 25
    obj = _misfit(oracle, lat, f0, n)
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    cells = I.random_fluid_cells(4, lat.material, 6)
    h = 1e-5
    base_gamma = lat.gamma.copy()
    for c in cells:
        vals = []
        for sgn in (1, -1):
            g = base_gamma.copy()
            g.reshape(-1)[c] += sgn * h
            lat.gamma = g
            f = f0.copy()
            lat.step(f, n)
            vals.append(lat.loss(f, obj))
        lat.gamma = base_gamma
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dg.reshape(-1)[c]) <= 1e-6 * abs(fd) + 1e-16
    ht = 1e-6
    vals = []
    for sgn in (1, -1):
        lat.tau = 0.8 + sgn * ht
        f = f0.copy()
        lat.step(f, n)
        vals.append(lat.loss(f, obj))
    lat.tau = 0.8
    fd = (vals[0] - vals[1]) / (2 * ht)
    assert abs(fd - dtau) <= 1e-6 * abs(fd)


def test_misfit_gradient_vanishes_at_the_reference_and_descends_near_it(oracle):
    """With u* the velocity of the current porosity the misfit is 0 and so is its
    gradient; moving the porosity away and then a small step against the gradient
    lowers the misfit (the steepest-descent step of the guide's optimisers)."""
    shape = (4, 6, 8)
    lat, f0 = _porous_channel(oracle, 1, shape)
    n = 20
    f = f0.copy()
    lat.step(f, n)
    _, u_ref = lat.moments(f)
    obj = oracle.Misfit(u_ref)
    loss, dg, dtau = lat.adjoint(f0, n, obj)
    assert loss == 0.0 and not dg.any() and dtau == 0.0
    g_true = lat.gamma.copy()
    fl = lat.material == I.FLUID
    lat.gamma = np.where(fl, np.clip(g_true - 0.2 * I.uniform(7, shape), 0.0, 1.0), g_true)
    loss1, dg1, _ = lat.adjoint(f0, n, obj)
    assert loss1 > 0
    step = 0.1 * loss1 / float((dg1 ** 2).sum())
    lat.gamma = lat.gamma - step * dg1
    f = f0.copy()
    lat.step(f, n)
    assert lat.loss(f, obj) < loss1 * (1 - 0.05)


def test_misfit_rejects_an_empty_region(oracle):
    lat, f0 = _porous_channel(oracle, 0, (1, 6, 6))
    region = np.zeros(lat.shape, bool)
    region[:, 0, :] = True  # wall row only
    with pytest.raises(ValueError):
        lat.adjoint(f0, 3, oracle.Misfit(np.zeros((3,) + lat.shape), region))
