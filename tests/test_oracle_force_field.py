"""Pins of the oracle's per-cell force field and of the adjoint gradient with
respect to it (the distributed force control of the guide's testFlowOpti3d, whose
controls are the field's three components at every mesh point).

* A field equal to the uniform force everywhere gives the uniform-force run.
* A collision adds exactly the cell's force F(x) to its momentum (Guo, gamma = 1).
* Transpose identity of one collision with a force direction (BGK and TRT).
* dL/dF(x) against the dual-number tangent of whole runs, against central
  differences, and summed over the cells against the uniform-force derivative.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


def _field(seed, shape, scale=2e-5):
    return scale * (I.uniform(seed, (3,) + shape) - 0.5)


def _channel(oracle, d, shape, moving=False, collision=0, seed=2):
    from test_oracle_adjoint import _porous_channel

    lat, f0 = _porous_channel(oracle, d, shape, moving=moving, seed=seed)
    F = _field(seed + 40, shape)
    F[:, :, :, :] += np.array(lat.force).reshape(3, 1, 1, 1)
    if d == 0:
        F[2] = 0.0
    lat.force_field = np.ascontiguousarray(F)
    lat.collision = collision
    lat.magic = 3.0 / 16.0
    return lat, f0


def test_uniform_field_is_the_uniform_force(oracle):
    from test_oracle_adjoint import _porous_channel

    shape = (4, 6, 8)
    a, f0 = _porous_channel(oracle, 1, shape, moving=True)
    b, _ = _porous_channel(oracle, 1, shape, moving=True)
    b.force_field = np.ascontiguousarray(np.broadcast_to(np.array(a.force).reshape(3, 1, 1, 1), (3,) + shape))
    fa, fb = f0.copy(), f0.copy()
    a.step(fa, 20)
    b.step(fb, 20)
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("d", [0, 1])
def test_collision_adds_the_cell_force_to_its_momentum(oracle, d):
    shape = (1, 6, 7) if d == 0 else (4, 5, 6)
    lat, f = _channel(oracle, d, shape)
    lat.gamma = None
    _, _, c, _, _, _ = oracle.descriptor(d)
    fs = lat.collide(f)
    fl = lat.material == I.FLUID
    dj = np.einsum("ia,i...->a...", c.astype(float), fs - f)
    assert np.max(np.abs(dj - lat.force_field)[:, fl]) <= 1e-16


@pytest.mark.parametrize("d,collision", [(0, 0), (1, 0), (1, 1)])
def test_collision_transpose_identity_with_a_force_direction(oracle, d, collision):
    shape = (1, 6, 7) if d == 0 else (4, 5, 6)
    lat, f = _channel(oracle, d, shape, collision=collision)
    q = lat.q
    v = I.uniform(271, (q,) + shape) - 0.5
    vg = I.uniform(272, shape) - 0.5
    vF = I.uniform(273, (3,) + shape) - 0.5
    w = I.uniform(274, (q,) + shape) - 0.5
    fl = lat.material == I.FLUID
    w[:, ~fl] = 0.0
    Jv = lat.collide_tangent(f, v, dgamma=vg, dtau=0.4, dforce=vF)
    lam, dg, dt, dF = lat.collide_adjoint(f, w, want_dforce=True)
    lhs = float((Jv * w).sum())
    rhs = float((v * lam).sum() + (vg * dg).sum() + 0.4 * dt + (vF * dF).sum())
    assert abs(lhs - rhs) <= 1e-14 * abs(lhs)
    # the force part alone
    lhs_f = float((lat.collide_tangent(f, np.zeros_like(v), dforce=vF) * w).sum())
    assert abs(lhs_f - float((vF * dF).sum())) <= 1e-13 * abs(lhs_f)


@pytest.mark.parametrize("d,moving,collision", [(0, False, 0), (1, False, 0), (1, True, 0), (0, True, 1),
                                                (1, True, 1)])
def test_force_gradient_matches_tangent_linear(oracle, d, moving, collision):
    shape = (1, 8, 10) if d == 0 else (5, 6, 8)
    lat, f0 = _channel(oracle, d, shape, moving=moving, collision=collision)
    n = 25
    f = f0.copy()
    lat.step(f, n)
    _, u = lat.moments(f)
    fl = lat.material == I.FLUID
    for obj in ((0, shape[2] - 1, 0), oracle.Misfit(u * 1.02 - 1e-4)):
        loss, dg, dtau, dF = lat.adjoint(f0, n, obj, want_dforce=True)
        assert not dF[:, ~fl].any()
        for seed in (281, 282):
            vF = np.where(fl[None], I.uniform(seed, (3,) + shape) - 0.5, 0.0)
            if d == 0:
                vF[2] = 0.0
            loss_t, dl = lat.tangent(f0, n, obj, dforce=vF)
            assert loss_t == loss
            pred = float((dF * vF).sum())
            assert abs(pred - dl) <= 1e-11 * abs(dl), (pred, dl)


def test_force_gradient_matches_central_differences(oracle):
    shape = (4, 6, 8)
    lat, f0 = _channel(oracle, 1, shape)
    n = 20
    obj = (0, shape[2] - 1, 0)
    loss, dg, dtau, dF = lat.adjoint(f0, n, obj, want_dforce=True)
    base = lat.force_field.copy()
    h = 1e-5  # the loss carries ~1e-16 of rounding noise: h = 1e-7 leaves ~5e-10 in the quotient
    for k, c in enumerate(I.random_fluid_cells(6, lat.material, 5)):
        b = k % 3
        vals = []
        for sgn in (1, -1):
            F = base.copy()
            F[b].reshape(-1)[c] += sgn * h
            lat.force_field = F
            f = f0.copy()
            lat.step(f, n)
            vals.append(lat.loss(f, obj))
        lat.force_field = base
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dF[b].reshape(-1)[c]) <= 1e-6 * abs(fd) + 1e-11


def test_force_gradient_sums_to_the_uniform_force_derivative(oracle):
    shape = (4, 6, 8)
    lat, f0 = _channel(oracle, 1, shape, moving=True)
    n = 20
    obj = (0, shape[2] - 1, 0)
    loss, dg, dtau, dF = lat.adjoint(f0, n, obj, want_dforce=True)
    fl = lat.material == I.FLUID
    for b in range(3):
        e = np.zeros((3,) + shape)
        e[b][fl] = 1.0
        _, dl = lat.tangent(f0, n, obj, dforce=e)
        assert abs(float(dF[b].sum()) - dl) <= 1e-11 * abs(dl)
