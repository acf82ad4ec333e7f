"""Lattice-level pins of the oracle: streaming against np.roll, permutation
property of streaming with bounce-back, rest-state fixed point, conservation
laws, and the rest-state statistics line of the guide's console listing."""
import os

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lat(oracle, d, material, tau=0.8, periodic=7, **kw):
    return oracle.Lattice(d, material, tau, periodic=periodic, **kw)


@pytest.mark.parametrize("d,shape", [(0, (1, 5, 7)), (1, (3, 5, 7))])
def test_periodic_streaming_is_a_roll(oracle, d, shape):
    """Streaming equation f_i(x + c_i) = f*_i(x) on a fully periodic box equals a
    cyclic shift of every population plane by c_i (numpy's roll)."""
    lat = _lat(oracle, d, I.periodic_box(shape[2], shape[1], shape[0]))
    dim, q, c, *_ = oracle.descriptor(d)
    fs = I.uniform(3, (q,) + shape)
    out = lat.stream(fs, fs)
    for i in range(q):
        expect = np.roll(fs[i], shift=(c[i][2], c[i][1], c[i][0]), axis=(0, 1, 2))
        assert np.array_equal(out[i], expect)


@pytest.mark.parametrize("d", [0, 1])
def test_streaming_with_walls_is_a_permutation(oracle, d):
    """Without moving walls streaming only moves values: its output on fluid cells
    is a permutation of its input on fluid cells, and the transpose undoes it."""
    n = 6
    m = I.cavity(n, dim=2 if d == 0 else 3)
    m[m == I.LID] = I.WALL
    lat = _lat(oracle, d, m, periodic=0)
    q = lat.q
    fs = I.uniform(9, (q,) + m.shape)
    out = lat.stream(fs, fs)
    fl = m == I.FLUID
    assert np.array_equal(np.sort(out[:, fl].ravel()), np.sort(fs[:, fl].ravel()))
    back, direct = lat.stream_adjoint(out)
    assert np.array_equal(back[:, fl], fs[:, fl])
    assert np.all(direct == 0)


@pytest.mark.parametrize("d", [0, 1])
def test_rest_state_is_a_fixed_point(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    m = I.cavity(8, dim=2 if d == 0 else 3)
    m[m == I.LID] = I.WALL
    lat = _lat(oracle, d, m, periodic=0)
    f = lat.init_equilibrium(*I.rest(m.shape))
    lat.step(f, 50)
    fl = m == I.FLUID
    assert np.max(np.abs(f[:, fl] - w[:, None])) <= 4e-16


@pytest.mark.parametrize("d", [0, 1])
def test_rest_statistics_match_console_listing(oracle, d):
    """avRho = 1 and avEnergy = 0 for a lattice initialised at rest, as the
    bstep2d console listing prints at step 0."""
    with open(os.path.join(GOLDEN, "console_bstep2d.txt")) as fh:
        line = [l for l in fh if not l.startswith("#")][0].split()
    golden = {k: float(v) for k, v in (t.split("=") for t in line)}
    m = I.channel(6, 5, 1 if d == 0 else 4)
    lat = _lat(oracle, d, m, periodic=1)
    f = lat.init_equilibrium(*I.rest(m.shape))
    diag = lat.diagnostics(f)
    nfluid = int((m == I.FLUID).sum())
    assert abs(diag[0] / nfluid - golden["avRho"]) < 1e-15
    assert abs(diag[4] / nfluid - golden["avEnergy"]) < 1e-30
    assert diag[5] < 1e-15 and diag[6] == 0.0


@pytest.mark.parametrize("d", [0, 1])
def test_mass_conserved_in_lid_driven_cavity(oracle, d):
    """Halfway bounce-back, moving lid (whole top plane, edges included) and no
    periodic axis: total mass is conserved to 1e-13 relative."""
    n = 10
    m = I.cavity(n, dim=2 if d == 0 else 3)
    wu = np.zeros((256, 3))
    wu[I.LID] = (0.05, 0, 0)
    lat = _lat(oracle, d, m, tau=0.56, periodic=0, wall_u=wu)
    f = lat.init_equilibrium(*I.rest(m.shape)) + I.population_noise(1, lat.q, m, 1e-6)
    m0 = lat.diagnostics(f)[0]
    lat.step(f, 200)
    diag = lat.diagnostics(f)
    assert abs(diag[0] - m0) / m0 < 1e-13
    assert diag[5] > 1e-3  # the lid has set the fluid in motion


@pytest.mark.parametrize("d", [0, 1])
def test_momentum_conserved_periodic_and_forced(oracle, d):
    shape = (1, 6, 8) if d == 0 else (4, 5, 6)
    m = I.periodic_box(shape[2], shape[1], shape[0])
    lat = _lat(oracle, d, m)
    dim, q, *_ = oracle.descriptor(d)
    rho = 1 + 0.01 * (I.uniform(2, shape) - 0.5)
    u = 0.02 * (I.uniform(3, (3,) + shape) - 0.5)
    if d == 0:
        u[2] = 0
    f = lat.init_equilibrium(rho, u)
    j0 = lat.diagnostics(f)[1:4].copy()
    lat.step(f, 100)
    assert np.allclose(lat.diagnostics(f)[1:4], j0, rtol=0, atol=1e-14)
    # With a uniform Guo force every fluid cell gains exactly F per step.
    F = np.array([2e-5, -1e-5, 3e-5 if d == 1 else 0.0])
    latF = _lat(oracle, d, m, force=F)
    f = latF.init_equilibrium(rho, u)
    j0 = latF.diagnostics(f)[1:4].copy()
    latF.step(f, 40)
    assert np.allclose(latF.diagnostics(f)[1:4] - j0, 40 * m.size * F, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("d", [0, 1])
def test_step_commutes_with_periodic_translation(oracle, d):
    shape = (1, 6, 7) if d == 0 else (5, 6, 7)
    m = I.periodic_box(shape[2], shape[1], shape[0])
    lat = _lat(oracle, d, m, force=(1e-5, 2e-5, 0))
    f = 1.0 / lat.q + 1e-3 * I.uniform(4, (lat.q,) + shape)
    g = np.roll(f, shift=(1, 2, 3), axis=(1, 2, 3)).copy()
    lat.step(f, 5)
    lat.step(g, 5)
    assert np.array_equal(np.roll(f, shift=(1, 2, 3), axis=(1, 2, 3)), g)
