"""GPU parity of the forward collide-and-stream path against the FP64 oracle.

Bars: populations within 1e-12 relative (max |f_gpu - f_oracle| / max |f_oracle|)
for FP64 storage and 1e-5 for FP32 storage; both streaming patterns, even and
odd step counts, ragged lattice sizes (no dimension a multiple of the 32-wide
thread row), periodic, bounce-back and moving-wall links, Guo force and porosity.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import (Case, cavity_case, porous_channel_case, rel_err, tgv2d_case,
                    tgv3d_case)

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3}


@pytest.fixture(scope="module")
def olb():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2307_11752_gb300 import build, olb as _olb
    build.build()
    _olb.load()
    return _olb


def _compare(oracle, case, steps, dtype, scheme, tol=None, split=None):
    lat_o = case.oracle(oracle)
    f = case.oracle_state(lat_o)
    lat_o.step(f, steps)
    g = case.gpu(dtype, scheme)
    if split:
        for k in split:
            g.step(k)
    else:
        g.step(steps)
    fg = g.get_populations().cpu().numpy()
    g.close()
    fl = case.material == I.FLUID
    err = rel_err(fg, f, fl)
    assert err <= (tol or TOL[dtype]), err
    return err, f, fg


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_tgv2d_64_f64(oracle, olb, scheme):
    """The D2Q9 64 x 64 vortex (tau 0.8, u0 0.01, 1000 steps) in FP64."""
    case = tgv2d_case()
    _, f, fg = _compare(oracle, case, 1000, "f64", scheme)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("steps", [60, 61])
def test_cavity_ragged(oracle, olb, dtype, scheme, steps):
    _compare(oracle, cavity_case(), steps, dtype, scheme)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_porous_forced_channel(oracle, olb, dtype, scheme):
    _compare(oracle, porous_channel_case(), 75, dtype, scheme)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_porous_channel_with_moving_wall_d2q9(oracle, olb, dtype):
    _compare(oracle, porous_channel_case(nx=45, ny=13, d=0, moving=True), 90, dtype, "pull")
    _compare(oracle, porous_channel_case(nx=45, ny=13, d=0, moving=True), 91, dtype, "aa")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_moving_walls_beyond_the_plane_form(oracle, olb, dtype, scheme):
    """Moving links that the link word cannot hold in plane form, next to cells
    whose links it can: a lid that stops short of the z edges (cells at its rim
    have links with c_y = +1 to the lid and to a fixed wall) and a second moving
    face x = nx - 1 with another velocity (cells at the shared edge see two moving
    materials)."""
    m = I.cavity_box(23, 19, 14)
    m[:, -1, :] = I.WALL
    m[1:-1, -1, :] = I.LID
    m[:, :, -1] = 4
    case = Case(1, m, 0, 0.58, walls={I.LID: (0.04, 0.0, 0.01), 4: (0.0, -0.02, 0.015)},
                noise=I.population_noise(9, 19, m, 1e-5))
    _compare(oracle, case, 37, dtype, scheme)


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_scattered_obstacles_and_partial_x_walls(oracle, olb, dtype, scheme):
    """Solid cells scattered at random (15 %), half-height walls on both x faces
    and a moving lid, periodic in z, even nx: every kind of pair of a wall cell and
    a fluid cell the paired kernels tell apart -- walls that cover a partner's whole
    side, walls with fluid next to them in the same column, wall cells with fluid on
    both sides -- in both store patterns."""
    nx, ny, nz = 32, 17, 12
    m = np.full((nz, ny, nx), I.FLUID, np.uint8)
    m[I.uniform(51, m.shape) < 0.15] = I.WALL
    m[:, : ny // 2, 0] = I.WALL
    m[:, ny // 2:, nx - 1] = I.WALL
    m[:, 0, :] = I.WALL
    m[:, -1, :] = I.LID
    case = Case(1, m, 4, 0.62, walls={I.LID: (0.04, 0.0, 0.01)}, noise=I.population_noise(52, 19, m, 1e-5))
    _compare(oracle, case, 43, dtype, scheme)


@pytest.mark.parametrize("dtype", ["f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_cavity_rows_of_one_tile(oracle, olb, dtype, scheme):
    """nx = 64: a row is exactly one tile of the paired kernel, and with walls on
    both x faces each warp holds one pair of a wall cell and a fluid cell.  The rows
    (21 x 13) do not fill the last block.  FP16 is held to its storage bound
    (shifted values carry 11 significant bits)."""
    case = cavity_case(64, 21, 13, lid=0.08)
    _compare(oracle, case, 40, dtype, scheme, tol=1e-5 if dtype == "f32" else 2e-3)
    _compare(oracle, case, 41, dtype, scheme, tol=1e-5 if dtype == "f32" else 2e-3)


def test_tgv3d_f64_and_f32(oracle, olb):
    case = tgv3d_case(24)
    _compare(oracle, case, 40, "f64", "pull")
    _compare(oracle, case, 41, "f32", "aa")


def test_scheme_switches_preserve_the_map(oracle, olb):
    """Changing pattern between batches (pull -> AA mid-pair -> pull) computes the
    same map as an uninterrupted run."""
    case = cavity_case(21, 18, 13)
    lat_o = case.oracle(oracle)
    f = case.oracle_state(lat_o)
    lat_o.step(f, 20)
    g = case.gpu("f64", "pull")
    g.step(5)
    g.set_scheme("aa")
    g.step(7)
    g.set_scheme("pull")
    g.step(3)
    g.set_scheme("aa")
    g.step(5)
    fg = g.get_populations().cpu().numpy()
    assert rel_err(fg, f, case.material == I.FLUID) <= 1e-12


def test_tiny_and_degenerate_lattices(oracle, olb):
    # 1 x 1 periodic D2Q9: every link returns to the same cell
    rho = np.array([[[1.01]]])
    u = np.zeros((3, 1, 1, 1))
    u[0] = 0.03
    case = Case(0, I.periodic_box(1, 1, 1), 3, 0.7, force=(1e-4, -2e-4, 0), rho=rho, u=u)
    _compare(oracle, case, 9, "f64", "pull")
    _compare(oracle, case, 9, "f64", "aa")
    # one-cell-wide periodic channel (Poiseuille set-up), D2Q9 and D3Q19
    for d, shape in ((0, (1, 11, 1)), (1, (1, 9, 2))):
        m = I.plates(shape[0], shape[1], shape[2])
        case = Case(d, m, 1 if d == 0 else 1 | 4, 0.9, force=(1e-5, 0, 0))
        _compare(oracle, case, 33, "f64", "pull")
        _compare(oracle, case, 33, "f64", "aa")
    # no periodic axis and no wall cells: the domain edge itself bounces back
    m = I.periodic_box(7, 5, 3)
    rho, u = I.rest(m.shape)
    case = Case(1, m, 0, 0.8, rho=rho, u=u, noise=I.population_noise(4, 19, m, 1e-3))
    _compare(oracle, case, 12, "f64", "pull")
    _compare(oracle, case, 13, "f64", "aa")


def test_zero_steps_is_identity(oracle, olb):
    case = cavity_case(12, 10, 9)
    _compare(oracle, case, 0, "f64", "pull")


def test_rest_state_stays_all_zero_bits(olb):
    """Stored populations are f - w: the rest state is exactly zero for every storage
    type, so reading it back gives the weights bit for bit after any number of steps."""
    import torch

    for dtype in ("f64", "f32", "f16", "bf16"):
        for scheme in ("pull", "aa"):
            m = I.cavity_box(20, 17, 9)
            case = Case(1, m, 0, 0.6)
            g = case.gpu(dtype, scheme)
            g.step(25)
            f = g.get_populations().cpu().numpy()
            w = np.array([1 / 3] + [1 / 18] * 3 + [1 / 36] * 6 + [1 / 18] * 3 + [1 / 36] * 6)
            fl = m == I.FLUID
            assert np.array_equal(f[:, fl], np.broadcast_to(w[:, None], f[:, fl].shape))
            d = g.diagnostics()
            assert d[0] == fl.sum() and d[1] == 0 and d[4] == 0 and d[5] == 0
            g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_moments_and_diagnostics(oracle, olb, dtype):
    case = porous_channel_case(nx=33, ny=12, nz=10)
    lat_o = case.oracle(oracle)
    f = case.oracle_state(lat_o)
    lat_o.step(f, 31)
    g = case.gpu(dtype, "aa")
    g.step(31)
    rho, u = g.moments()
    ro, uo = lat_o.moments(f)
    tol = TOL[dtype]
    assert rel_err(rho.cpu().numpy(), ro) <= tol
    assert np.max(np.abs(u.cpu().numpy() - uo)) <= tol * 10 * np.max(np.abs(uo))
    dg = g.diagnostics()
    do = lat_o.diagnostics(f)
    assert abs(dg[0] - do[0]) <= 1e-12 * do[0] if dtype == "f64" else abs(dg[0] - do[0]) <= 1e-6 * do[0]
    assert np.allclose(dg[1:4], do[1:4], rtol=tol * 100, atol=tol * 1e-2)
    assert abs(dg[4] - do[4]) <= tol * 100 * do[4]
    assert abs(dg[5] - do[5]) <= tol * 10 * do[5]
    assert dg[6] == 0 and do[6] == 0
    g.close()


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_step_stats_are_those_of_the_last_collided_state(oracle, olb, scheme):
    case = cavity_case(19, 17, 15)
    lat_o = case.oracle(oracle)
    f = case.oracle_state(lat_o)
    lat_o.step(f, 14)  # the 15th step collides f(14)
    do = lat_o.diagnostics(f)
    g = case.gpu("f64", scheme)
    dg = g.step_stats(15)
    assert abs(dg[0] - do[0]) <= 1e-13 * do[0]
    assert np.allclose(dg[1:4], do[1:4], rtol=1e-9, atol=1e-15)
    assert abs(dg[4] - do[4]) <= 1e-10 * do[4]
    assert abs(dg[5] - do[5]) <= 1e-10 * do[5]
    assert g.counters()[0] == 15
    g.close()


def test_nonfinite_population_is_reported(olb):
    from paper_2307_11752_gb300 import olb as O
    import torch

    case = cavity_case(10, 9, 8)
    g = case.gpu("f32", "pull")
    f = g.get_populations()
    f[3, 4, 4, 4] = float("nan")
    g.set_populations(f)
    with pytest.raises(O.OlbError) as e:
        g.diagnostics()
    assert e.value.status == -5
    d = g.diagnostics(check=False)
    assert d[6] == 1
    g.close()


def test_invalid_arguments_leave_the_state_unchanged(olb):
    from paper_2307_11752_gb300 import olb as O

    case = cavity_case(10, 9, 8)
    g = case.gpu("f64", "pull")
    g.step(3)
    before = g.get_populations().cpu().numpy()
    for call in (lambda: g.set_bgk(0.5), lambda: g.set_bgk(float("nan")), lambda: g.step(-1),
                 lambda: g.set_wall_velocity(2, (0.1, 0, 0)),
                 lambda: g.adjoint_run(5, 2, (1, 0, 0))):
        with pytest.raises(O.OlbError) as e:
            call()
        assert e.value.status == -1
    with pytest.raises(O.OlbError):
        O._call("olb_set_material", g.handle, None, 0)
    assert np.array_equal(g.get_populations().cpu().numpy(), before)
    with pytest.raises(O.OlbError):
        O.Lattice(O.D2Q9, (4, 4, 2))
    g.close()


def test_host_and_device_arrays_agree(oracle, olb):
    import torch

    case = porous_channel_case(nx=20, ny=9, nz=7)
    g1 = case.gpu("f64", "pull")
    g2 = case.gpu("f64", "pull")
    f0 = g1.get_populations().cpu().numpy()
    g2.set_populations(np.ascontiguousarray(f0))          # host pointer
    g1.set_populations(torch.from_numpy(f0).cuda())        # device pointer
    g1.step(9)
    g2.step(9)
    host = np.zeros_like(f0)
    g2.get_populations(host)
    assert np.array_equal(g1.get_populations().cpu().numpy(), host)
    rho = np.zeros(case.material.shape)
    u = np.zeros((3,) + case.material.shape)
    g2.moments(rho, u)
    r1, u1 = g1.moments()
    assert np.array_equal(r1.cpu().numpy(), rho) and np.array_equal(u1.cpu().numpy(), u)
    g1.close()
    g2.close()
