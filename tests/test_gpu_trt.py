"""GPU parity of the TRT collision (olb_set_trt) against the oracle's TRT:
populations within 1e-12 (FP64) and 1e-5 (FP32) relative, both streaming patterns,
the one-cell-per-thread kernel (odd nx) and the paired kernel (even nx), moving
walls, Guo force and porosity; FP16 within its storage bound; the exact Poiseuille
parabola at Lambda = 3/16; the adjoint of the TRT map against the oracle's TRT
adjoint (FP64 to 1e-10), against central differences, and with reduced storage."""
import dataclasses

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import Case, assert_cells_close, cavity_case, porous_channel_case, rel_err

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


def _compare(oracle, case, steps, dtype, scheme, tol):
    lat_o = case.oracle(oracle)
    f = case.oracle_state(lat_o)
    lat_o.step(f, steps)
    g = case.gpu(dtype, scheme)
    g.step(steps)
    fg = g.get_populations().cpu().numpy()
    g.close()
    err = rel_err(fg, f, case.material == I.FLUID)
    assert err <= tol, err
    return err


TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 2e-3}


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("magic", [3.0 / 16.0, 1.0 / 12.0])
def test_trt_cavity_odd_nx(oracle, olb, dtype, scheme, magic):
    case = dataclasses.replace(cavity_case(37, 29, 23, tau=0.58), collision="trt", magic=magic)
    _compare(oracle, case, 61, dtype, scheme, TOL[dtype])


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16"])
@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_trt_forced_porous_channel_even_nx(oracle, olb, dtype, scheme):
    case = dataclasses.replace(porous_channel_case(nx=40, ny=14, nz=11, moving=True), collision="trt",
                               magic=3.0 / 16.0)
    _compare(oracle, case, 50, dtype, scheme, TOL[dtype])


def test_trt_cavity_paired_kernel_rows_of_one_tile(oracle, olb):
    case = dataclasses.replace(cavity_case(64, 21, 13, lid=0.08), collision="trt", magic=0.3)
    _compare(oracle, case, 41, "f32", "pull", 1e-5)
    _compare(oracle, case, 40, "f64", "aa", 1e-12)


def test_trt_d2q9(oracle, olb):
    case = dataclasses.replace(porous_channel_case(nx=45, ny=13, d=0, moving=True), collision="trt",
                               magic=3.0 / 16.0)
    _compare(oracle, case, 90, "f64", "pull", 1e-12)
    _compare(oracle, case, 91, "f32", "aa", 1e-5)


@pytest.mark.parametrize("tau", [0.6, 1.5])
def test_trt_poiseuille_exact_on_the_gpu(olb, tau):
    import torch

    ny, F = 12, 1e-6
    m = I.plates(2, ny, 2)
    lat = olb.Lattice(olb.D3Q19, (2, ny, 2), dtype="f64", scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1 | 4)
    lat.set_trt(tau, 3.0 / 16.0)
    lat.set_force((F, 0.0, 0.0))
    lat.init_equilibrium()
    prev = None
    for _ in range(200):
        lat.step(500)
        _, u = lat.moments()
        prof = u[0, 0, 1:-1, 0].cpu().numpy()
        if prev is not None and np.max(np.abs(prof - prev)) <= 1e-15 * prof.max():
            break
        prev = prof
    y = np.arange(1, ny - 1, dtype=float)
    nu = I.viscosity(tau)
    exact = F / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
    assert np.max(np.abs(prof - exact)) <= 1e-9 * exact.max()
    lat.close()


@pytest.mark.parametrize("d,moving", [(1, False), (0, True), (1, True)])
@pytest.mark.parametrize("magic", [3.0 / 16.0, 1.0 / 12.0])
def test_trt_adjoint_f64_matches_oracle(oracle, olb, d, moving, magic):
    """The GPU adjoint of the TRT map (moment form) against the oracle's explicit TRT
    Jacobian: loss, dL/dgamma and dL/dtau at fixed magic parameter."""
    case = dataclasses.replace(porous_channel_case(nx=22, ny=10, nz=8, d=d, moving=moving),
                               collision="trt", magic=magic)
    steps, K = 23, 7
    obj = (0, case.shape[2] - 1, 0)
    lat = case.oracle(oracle)
    lo, go, to = lat.adjoint(case.oracle_state(lat), steps, obj)
    g = case.gpu("f64", "pull")
    lg, gg, tg = g.adjoint_run(steps, K, obj)
    gg = gg.cpu().numpy()
    g.close()
    assert abs(lg - lo) <= 1e-13 * abs(lo)
    assert np.max(np.abs(gg - go)) <= 1e-10 * np.max(np.abs(go))
    assert abs(tg - to) <= 1e-10 * abs(to)


def test_trt_adjoint_misfit_f64_matches_oracle(oracle, olb):
    case = dataclasses.replace(porous_channel_case(nx=20, ny=10, nz=8, moving=True), collision="trt",
                               magic=3.0 / 16.0)
    steps = 19
    target = 0.01 * (I.uniform(31, (3,) + case.shape) - 0.5)
    region = (I.uniform(32, case.shape) < 0.5).astype(np.uint8)
    lat = case.oracle(oracle)
    lo, go, to = lat.adjoint(case.oracle_state(lat), steps, oracle.Misfit(target, region))
    g = case.gpu("f64", "pull")
    lg, gg, tg = g.adjoint_run_misfit(steps, 5, target, region)
    gg = gg.cpu().numpy()
    g.close()
    assert abs(lg - lo) <= 1e-12 * abs(lo)
    assert np.max(np.abs(gg - go)) <= 1e-10 * np.max(np.abs(go))
    assert abs(tg - to) <= 1e-10 * abs(to)


def test_trt_adjoint_matches_gpu_central_differences(olb):
    """dL/dgamma and dL/dtau (magic parameter fixed) of the TRT map against central
    differences of FP64 forward runs on the GPU."""
    import torch

    case = dataclasses.replace(porous_channel_case(nx=24, ny=11, nz=9), collision="trt", magic=3.0 / 16.0)
    steps = 30
    obj = (0, case.shape[2] - 1, 0)
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    loss, dg, dtau = g.adjoint_run(steps, 8, obj)
    dg = dg.cpu().numpy().reshape(-1)

    def run(gamma=None, tau=None):
        g.set_porosity(torch.from_numpy((gamma if gamma is not None else case.gamma).reshape(-1).copy()).cuda())
        g.set_trt(tau if tau is not None else case.tau, case.magic)
        g.set_populations(f0)
        g.step(steps)
        _, u = g.moments()
        plane = torch.from_numpy(case.material[:, :, -1] == I.FLUID).cuda()
        return float(u[0, :, :, -1][plane].mean())

    h = 1e-5
    for c in I.random_fluid_cells(4, case.material, 8):
        gp = case.gamma.copy().reshape(-1)
        gm = gp.copy()
        gp[c] += h
        gm[c] -= h
        fd = (run(gamma=gp.reshape(case.shape)) - run(gamma=gm.reshape(case.shape))) / (2 * h)
        assert abs(fd - dg[c]) <= 1e-4 * abs(fd) + 1e-15
    ht = 1e-6
    fd = (run(tau=case.tau + ht) - run(tau=case.tau - ht)) / (2 * ht)
    assert abs(fd - dtau) <= 1e-4 * abs(fd)
    g.close()


@pytest.mark.parametrize("dtype,scheme", [("f32", "pull"), ("f32", "aa"), ("f16", "pull")])
def test_trt_adjoint_reduced_storage(oracle, olb, dtype, scheme):
    case = dataclasses.replace(porous_channel_case(nx=30, ny=12, nz=10, moving=True), collision="trt",
                               magic=3.0 / 16.0)
    steps = 40
    obj = (0, case.shape[2] - 1, 0)
    lat = case.oracle(oracle)
    lo, go, to = lat.adjoint(case.oracle_state(lat), steps, obj)
    g = case.gpu(dtype, scheme)
    lg, gg, tg = g.adjoint_run(steps, 9, obj)
    gg = gg.cpu().numpy()
    g.close()
    tol, floor = {"f32": (1e-4, 1e-6), "f16": (2e-2, 5e-4)}[dtype]
    assert abs(lg - lo) <= tol * abs(lo)
    assert_cells_close(gg, go, tol, floor)
    assert abs(tg - to) <= tol * abs(to)


def test_switching_collision_between_adjoint_runs(olb):
    """BGK and TRT runs on one handle: each adjoint follows the collision selected
    when it starts, and TRT at Lambda = (tau - 1/2)^2 gives the BGK loss and
    dL/dgamma (not dL/dtau: TRT's holds Lambda fixed while BGK's moves it with tau)."""
    case = porous_channel_case(nx=16, ny=8, nz=6)
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    obj = (0, 15, 0)
    g.set_populations(f0)  # every run starts from the same stored state
    lb, gb, tb = g.adjoint_run(9, 4, obj)
    g.set_trt(case.tau, (case.tau - 0.5) ** 2)
    g.set_populations(f0)
    lt, gt, tt = g.adjoint_run(9, 4, obj)
    g.set_bgk(case.tau)
    g.set_populations(f0)
    lb2, gb2, tb2 = g.adjoint_run(9, 4, obj)
    g.close()
    gb, gt, gb2 = (x.cpu().numpy() for x in (gb, gt, gb2))
    assert lb2 == lb and np.array_equal(gb2, gb) and tb2 == tb
    assert abs(lt - lb) <= 1e-14 * abs(lb)
    assert np.max(np.abs(gt - gb)) <= 1e-11 * np.max(np.abs(gb))
    assert np.isfinite(tt) and tt != tb
    with pytest.raises(olb.OlbError):
        g2 = case.gpu("f64", "pull")
        try:
            g2.set_trt(0.8, 0.0)
        finally:
            g2.close()
