"""GPU parity of the TRT collision (olb_set_trt) against the oracle's TRT:
populations within 1e-12 (FP64) and 1e-5 (FP32) relative, both streaming patterns,
the one-cell-per-thread kernel (odd nx) and the paired kernel (even nx), moving
walls, Guo force and porosity; FP16 within its storage bound; the exact Poiseuille
parabola at Lambda = 3/16; the adjoint refuses TRT."""
import dataclasses

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import Case, cavity_case, porous_channel_case, rel_err

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


def test_adjoint_refuses_trt_and_bgk_restores(olb):
    case = dataclasses.replace(porous_channel_case(nx=12, ny=8, nz=6), collision="trt")
    g = case.gpu("f64", "pull")
    with pytest.raises(olb.OlbError) as e:
        g.adjoint_run(3, 2, (0, 11, 0))
    assert e.value.status == -7
    with pytest.raises(olb.OlbError) as e:
        g.adjoint_run_misfit(3, 2, np.zeros((3,) + case.shape), None)
    assert e.value.status == -7
    with pytest.raises(olb.OlbError):
        g.set_trt(0.8, 0.0)
    g.set_bgk(case.tau)
    g.adjoint_run(3, 2, (0, 11, 0))
    g.close()
