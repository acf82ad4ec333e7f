"""olb_statistics_noalloc: the statistics reduction for callers that cannot
allocate device memory (their GPU memory is held by another allocator, or they
cannot accept cudaMalloc's device-wide synchronisation).  It keeps its partial
sums in a fixed array inside the library instead of allocating.

Checked through the C ABI against the existing entry point olb_diagnostics and
against the oracle's statistics of the same population array, on two calls in
a row (the second on a later state, so a stale partial sum left by the first
call would show), within the FP64 tolerances of the other statistics tests; once
with a material array and a force, once on an all-fluid periodic lattice with
neither (NULL material: every cell fluid; NULL force: F = 0).  This file is
collected last so that a run stopping at its first failure has already run every
other test.
"""
import ctypes

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


def _noalloc(olb, lat, f, material, force, stream):
    import torch

    out = torch.full((7,), float("nan"), dtype=torch.float64, device="cuda")
    F = None if force is None else (ctypes.c_double * 3)(*force)
    mat = None if material is None else material.data_ptr()
    rc = olb.load().olb_statistics_noalloc(lat.descriptor, lat.nx, lat.ny, lat.nz, f.data_ptr(),
                                           mat, F, out.data_ptr(),
                                           ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0, olb.load().olb_last_error().decode()
    stream.synchronize()
    return out.cpu().numpy()


def _agree(a, b):
    assert abs(a[0] - b[0]) <= 1e-12 * abs(b[0])                      # mass
    # momentum: a component that cancels over the cells (a flow symmetric in it) is
    # FP64 rounding noise whose value depends on the order of the sum, so it is
    # compared on the scale of sum_x |j(x)|, which sqrt(sum rho * sum rho |u|^2)
    # bounds (Cauchy-Schwarz; the energy is half the second sum)
    scale = np.sqrt(2.0 * b[0] * b[4])
    assert np.all(np.abs(a[1:4] - b[1:4]) <= 1e-9 * np.abs(b[1:4]) + 1e-13 * scale)
    assert abs(a[4] - b[4]) <= 1e-10 * abs(b[4])                      # energy
    assert abs(a[5] - b[5]) <= 1e-12 * abs(b[5])                      # max |u|
    assert a[6] == b[6] == 0


def _oracle_stats(oracle, d, m, periodic, force, f):
    o = oracle.Lattice(d, m, 0.6, periodic=periodic, force=force or (0.0, 0.0, 0.0))
    q = 19 if d == 1 else 9
    return o.diagnostics(np.ascontiguousarray(f.cpu().numpy().reshape((q,) + m.shape)))


@pytest.mark.parametrize("d,shape,walls", [(1, (30, 22, 17), True), (0, (45, 33, 1), True),
                                           (1, (24, 18, 14), False), (0, (40, 28, 1), False)])
def test_noalloc_statistics_match_diagnostics_twice(olb, oracle, d, shape, walls):
    """walls=True: a cavity with a moving lid, a material array and a force.
    walls=False: an all-fluid periodic vortex with NULL material and NULL force."""
    import torch

    nx, ny, nz = shape
    lat = olb.Lattice(d, shape, dtype="f64", scheme="pull")
    if walls:
        m = I.cavity_box(nx, ny, nz)
        periodic = 0
        force = (2e-6, -1e-6, 0.0)
        lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), periodic)
        lat.set_wall_velocity(I.LID, (0.05, 0.0, 0.0))
        lat.set_force(force)
        lat.set_bgk(0.6)
        lat.init_equilibrium()
        mat = torch.from_numpy(m.reshape(-1).copy()).cuda()
    else:
        m = I.periodic_box(nx, ny, nz)
        periodic = 7 if d == 1 else 3
        force = None
        lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), periodic)
        lat.set_bgk(0.6)
        rho, u = I.tgv3d(nx, 0.02) if d == 1 else I.tgv2d(nx, 0.02)
        rho, u = rho[:nz, :ny, :nx], u[:, :nz, :ny, :nx]
        lat.init_equilibrium(torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).cuda())
        mat = None
    stream = torch.cuda.current_stream()
    for steps in (25, 40):  # two calls in a row, on different states
        lat.step(steps)
        f = lat.get_populations()
        got = _noalloc(olb, lat, f, mat, force, stream)
        _agree(got, lat.diagnostics())
        _agree(got, _oracle_stats(oracle, d, m, periodic, force, f))
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_fixed_array(olb):
    import torch

    dummy = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(7, dtype=torch.float64, device="cuda")
    lib = olb.load()
    rc = lib.olb_statistics_noalloc(1, 257, 256, 256, dummy.data_ptr(), None, None, out.data_ptr(), None)
    assert rc == -1
    assert "16,777,216" in lib.olb_last_error().decode()
    # host memory is refused rather than staged (staging would allocate)
    host = np.zeros(19 * 8, dtype=np.float64)
    rc = lib.olb_statistics_noalloc(1, 2, 2, 2, host.ctypes.data, None, None, out.data_ptr(), None)
    assert rc == -1
