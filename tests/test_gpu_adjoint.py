"""GPU parity of the checkpointed discrete adjoint (olb_adjoint_run) against the
oracle's adjoint, against central difference quotients of the GPU's own FP64
forward runs, and through the torch.autograd wrapper."""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import assert_cells_close, porous_channel_case

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


def _oracle_adjoint(oracle, case, steps, obj):
    lat = case.oracle(oracle)
    f0 = case.oracle_state(lat)
    return lat.adjoint(f0, steps, obj)


@pytest.mark.parametrize("d,moving", [(1, False), (0, False), (1, True), (0, True)])
@pytest.mark.parametrize("K", [1, 7, 50])
def test_adjoint_f64_matches_oracle(oracle, olb, d, moving, K):
    case = porous_channel_case(nx=22, ny=10, nz=8, d=d, moving=moving)
    steps = 23
    obj = (0, case.shape[2] - 1, 0)
    lo, go, to = _oracle_adjoint(oracle, case, steps, obj)
    g = case.gpu("f64", "pull")
    lg, gg, tg = g.adjoint_run(steps, K, obj)
    gg = gg.cpu().numpy()
    assert abs(lg - lo) <= 1e-13 * abs(lo)
    assert np.max(np.abs(gg - go)) <= 1e-10 * np.max(np.abs(go))
    assert abs(tg - to) <= 1e-10 * abs(to)
    assert g.counters()[0] == steps  # the handle ends in the final forward state
    g.close()


@pytest.mark.parametrize("scheme", ["pull", "aa"])
@pytest.mark.parametrize("moving", [False, True])
def test_adjoint_f32_storage_within_1e4(oracle, olb, scheme, moving):
    """Per cell: |dL/dgamma - oracle| <= 1e-4 |oracle| + 1e-6 max|oracle| (the floor
    covers the few cells whose gradient is ~1e-5 of the largest, next to a moving
    wall)."""
    case = porous_channel_case(nx=30, ny=12, nz=10, moving=moving)
    steps = 40
    obj = (0, case.shape[2] - 1, 0)
    lo, go, to = _oracle_adjoint(oracle, case, steps, obj)
    g = case.gpu("f32", scheme)
    g.step(0)
    lg, gg, tg = g.adjoint_run(steps, 9, obj)
    gg = gg.cpu().numpy()
    assert abs(lg - lo) <= 1e-5 * abs(lo)
    assert_cells_close(gg, go, 1e-4, 1e-6)
    assert abs(tg - to) <= 2e-5 * abs(to)
    g.close()


def test_adjoint_matches_gpu_central_differences(olb):
    """dL/dgamma at seeded random fluid cells and dL/dtau against central
    difference quotients (OptiCaseCDQ) of FP64 forward runs on the GPU."""
    case = porous_channel_case(nx=26, ny=12, nz=9)
    steps = 30
    obj = (0, case.shape[2] - 1, 0)
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    loss, dg, dtau = g.adjoint_run(steps, 8, obj)
    dg = dg.cpu().numpy().reshape(-1)
    import torch

    def run(gamma=None, tau=None):
        g.set_porosity(torch.from_numpy((gamma if gamma is not None else case.gamma).reshape(-1).copy()).cuda())
        g.set_bgk(tau if tau is not None else case.tau)
        g.set_populations(f0)
        l, _, _ = g.adjoint_run(steps, steps, obj)
        return l

    h = 1e-5
    for c in I.random_fluid_cells(3, case.material, 8):
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


def test_autograd_function(olb):
    import torch

    case = porous_channel_case(nx=20, ny=10, nz=8)
    obj = (0, case.shape[2] - 1, 0)
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    gamma = torch.from_numpy(case.gamma.copy()).cuda().requires_grad_(True)
    tau = torch.tensor(case.tau, dtype=torch.float64, requires_grad=True)
    loss = olb.plane_velocity_loss(g, gamma, tau, f0, 15, 4, obj)
    loss.backward()
    g.set_porosity(torch.from_numpy(case.gamma.reshape(-1).copy()).cuda())
    g.set_bgk(case.tau)
    g.set_populations(f0)
    l2, dg, dtau = g.adjoint_run(15, 4, obj)
    assert float(loss.detach()) == l2
    assert torch.equal(gamma.grad, dg.view_as(gamma))
    assert float(tau.grad) == dtau
    g.close()
