"""GPU parity of the velocity-misfit adjoint (olb_adjoint_run_misfit: J = 1/2 sum
over a region of |u - u*|^2, the objective of the guide's domainIdentification3d)
against the oracle's adjoint, through the autograd wrapper, and the porosity
identification driver on the GPU."""
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


def _target(oracle, case, steps, seed=5):
    """u* = final velocity of an oracle run with a perturbed porosity, plus a small
    seeded offset; region = an interior box."""
    lat = case.oracle(oracle)
    lat.gamma = np.clip(case.gamma * (0.8 + 0.4 * I.uniform(seed, case.shape)), 0.0, 1.0)
    f = case.oracle_state(lat)
    lat.step(f, steps)
    _, u = lat.moments(f)
    u_t = np.ascontiguousarray(u + 1e-3 * (I.uniform(seed + 1, u.shape) - 0.5))
    nz, ny, nx = case.shape
    region = np.zeros(case.shape, np.uint8)
    region[:, 1:ny - 1, nx // 3:] = 1
    return u_t, region


def _oracle(oracle, case, steps, u_t, region):
    lat = case.oracle(oracle)
    f0 = case.oracle_state(lat)
    return lat.adjoint(f0, steps, oracle.Misfit(u_t, None if region is None else region.astype(bool)))


@pytest.mark.parametrize("d,moving", [(1, False), (0, False), (1, True), (0, True)])
@pytest.mark.parametrize("K", [1, 9])
def test_misfit_adjoint_f64_matches_oracle(oracle, olb, d, moving, K):
    case = porous_channel_case(nx=22, ny=10, nz=8, d=d, moving=moving)
    steps = 23
    u_t, region = _target(oracle, case, steps)
    lo, go, to = _oracle(oracle, case, steps, u_t, region)
    g = case.gpu("f64", "pull")
    lg, gg, tg = g.adjoint_run_misfit(steps, K, u_t, region)
    gg = gg.cpu().numpy()
    assert abs(lg - lo) <= 1e-12 * abs(lo)
    assert np.max(np.abs(gg - go)) <= 1e-10 * np.max(np.abs(go))
    assert abs(tg - to) <= 1e-10 * abs(to)
    assert g.counters()[0] == steps
    g.close()


def test_misfit_region_forms_agree(oracle, olb):
    """Region as a device tensor, as a host array, and absent (every fluid cell);
    target as a device tensor or host array."""
    import torch

    case = porous_channel_case(nx=20, ny=10, nz=8)
    steps = 17
    u_t, region = _target(oracle, case, steps)
    out = []
    for ut, rg in ((u_t, region), (torch.from_numpy(u_t).cuda(), torch.from_numpy(region).cuda())):
        g = case.gpu("f64", "pull")
        out.append(g.adjoint_run_misfit(steps, 5, ut, rg))
        g.close()
    assert out[0][0] == out[1][0] and torch.equal(out[0][1], out[1][1]) and out[0][2] == out[1][2]
    lo, go, to = _oracle(oracle, case, steps, u_t, None)
    g = case.gpu("f64", "pull")
    lg, gg, tg = g.adjoint_run_misfit(steps, 5, u_t, None)
    assert abs(lg - lo) <= 1e-12 * abs(lo)
    assert np.max(np.abs(gg.cpu().numpy() - go)) <= 1e-10 * np.max(np.abs(go))
    g.close()


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_misfit_adjoint_reduced_storage(oracle, olb, dtype):
    case = porous_channel_case(nx=30, ny=12, nz=10)
    steps = 40
    u_t, region = _target(oracle, case, steps)
    lo, go, to = _oracle(oracle, case, steps, u_t, region)
    g = case.gpu(dtype, "pull")
    lg, gg, tg = g.adjoint_run_misfit(steps, 9, u_t, region)
    gg = gg.cpu().numpy()
    tol, floor = (1e-4, 1e-6) if dtype == "f32" else (2e-2, 5e-4)
    assert abs(lg - lo) <= tol * abs(lo)
    assert_cells_close(gg, go, tol, floor)
    assert abs(tg - to) <= tol * abs(to)
    g.close()


def test_misfit_rejects_bad_arguments(olb):
    import torch

    case = porous_channel_case(nx=12, ny=8, nz=6)
    g = case.gpu("f64", "pull")
    u_t = np.zeros((3,) + case.shape)
    region = np.zeros(case.shape, np.uint8)
    region[:, 0, :] = 1  # wall cells only
    with pytest.raises(olb.OlbError):
        g.adjoint_run_misfit(5, 2, u_t, region)
    with pytest.raises(olb.OlbError):
        g.adjoint_run_misfit(0, 2, u_t, None)
    lib = olb.load()
    assert lib.olb_adjoint_run_misfit(g.handle, 5, 2, None, None, None, None, None) == -1
    assert g.counters()[0] == 0  # nothing ran
    g.close()


def test_misfit_autograd_function(oracle, olb):
    import torch

    case = porous_channel_case(nx=20, ny=10, nz=8)
    steps = 15
    u_t, region = _target(oracle, case, steps)
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    gamma = torch.from_numpy(case.gamma.copy()).cuda().requires_grad_(True)
    tau = torch.tensor(case.tau, dtype=torch.float64, requires_grad=True)
    loss = olb.velocity_misfit_loss(g, gamma, tau, f0, steps, 4, u_t, region)
    loss.backward()
    g.set_porosity(torch.from_numpy(case.gamma.reshape(-1).copy()).cuda())
    g.set_bgk(case.tau)
    g.set_populations(f0)
    l2, dg, dtau = g.adjoint_run_misfit(steps, 4, u_t, region)
    assert float(loss.detach()) == l2
    assert torch.equal(gamma.grad, dg.view_as(gamma))
    assert float(tau.grad) == dtau
    g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_identify_a_porous_block_on_the_gpu(olb, dtype):
    """Domain identification (domainIdentification3d in small): a cube of low
    porosity in a forced channel is recovered from the flow around it with the
    GPU adjoint and torch's L-BFGS."""
    import torch

    from paper_2307_11752_gb300 import opti

    nx, ny, nz, steps = 32, 14, 14, 200
    m = I.channel(nx, ny, nz)
    tau = 0.8
    F = (I.channel_force(ny, tau, 0.05), 0.0, 0.0)
    lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype=dtype, scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    lat.set_bgk(tau)
    lat.set_force(F)
    lat.init_equilibrium()
    f0 = lat.get_populations().clone()
    truth = torch.ones((nz, ny, nx), dtype=torch.float64, device="cuda")
    truth[5:9, 5:9, 12:16] = 0.05
    lat.set_porosity(truth.reshape(-1).contiguous())
    lat.step(steps)
    _, u_ref = lat.moments()
    fl = torch.from_numpy(m == I.FLUID).cuda()
    design = torch.zeros_like(fl)
    design[3:11, 3:11, 9:19] = True
    design &= fl
    region = (fl & ~design).to(torch.uint8)
    tau_t = torch.tensor(tau, dtype=torch.float64)

    def evaluate(gamma):
        return olb.velocity_misfit_loss(lat, gamma, tau_t, f0, steps, 50, u_ref, region)

    res = opti.identify_porosity(evaluate, torch.ones_like(truth), design, 0.7, iterations=15)
    J = res.objective
    assert J[-1] <= 1e-3 * J[0], J
    inside = truth < 0.5
    assert float(res.gamma[inside].mean()) < 0.5 < float(res.gamma[design & ~inside].mean())
    lat.close()
