"""GPU parity of the per-cell force field (olb_set_force_field) and of the adjoint
gradient with respect to it (olb_adjoint_gradients, dL/dF) against the oracle's
force-field map and adjoint: populations within 1e-12 (FP64) and 1e-5 (FP32)
relative; dL/dF, dL/dgamma and dL/dtau within 1e-10 (FP64) for the plane and the
misfit objectives, BGK and TRT, moving walls; dL/dF against central differences
of FP64 GPU runs; and force-field identification in the manner of the guide's
testFlowOpti3d (control: three force components at every cell)."""
import dataclasses

import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import porous_channel_case, rel_err

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


def _field(case, seed, scale=2e-5):
    """The case's uniform force plus a seeded per-cell part (z row 0 on D2Q9)."""
    F = scale * (I.uniform(seed, (3,) + case.shape) - 0.5)
    F += np.array(case.force).reshape(3, 1, 1, 1)
    if case.d == 0:
        F[2] = 0.0
    return np.ascontiguousarray(F)


def _pair(oracle, case, F):
    """Oracle lattice and initial state, and the GPU lattice, both with field F."""
    import torch

    lat = case.oracle(oracle)
    lat.force_field = F
    return lat, case.oracle_state(lat)


def _gpu(case, F, dtype, scheme="pull"):
    import torch

    g = case.gpu(dtype, scheme)
    g.set_force_field(torch.from_numpy(F.reshape(-1).copy()).cuda())
    return g


@pytest.mark.parametrize("dtype,scheme,nx,tol", [("f64", "pull", 24, 1e-12), ("f64", "aa", 23, 1e-12),
                                                 ("f32", "pull", 24, 1e-5), ("f32", "aa", 23, 1e-5)])
@pytest.mark.parametrize("d", [1, 0])
def test_force_field_forward_matches_oracle(oracle, olb, dtype, scheme, nx, tol, d):
    case = porous_channel_case(nx=nx, ny=11, nz=9, d=d, moving=True)
    F = _field(case, 7)
    lat, f = _pair(oracle, case, F)
    lat.step(f, 37)
    g = _gpu(case, F, dtype, scheme)
    g.step(37)
    fg = g.get_populations().cpu().numpy()
    fl = case.material == I.FLUID
    assert rel_err(fg, f, fl) <= tol
    # moments and statistics use the cell's own force in u = (j + F/2)/rho
    rho_o, u_o = lat.moments(f)
    _, u_g = g.moments()
    u_g = u_g.cpu().numpy()
    assert np.max(np.abs(u_g - u_o)[:, fl]) <= 100 * tol * np.max(np.abs(u_o[:, fl]))
    diag = g.diagnostics()
    ref = lat.diagnostics(f)
    assert abs(diag[4] - ref[4]) <= 100 * tol * ref[4]
    # removing the field restores the uniform force
    g.set_force_field(None)
    g.set_populations(lat.init_equilibrium(*I.rest(case.shape)))
    g.step(3)
    lat.force_field = None
    f2 = lat.init_equilibrium(*I.rest(case.shape))
    lat.step(f2, 3)
    assert rel_err(g.get_populations().cpu().numpy(), f2, fl) <= tol
    g.close()


@pytest.mark.parametrize("collision", ["bgk", "trt"])
@pytest.mark.parametrize("d,moving", [(1, True), (0, True), (1, False)])
@pytest.mark.parametrize("objective", ["plane", "misfit"])
def test_force_gradient_f64_matches_oracle(oracle, olb, collision, d, moving, objective):
    case = dataclasses.replace(porous_channel_case(nx=20, ny=10, nz=8, d=d, moving=moving), collision=collision,
                               magic=3.0 / 16.0)
    F = _field(case, 9)
    lat, f0 = _pair(oracle, case, F)
    steps, K = 17, 5
    if objective == "plane":
        obj = (0, case.shape[2] - 1, 0)
        kw = {"objective": obj}
    else:
        target = 0.01 * (I.uniform(33, (3,) + case.shape) - 0.5)
        region = (I.uniform(34, case.shape) < 0.6).astype(np.uint8)
        obj = oracle.Misfit(target, region)
        kw = {"u_target": target, "region": region}
    lo, go, to, Fo = lat.adjoint(f0, steps, obj, want_dforce=True)
    g = _gpu(case, F, "f64")
    r = g.adjoint_gradients(steps, K, **kw)
    g.close()
    dF = r["dforce"].cpu().numpy()
    assert abs(r["loss"] - lo) <= 1e-12 * abs(lo)
    assert np.max(np.abs(dF - Fo)) <= 1e-10 * np.max(np.abs(Fo))
    assert np.max(np.abs(r["dgamma"].cpu().numpy() - go)) <= 1e-10 * np.max(np.abs(go))
    assert abs(r["dtau"] - to) <= 1e-10 * abs(to)
    assert np.all(dF[:, case.material != I.FLUID] == 0)


def test_force_gradient_with_a_uniform_force(oracle, olb):
    """Without a field, dL/dF(x) is the gradient with respect to each cell's share of
    the uniform force: it equals the oracle's per-cell gradient, and its sum over the
    cells is the derivative with respect to the uniform force."""
    case = porous_channel_case(nx=18, ny=10, nz=8, moving=True)
    lat = case.oracle(oracle)
    f0 = case.oracle_state(lat)
    obj = (0, 17, 0)
    lo, go, to, Fo = lat.adjoint(f0, 15, obj, want_dforce=True)
    g = case.gpu("f64", "pull")
    r = g.adjoint_gradients(15, 4, objective=obj, want=("dforce",))
    g.close()
    dF = r["dforce"].cpu().numpy()
    assert np.max(np.abs(dF - Fo)) <= 1e-10 * np.max(np.abs(Fo))
    # d/deps L(F + eps e_x) by the oracle's tangent: sum of dL/dF_x over the cells
    e = np.zeros((3,) + case.shape)
    e[0] = 1.0
    _, dl = lat.tangent(f0, 15, obj, dforce=e)
    assert abs(dF[0].sum() - dl) <= 1e-10 * abs(dl)


def test_force_gradient_matches_gpu_central_differences(olb):
    import torch

    case = porous_channel_case(nx=22, ny=10, nz=8)
    F = _field(case, 11)
    steps = 25
    obj = (0, case.shape[2] - 1, 0)
    g = _gpu(case, F, "f64")
    f0 = g.get_populations().clone()
    dF = g.adjoint_gradients(steps, 6, objective=obj, want=("dforce",))["dforce"].cpu().numpy()
    plane = torch.from_numpy(case.material[:, :, -1] == I.FLUID).cuda()

    def run(Fv):
        g.set_force_field(torch.from_numpy(Fv.reshape(-1).copy()).cuda())
        g.set_populations(f0)
        g.step(steps)
        _, u = g.moments()
        return float(u[0, :, :, -1][plane].mean())

    h = 1e-6
    cells = I.random_fluid_cells(5, case.material, 6)
    for k, c in enumerate(cells):
        a = k % 3
        Fp = F.copy().reshape(3, -1)
        Fm = Fp.copy()
        Fp[a, c] += h
        Fm[a, c] -= h
        fd = (run(Fp) - run(Fm)) / (2 * h)
        assert abs(fd - dF.reshape(3, -1)[a, c]) <= 1e-5 * abs(fd) + 1e-13, (c, a, fd)
    g.close()


def test_force_misfit_autograd_function(olb):
    import torch

    case = porous_channel_case(nx=16, ny=8, nz=8)
    F = torch.from_numpy(_field(case, 13)).cuda()
    g = case.gpu("f64", "pull")
    f0 = g.get_populations().clone()
    target = torch.zeros((3,) + case.shape, dtype=torch.float64, device="cuda")
    Fv = F.clone().requires_grad_(True)
    J = olb.force_misfit_loss(g, Fv, f0, 12, 4, target)
    J.backward()
    g.set_force_field(F.contiguous())
    g.set_populations(f0)
    r = g.adjoint_gradients(12, 4, u_target=target, want=("dforce",))
    assert float(J.detach()) == r["loss"]
    assert torch.equal(Fv.grad, r["dforce"])
    g.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_identify_a_force_field_on_the_gpu(olb, dtype):
    """testFlowOpti3d with the adjoint LBM, in small: the reference flow u* comes
    from a spatially varying force field F*; the force field is identified from u*
    on every fluid cell, starting from zero, with three control components per cell,
    the GPU adjoint and torch's L-BFGS."""
    import torch

    from paper_2307_11752_gb300 import opti

    nx, ny, nz, steps, tau = 24, 12, 12, 150, 0.8
    m = I.channel(nx, ny, nz)
    lat = olb.Lattice(olb.D3Q19, (nx, ny, nz), dtype=dtype, scheme="pull")
    lat.set_material(torch.from_numpy(m.reshape(-1).copy()).cuda(), 1)
    lat.set_bgk(tau)
    lat.init_equilibrium()
    f0 = lat.get_populations().clone()
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    F0 = I.channel_force(ny, tau, 0.05)
    truth = np.zeros((3, nz, ny, nx))
    # divergence-free (F_x varies in z, F_y in x): a gradient part of a force is
    # balanced by pressure and moves no fluid, so only the solenoidal part is
    # identifiable from the flow
    truth[0] = F0 * (1.0 + 0.5 * np.sin(2 * np.pi * z / nz))
    truth[1] = 0.3 * F0 * np.cos(2 * np.pi * x / nx)
    truth = torch.from_numpy(truth).cuda()
    lat.set_force_field(truth.contiguous())
    lat.step(steps)
    _, u_ref = lat.moments()
    fl = torch.from_numpy(m == I.FLUID).cuda()

    def evaluate(F):
        return olb.force_misfit_loss(lat, F, f0, steps, 50, u_ref)

    zero = torch.zeros_like(truth)
    res = opti.identify_force(evaluate, zero, fl, 0.0, iterations=12)
    J = res.objective
    assert J[-1] <= 1e-4 * J[0], J
    # What the flow determines: the driving x component away from the no-slip walls
    # (next to them the flow barely responds to the force), and the field as a whole
    # up to the parts the pressure balances (F_y pushes towards the closed walls).
    dist = np.minimum.reduce([y - 1, ny - 2 - y, z - 1, nz - 2 - z])
    inner = torch.from_numpy((m == I.FLUID) & (dist >= 2)).cuda()
    err_x = float((res.gamma[0] - truth[0])[inner].norm() / truth[0][inner].norm())
    assert err_x <= 0.2, err_x
    g, t = res.gamma[:, fl], truth[:, fl]
    cos = float((g * t).sum() / (g.norm() * t.norm()))
    assert cos >= 0.95, cos
    lat.close()
