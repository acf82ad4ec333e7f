"""The porosity identification driver (paper_2307_11752_gb300/opti.py) on the CPU,
with the FP64 oracle's adjoint as the objective and gradient: the guide's
domainIdentification3d set-up in small, on D2Q9.  A block of low porosity in a
forced periodic channel is recovered from the velocity field it produces."""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

torch = pytest.importorskip("torch")


def _channel(oracle, nx=24, ny=12, tau=0.8):
    m = I.channel(nx, ny, 1)
    F = (I.channel_force(ny, tau, 0.05), 0.0, 0.0)
    lat = oracle.Lattice(0, m, tau, periodic=1, force=F, gamma=np.ones(m.shape))
    f0 = lat.init_equilibrium(*I.rest(m.shape))
    return lat, f0


def _oracle_misfit(lat, f0, n, obj):
    class Misfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g):
            lat.gamma = g.detach().numpy().copy()
            loss, dg, _ = lat.adjoint(f0, n, obj)
            ctx.save_for_backward(torch.from_numpy(dg))
            return torch.tensor(loss, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad):
            (dg,) = ctx.saved_tensors
            return grad * dg

    return Misfit.apply


@pytest.mark.parametrize("projection", ["sigmoid", "rectifier"])
def test_identify_a_porous_block_from_its_flow(oracle, projection):
    from paper_2307_11752_gb300 import opti

    lat, f0 = _channel(oracle)
    n = 150
    shape = lat.shape
    truth = np.ones(shape)
    truth[0, 4:8, 10:14] = 0.05  # the obstacle
    lat.gamma = truth
    f = f0.copy()
    lat.step(f, n)
    _, u_ref = lat.moments(f)
    fl = lat.material == I.FLUID
    design = np.zeros(shape, bool)
    design[0, 2:10, 7:17] = True
    design &= fl
    obj = oracle.Misfit(u_ref, fl & ~design)  # only the flow around the design domain is observed
    evaluate = _oracle_misfit(lat, f0, n, obj)
    res = opti.identify_porosity(evaluate, torch.ones(shape, dtype=torch.float64), torch.from_numpy(design),
                                 0.7, projection=projection, iterations=25)
    J = res.objective
    assert len(J) >= 2 and all(np.isfinite(J))
    assert J[-1] <= 1e-3 * J[0], J
    g = res.gamma.numpy()
    inside = truth < 0.5
    assert g[inside].mean() < 0.5 < g[design & ~inside].mean()
    assert np.all(g[~design] == 1.0)
    assert res.evaluations >= len(J)


def test_projection_round_trip_and_bad_arguments():
    from paper_2307_11752_gb300 import opti

    g = torch.tensor([0.01, 0.3, 0.5, 0.99], dtype=torch.float64)
    for name in opti.PROJECTIONS:
        assert torch.allclose(opti.project(opti.unproject(g, name), name), g, rtol=1e-12, atol=0)
    with pytest.raises(ValueError):
        opti.project(g, "baron")
    with pytest.raises(ValueError):
        opti.identify_porosity(lambda x: x.sum(), torch.ones(2, 2), torch.zeros(2, 2, dtype=torch.bool), 0.5)
