"""GPU parity of the advection-diffusion lattice (olb_ade_*, D2Q5 / D3Q7 BGK with
the first-order equilibrium) against the oracle's: the scalar C within 1e-13
(FP64) and 1e-5 (FP32) relative after 60 steps, uniform and per-cell velocity,
sizes that are not multiples of the thread block; conservation; argument errors."""
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


def _velocity(desc, shape, field):
    nz, ny, nx = shape
    if not field:
        return np.array([0.05, -0.03, 0.02 if desc == 3 else 0.0])
    v = 0.1 * (I.uniform(21, (3, nz, ny, nx)) - 0.5)
    if desc == 2:
        v[2] = 0.0
    return np.ascontiguousarray(v)


@pytest.mark.parametrize("desc,dims", [(2, (37, 29, 1)), (3, (21, 17, 13))])
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 1e-5)])
@pytest.mark.parametrize("field", [False, True])
def test_ade_matches_oracle(oracle, olb, desc, dims, dtype, tol, field):
    import torch

    nx, ny, nz = dims
    shape = (nz, ny, nx)
    tau, steps = 0.74, 60
    C0 = np.ascontiguousarray(1.0 + 0.5 * I.uniform(22, shape))
    v = _velocity(desc, shape, field)
    lat_o = oracle.AdeLattice(0 if desc == 2 else 1, shape, tau, v)
    g = lat_o.init(C0)
    lat_o.step(g, steps)
    Co = lat_o.density(g)
    a = olb.AdeLattice(desc, dims, dtype)
    a.set_tau(tau)
    if field:
        a.set_velocity(field=torch.from_numpy(v).cuda())
    else:
        a.set_velocity(v)
    a.init(torch.from_numpy(C0).cuda())
    a.step(steps)
    Cg = a.density().cpu().numpy()
    a.close()
    assert np.max(np.abs(Cg - Co)) <= tol * np.max(np.abs(Co))


def test_ade_host_arrays_and_conservation(olb):
    dims = (16, 12, 10)
    shape = (10, 12, 16)
    a = olb.AdeLattice(3, dims, "f64")
    a.set_tau(0.9)
    a.set_velocity((0.04, 0.01, -0.02))
    C0 = np.ascontiguousarray(1.0 + I.uniform(23, shape))
    a.init(C0)
    a.step(101)
    out = np.zeros(shape)
    a.density(out)
    assert abs(out.sum() - C0.sum()) <= 1e-13 * C0.sum()
    a.close()


def test_ade_rejects_bad_arguments(olb):
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(0, (8, 8, 1))          # a fluid descriptor
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(2, (8, 8, 2))          # D2Q5 with nz > 1
    with pytest.raises(olb.OlbError):
        olb.AdeLattice(3, (8, 8, 8), "f16")   # 16-bit storage is not offered here
    a = olb.AdeLattice(3, (8, 8, 8))
    with pytest.raises(olb.OlbError):
        a.set_tau(0.5)
    with pytest.raises(olb.OlbError):
        a.set_velocity()
    a.close()
