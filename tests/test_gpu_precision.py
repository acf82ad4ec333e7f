"""Storage precision: FP32, FP16-shifted and BF16-shifted populations (FP32
arithmetic) against the FP64 oracle on the 3D Taylor-Green vortex.

The relative L2 velocity error ||u - u_oracle|| / ||u_oracle|| is reported for
every storage type.  Bars: FP32 within 1e-5 (populations, as elsewhere);
FP16-shifted within 1e-3 (the precision target of the 16-bit storage form);
BF16-shifted (8 significant bits) is only required to stay bounded.
"""
import numpy as np
import pytest

from _cases import rel_err, tgv3d_case

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


@pytest.fixture(scope="module")
def reference(oracle):
    """Oracle run of the 32^3 vortex (u0 0.02, tau 0.6) for 600 steps."""
    case = tgv3d_case(32, 0.02, 0.6)
    lat = case.oracle(oracle)
    f = case.oracle_state(lat)
    lat.step(f, 600)
    rho, u = lat.moments(f)
    return case, f, u


def _vel_err(u, uo):
    return float(np.linalg.norm(u - uo) / np.linalg.norm(uo))


@pytest.mark.parametrize("scheme", ["pull", "aa"])
def test_storage_precision_tgv3d(olb, reference, scheme, record_property):
    case, f_ref, u_ref = reference
    errs = {}
    for dtype in ("f32", "f16", "bf16"):
        g = case.gpu(dtype, scheme)
        g.step(600)
        f = g.get_populations().cpu().numpy()
        rho, u = g.moments()
        errs[dtype] = (_vel_err(u.cpu().numpy(), u_ref), rel_err(f, f_ref))
        g.close()
    for k, v in errs.items():
        record_property(f"{k}_velocity_rel_l2", v[0])
        record_property(f"{k}_population_rel_max", v[1])
    print("velocity / population errors vs FP64 oracle:", errs)
    assert errs["f32"][1] <= 1e-5
    assert errs["f32"][0] <= 1e-4
    assert errs["f16"][0] <= 1e-3
    assert errs["bf16"][0] <= 5e-2
    # 16-bit storage is coarser than FP32, and BF16 coarser than FP16
    assert errs["f32"][0] < errs["f16"][0] < errs["bf16"][0]
