"""The device-side timeout path of the TMA-fed step, made to run out on purpose.

The TMA-fed pull kernel waits on mbarriers for its own tile copies, each wait
bounded in time.  olb_inject_stalled_copy makes the next such step expect more
bytes than its copies deliver (a phase that nothing completes), with a 20 ms
limit: every block must give up, record the failure, let its copies land and
return, and the host must report OLB_ERR_TIMEOUT at the next synchronising call.
Afterwards the context must still be usable: the same handle reruns the workload
and matches the oracle.  No fault, trap or endless wait is involved."""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I

from _cases import cavity_case, rel_err

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


@pytest.mark.parametrize("dtype", ["f32", "f16"])
def test_stalled_tile_copy_reports_timeout_and_the_context_survives(oracle, olb, dtype):
    import time

    lib = olb.load()
    case = cavity_case(64, 21, 13)  # even nx: the pull steps after the first run the TMA-fed kernel
    g = case.gpu(dtype, "pull")
    g.step(2)
    assert lib.olb_synchronize(g.handle) == 0
    assert lib.olb_inject_stalled_copy(g.handle, 16, 20_000_000) == 0
    t = time.perf_counter()
    g.step(1)
    rc = lib.olb_synchronize(g.handle)
    took = time.perf_counter() - t
    assert rc == -6, (rc, lib.olb_last_error().decode())
    assert "waiting" in lib.olb_last_error().decode()
    assert took < 5.0  # each block gave up after its 20 ms limits
    assert lib.olb_synchronize(g.handle) == 0  # the error word was cleared
    # injection arguments are checked
    assert lib.olb_inject_stalled_copy(g.handle, 16, 10) == -1
    assert lib.olb_inject_stalled_copy(g.handle, 1 << 20, 20_000_000) == -1
    # the context and the handle still work: rerun from the initial state
    lat = case.oracle(oracle)
    f = case.oracle_state(lat)
    g.set_populations(f)
    g.step(30)
    lat.step(f, 30)
    tol = {"f32": 1e-5, "f16": 2e-3}[dtype]
    assert rel_err(g.get_populations().cpu().numpy(), f, case.material == I.FLUID) <= tol
    g.close()
