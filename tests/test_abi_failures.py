"""Failure injection on the host (no GPU needed): the device-memory provider
returns NULL, as an exhausted allocator would, and the library reports
OLB_ERR_OOM with a message instead of crashing; argument errors that are
detected before any CUDA call return OLB_ERR_ARG."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2307_11752_gb300 import build, olb
    build.build()
    return olb.load()


def test_allocator_failure_is_reported_as_oom(lib):
    from paper_2307_11752_gb300 import olb

    calls = []

    @olb._ALLOC_T
    def failing_alloc(size, ctx):
        calls.append(size)
        return None

    @olb._FREE_T
    def never_free(ptr, ctx):
        raise AssertionError("nothing was allocated")

    assert lib.olb_set_allocator(ctypes.cast(failing_alloc, ctypes.c_void_p),
                                 ctypes.cast(never_free, ctypes.c_void_p), None) == 0
    try:
        h = ctypes.c_void_p()
        rc = lib.olb_lattice_create(olb.D3Q19, 16, 16, 16, olb.F32, ctypes.byref(h))
        assert rc == -3
        assert h.value is None
        assert "allocator returned no memory" in lib.olb_last_error().decode()
        assert calls and calls[0] == 19 * (16 ** 3 + 256) * 4  # the first population buffer
    finally:
        assert lib.olb_set_allocator(None, None, None) == 0


def test_arguments_rejected_before_any_device_call(lib):
    from paper_2307_11752_gb300 import olb

    h = ctypes.c_void_p()
    assert lib.olb_lattice_create(olb.D2Q9, 8, 8, 2, olb.F32, ctypes.byref(h)) == -1
    assert "nz == 1" in lib.olb_last_error().decode()
    assert lib.olb_lattice_create(5, 8, 8, 1, olb.F32, ctypes.byref(h)) == -1
    assert lib.olb_lattice_create(olb.D3Q19, 0, 8, 8, olb.F32, ctypes.byref(h)) == -1
    assert lib.olb_lattice_create(olb.D3Q19, 8, 8, 8, 9, ctypes.byref(h)) == -1
    assert lib.olb_lattice_create(olb.D3Q19, 8, 8, 8, olb.F32, None) == -1
    assert lib.olb_set_bgk(None, 0.8) == -1
    assert lib.olb_step(None, 1) == -1
    assert lib.olb_lattice_destroy(None) == -1
    assert lib.olb_set_allocator(ctypes.c_void_p(1), None, None) == -1  # alloc without free


def test_new_entry_points_reject_bad_arguments_on_the_host(lib):
    """Argument errors of the TRT, misfit and advection-diffusion calls are reported
    before any device work."""
    from paper_2307_11752_gb300 import olb

    h = ctypes.c_void_p()
    assert lib.olb_set_trt(None, 0.8, 0.25) == -1
    assert lib.olb_adjoint_run_misfit(None, 5, 2, None, None, None, None, None) == -1
    assert lib.olb_ade_create(olb.D2Q9, 8, 8, 1, olb.F32, ctypes.byref(h)) == -1
    assert "D2Q5 or D3Q7" in lib.olb_last_error().decode()
    assert lib.olb_ade_create(olb.D2Q5, 8, 8, 2, olb.F32, ctypes.byref(h)) == -1
    assert lib.olb_ade_create(olb.D3Q7, 8, 8, 8, olb.F16_SHIFTED, ctypes.byref(h)) == -1
    assert lib.olb_ade_create(olb.D3Q7, 0, 8, 8, olb.F32, ctypes.byref(h)) == -1
    assert lib.olb_ade_create(olb.D3Q7, 8, 8, 8, olb.F32, None) == -1
    calls = {"olb_ade_destroy": (None,), "olb_ade_step": (None, 1), "olb_ade_set_tau": (None, 0.8),
             "olb_ade_init": (None, None), "olb_ade_density": (None, None)}
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == -1, name


def test_oversized_lattices_are_rejected_before_allocation(lib):
    """The largest lattices the 32-bit cell index supports: beyond them creation
    fails with OLB_ERR_ARG and allocates nothing (no GPU needed to see it)."""
    from paper_2307_11752_gb300 import olb

    h = ctypes.c_void_p()
    assert lib.olb_lattice_create(olb.D3Q19, 2048, 1024, 1024, olb.F32, ctypes.byref(h)) == -1
    assert "2^31" in lib.olb_last_error().decode()
    assert lib.olb_lattice_create(olb.D3Q19, 1, 1, 70000, olb.F32, ctypes.byref(h)) == -1
    assert "nz" in lib.olb_last_error().decode()
    assert lib.olb_ade_create(olb.D3Q7, 1024, 1024, 512, olb.F32, ctypes.byref(h)) == -1
    assert "too large" in lib.olb_last_error().decode()
    assert h.value is None


def test_every_handle_call_rejects_a_null_handle_on_the_host(lib):
    """Every entry point that takes a lattice or scalar-lattice handle refuses NULL with
    OLB_ERR_ARG and a message, before any device call (this runs without a GPU)."""
    u3 = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    i64 = ctypes.c_int64()
    i32 = ctypes.c_int()
    calls = {
        "olb_set_stream": (None, None), "olb_set_scheme": (None, 0),
        "olb_set_material": (None, None, 0), "olb_set_wall_velocity": (None, 3, u3),
        "olb_set_force": (None, u3), "olb_set_force_field": (None, None), "olb_set_porosity": (None, None),
        "olb_init_equilibrium": (None, None, None), "olb_perturb_populations": (None, None),
        "olb_set_populations": (None, None), "olb_get_populations": (None, None),
        "olb_step_stats": (None, 1, None), "olb_moments": (None, None, None), "olb_diagnostics": (None, None),
        "olb_adjoint_run": (None, 5, 2, None, None, None, None),
        "olb_adjoint_gradients": (None, 5, 2, None, None, None, None),
        "olb_synchronize": (None,), "olb_set_active_planes": (None, 1, 2),
        "olb_halo_size": (None, ctypes.byref(i64), ctypes.byref(i32)),
        "olb_halo_pack": (None, 0, None), "olb_halo_unpack": (None, 0, None),
        "olb_inject_stalled_copy": (None, 0, 0), "olb_counters": (None, ctypes.byref(i64), ctypes.byref(i64)),
        "olb_ade_set_stream": (None, None), "olb_ade_set_velocity": (None, u3, None),
        "olb_ade_set_material": (None, None, 0, None), "olb_ade_set_velocity_from": (None, None),
    }
    for name, args in calls.items():
        fn = getattr(lib, name)
        assert fn(*args) == -1, name
        assert lib.olb_last_error().decode(), name
