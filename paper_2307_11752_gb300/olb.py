"""ctypes binding of libolb.so (C ABI in include/olb.h).

Argument marshalling only: every step of the lattice Boltzmann update runs in
the CUDA kernels of libolb.so.  PyTorch supplies device memory (the library
allocates through torch's caching allocator) and the CUDA stream.  There is no
CPU fallback: if libolb.so is missing or no GPU is present, the calls raise.

The functions ``olb_*`` mirror the C names one to one.
  :class:`Lattice`               the fluid lattice (BGK or TRT collision, pull or AA)
  :func:`plane_velocity_loss`    ``olb_adjoint_run`` behind ``torch.autograd``
  :func:`velocity_misfit_loss`   ``olb_adjoint_run_misfit`` behind ``torch.autograd``
  :class:`AdeLattice`            the advection-diffusion lattice (D2Q5 / D3Q7)
The porosity identification driver built on these is ``paper_2307_11752_gb300.opti``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libolb.so")

D2Q9, D3Q19 = 0, 1
F64, F32, F16_SHIFTED, BF16_SHIFTED = 0, 1, 2, 3
PULL, AA = 0, 1
DTYPES = {"f64": F64, "f32": F32, "f16": F16_SHIFTED, "bf16": BF16_SHIFTED}
SCHEMES = {"pull": PULL, "aa": AA}
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_STATE",
          -5: "ERR_NONFINITE", -6: "ERR_TIMEOUT", -7: "ERR_UNSUPPORTED"}
Q = {D2Q9: 9, D3Q19: 19}
# bytes each population moves per cell update (read once + written once)
STATE_ELEM = {F64: 8, F32: 4, F16_SHIFTED: 2, BF16_SHIFTED: 2}

# Exported symbols and their argument types (the declarations of include/olb.h).
_P, _I, _I64, _D, _U = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_uint
SIGNATURES = {
    "olb_set_allocator": [_P, _P, _P],
    "olb_lattice_create": [_I, _I, _I, _I, _I, _P],
    "olb_lattice_destroy": [_P],
    "olb_set_stream": [_P, _P],
    "olb_set_scheme": [_P, _I],
    "olb_set_material": [_P, _P, _U],
    "olb_set_wall_velocity": [_P, _I, _P],
    "olb_set_bgk": [_P, _D],
    "olb_set_trt": [_P, _D, _D],
    "olb_set_force": [_P, _P],
    "olb_set_porosity": [_P, _P],
    "olb_init_equilibrium": [_P, _P, _P],
    "olb_perturb_populations": [_P, _P],
    "olb_set_populations": [_P, _P],
    "olb_get_populations": [_P, _P],
    "olb_step": [_P, _I64],
    "olb_step_stats": [_P, _I64, _P],
    "olb_moments": [_P, _P, _P],
    "olb_diagnostics": [_P, _P],
    "olb_adjoint_run": [_P, _I64, _I64, _P, _P, _P, _P],
    "olb_adjoint_run_misfit": [_P, _I64, _I64, _P, _P, _P, _P, _P],
    "olb_set_force_field": [_P, _P],
    "olb_inject_stalled_copy": [_P, _U, _I64],
    "olb_set_active_planes": [_P, _I, _I],
    "olb_halo_size": [_P, _P, _P],
    "olb_halo_pack": [_P, _I, _P],
    "olb_halo_unpack": [_P, _I, _P],
    "olb_adjoint_gradients": [_P, _I64, _I64, _P, _P, _P, _P],
    "olb_ade_create": [_I, _I, _I, _I, _I, _P],
    "olb_ade_destroy": [_P],
    "olb_ade_set_stream": [_P, _P],
    "olb_ade_set_tau": [_P, _D],
    "olb_ade_set_velocity": [_P, _P, _P],
    "olb_ade_init": [_P, _P],
    "olb_ade_set_material": [_P, _P, _U, _P],
    "olb_ade_set_velocity_from": [_P, _P],
    "olb_ade_step": [_P, _I64],
    "olb_ade_density": [_P, _P],
    "olb_synchronize": [_P],
    "olb_counters": [_P, _P, _P],
    "olb_statistics_noalloc": [_I, _I, _I, _I, _P, _P, _P, _P, _P],
    "olb_last_error": [],
    "olb_build_info": [],
}


class OlbError(RuntimeError):
    def __init__(self, status: int, func: str, message: str):
        super().__init__(f"{func}: {STATUS.get(status, status)}: {message}")
        self.status = status


class Objective(ctypes.Structure):
    _fields_ = [("plane_axis", ctypes.c_int32), ("plane_index", ctypes.c_int32),
                ("component", ctypes.c_int32)]


class Gradients(ctypes.Structure):
    """olb_gradients: output pointers of olb_adjoint_gradients (NULL = not computed)."""
    _fields_ = [("loss", ctypes.c_void_p), ("dL_dgamma", ctypes.c_void_p), ("dL_dtau", ctypes.c_void_p),
                ("dL_dF", ctypes.c_void_p)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libolb.so (built by ``paper_2307_11752_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2307_11752_gb300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name in ("olb_last_error", "olb_build_info") else ctypes.c_int
    _lib = lib
    return lib


def build_info() -> str:
    return load().olb_build_info().decode()


def _call(name: str, *args) -> int:
    rc = getattr(load(), name)(*args)
    if rc != 0:
        msg = load().olb_last_error().decode()
        raise OlbError(rc, name, msg)
    return rc


# --------------------------------------------------------------------------------------
# torch plumbing: allocator and stream
# --------------------------------------------------------------------------------------
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_callbacks = None


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _callbacks
    import torch

    if not enable:
        _call("olb_set_allocator", None, None, None)
        _callbacks = None
        return

    def _alloc(size, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(size))
        except Exception:  # out of memory -> NULL -> OLB_ERR_OOM
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _callbacks = (_ALLOC_T(_alloc), _FREE_T(_free))
    _call("olb_set_allocator", ctypes.cast(_callbacks[0], ctypes.c_void_p),
          ctypes.cast(_callbacks[1], ctypes.c_void_p), None)


def _ptr(a) -> Tuple[Optional[int], object]:
    """Address of a torch tensor (CUDA or CPU) or numpy array; keeps it alive."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, a
    import torch

    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), a
    raise TypeError(f"unsupported array type {type(a)}")


def _check_array(a, dtype_name: str, count: int, what: str):
    import torch

    if isinstance(a, np.ndarray):
        ok = a.dtype == np.dtype(dtype_name)
    elif isinstance(a, torch.Tensor):
        ok = a.dtype == getattr(torch, {"float64": "float64", "uint8": "uint8"}[dtype_name])
    else:
        raise TypeError(f"{what}: unsupported array type {type(a)}")
    if not ok:
        raise TypeError(f"{what} must be {dtype_name}")
    n = a.size if isinstance(a, np.ndarray) else a.numel()
    if n != count:
        raise ValueError(f"{what} has {n} elements, expected {count}")


# --------------------------------------------------------------------------------------
# Object wrapper
# --------------------------------------------------------------------------------------
class Lattice:
    """One lattice on the current CUDA device.  ``shape`` is (nx, ny, nz)."""

    def __init__(self, descriptor: int, shape: Sequence[int], dtype="f32", scheme="pull",
                 stream=None, torch_allocator: bool = True):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("libolb needs a CUDA GPU (no CPU fallback)")
        load()
        if torch_allocator and _callbacks is None:
            use_torch_allocator(True)
        self.descriptor = int(descriptor)
        nx, ny, nz = (list(shape) + [1, 1])[:3]
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.cells = self.nx * self.ny * self.nz
        self.q = Q[self.descriptor]
        self.dtype = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
        h = ctypes.c_void_p()
        _call("olb_lattice_create", self.descriptor, self.nx, self.ny, self.nz, self.dtype,
              ctypes.byref(h))
        self.handle = h
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _call("olb_set_stream", self.handle, ctypes.c_void_p(self.stream.cuda_stream))
        self.set_scheme(scheme)

    # -- lifetime --------------------------------------------------------------------
    def close(self):
        if getattr(self, "handle", None):
            load().olb_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration ---------------------------------------------------------------
    def set_scheme(self, scheme):
        _call("olb_set_scheme", self.handle, SCHEMES[scheme] if isinstance(scheme, str) else int(scheme))

    def set_material(self, material, periodic: int = 0):
        _check_array(material, "uint8", self.cells, "material")
        p, keep = _ptr(material)
        _call("olb_set_material", self.handle, p, int(periodic))

    def set_wall_velocity(self, material_id: int, u):
        uu = (ctypes.c_double * 3)(*[float(v) for v in (list(u) + [0, 0, 0])[:3]])
        _call("olb_set_wall_velocity", self.handle, int(material_id), uu)

    def set_bgk(self, tau: float):
        _call("olb_set_bgk", self.handle, float(tau))

    def set_trt(self, tau: float, magic: float = 0.25):
        """TRT collision: viscosity from tau, odd-part rate from the magic parameter."""
        _call("olb_set_trt", self.handle, float(tau), float(magic))

    def set_force(self, F):
        FF = (ctypes.c_double * 3)(*[float(v) for v in (list(F) + [0, 0, 0])[:3]])
        _call("olb_set_force", self.handle, FF)

    def set_force_field(self, F):
        """Per-cell force density float64 [3, nz, ny, nx] (CUDA tensor or host array),
        replacing the uniform force; None removes it."""
        if F is None:
            _call("olb_set_force_field", self.handle, None)
            return
        _check_array(F, "float64", 3 * self.cells, "F")
        p, keep = _ptr(F)
        _call("olb_set_force_field", self.handle, p)

    def set_porosity(self, gamma):
        if gamma is None:
            _call("olb_set_porosity", self.handle, None)
            return
        _check_array(gamma, "float64", self.cells, "gamma")
        p, keep = _ptr(gamma)
        _call("olb_set_porosity", self.handle, p)

    # -- state -----------------------------------------------------------------------
    def init_equilibrium(self, rho=None, u=None):
        if rho is not None:
            _check_array(rho, "float64", self.cells, "rho")
        if u is not None:
            _check_array(u, "float64", 3 * self.cells, "u")
        pr, kr = _ptr(rho)
        pu, ku = _ptr(u)
        _call("olb_init_equilibrium", self.handle, pr, pu)

    def perturb(self, df):
        _check_array(df, "float64", self.q * self.cells, "df")
        p, keep = _ptr(df)
        _call("olb_perturb_populations", self.handle, p)

    def set_populations(self, f):
        _check_array(f, "float64", self.q * self.cells, "f")
        p, keep = _ptr(f)
        _call("olb_set_populations", self.handle, p)

    def get_populations(self, out=None):
        import torch

        if out is None:
            out = torch.empty((self.q, self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        _check_array(out, "float64", self.q * self.cells, "out")
        p, keep = _ptr(out)
        _call("olb_get_populations", self.handle, p)
        return out

    def step(self, n: int = 1):
        _call("olb_step", self.handle, int(n))

    def step_stats(self, n: int) -> np.ndarray:
        out = np.zeros(7)
        _call("olb_step_stats", self.handle, int(n), out.ctypes.data)
        return out

    def moments(self, rho=None, u=None):
        import torch

        if rho is None:
            rho = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        if u is None:
            u = torch.empty((3, self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        _check_array(rho, "float64", self.cells, "rho")
        _check_array(u, "float64", 3 * self.cells, "u")
        pr, kr = _ptr(rho)
        pu, ku = _ptr(u)
        _call("olb_moments", self.handle, pr, pu)
        return rho, u

    def diagnostics(self, check: bool = True) -> np.ndarray:
        out = np.zeros(7)
        rc = load().olb_diagnostics(self.handle, out.ctypes.data)
        if rc != 0 and (check or rc != -5):
            raise OlbError(rc, "olb_diagnostics", load().olb_last_error().decode())
        return out

    def adjoint_run(self, n_steps: int, checkpoint_every: int, objective, dgamma=None):
        """(loss, dL/dgamma as a CUDA float64 tensor [nz, ny, nx], dL/dtau)."""
        import torch

        if dgamma is None:
            dgamma = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        _check_array(dgamma, "float64", self.cells, "dgamma")
        obj = Objective(*[int(v) for v in objective])
        loss, dtau = ctypes.c_double(), ctypes.c_double()
        p, keep = _ptr(dgamma)
        _call("olb_adjoint_run", self.handle, int(n_steps), int(checkpoint_every), ctypes.byref(obj),
              ctypes.byref(loss), p, ctypes.byref(dtau))
        return loss.value, dgamma, dtau.value

    def adjoint_run_misfit(self, n_steps: int, checkpoint_every: int, u_target, region=None, dgamma=None):
        """Velocity misfit J = 1/2 sum over the region's fluid cells of |u - u*|^2 after
        ``n_steps`` steps: (J, dJ/dgamma as a CUDA float64 tensor [nz, ny, nx], dJ/dtau).
        ``u_target``: float64 [3, nz, ny, nx] (CUDA tensor or host array); ``region``:
        uint8 [nz, ny, nx] or None (every fluid cell)."""
        import torch

        if dgamma is None:
            dgamma = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        _check_array(dgamma, "float64", self.cells, "dgamma")
        _check_array(u_target, "float64", 3 * self.cells, "u_target")
        if region is not None:
            _check_array(region, "uint8", self.cells, "region")
        loss, dtau = ctypes.c_double(), ctypes.c_double()
        pg, kg = _ptr(dgamma)
        pu, ku = _ptr(u_target)
        pr, kr = _ptr(region)
        _call("olb_adjoint_run_misfit", self.handle, int(n_steps), int(checkpoint_every), pu, pr,
              ctypes.byref(loss), pg, ctypes.byref(dtau))
        return loss.value, dgamma, dtau.value

    def adjoint_gradients(self, n_steps: int, checkpoint_every: int, objective=None, u_target=None, region=None,
                          want=("dgamma", "dtau", "dforce")):
        """Checkpointed adjoint of the plane objective (``objective`` = (axis, index,
        component)) or of the velocity misfit (``u_target``, ``region``) with the
        outputs named in ``want``: a dict with "loss" and any of "dgamma" (CUDA float64
        [nz, ny, nx]), "dtau" (float), "dforce" (CUDA float64 [3, nz, ny, nx])."""
        import torch

        if (objective is None) == (u_target is None):
            raise ValueError("give either objective or u_target")
        loss, dtau = ctypes.c_double(), ctypes.c_double()
        dg = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda") \
            if "dgamma" in want else None
        dF = torch.empty((3, self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda") \
            if "dforce" in want else None
        out = Gradients(ctypes.addressof(loss), None if dg is None else dg.data_ptr(),
                        ctypes.addressof(dtau) if "dtau" in want else None,
                        None if dF is None else dF.data_ptr())
        obj = None if objective is None else Objective(*[int(v) for v in objective])
        pu = pr = None
        keep = []
        if u_target is not None:
            _check_array(u_target, "float64", 3 * self.cells, "u_target")
            pu, k = _ptr(u_target)
            keep.append(k)
        if region is not None:
            _check_array(region, "uint8", self.cells, "region")
            pr, k = _ptr(region)
            keep.append(k)
        _call("olb_adjoint_gradients", self.handle, int(n_steps), int(checkpoint_every),
              None if obj is None else ctypes.byref(obj), pu, pr, ctypes.byref(out))
        res = {"loss": loss.value}
        if dg is not None:
            res["dgamma"] = dg
        if "dtau" in want:
            res["dtau"] = dtau.value
        if dF is not None:
            res["dforce"] = dF
        return res

    def set_active_planes(self, z_first: int, z_last: int):
        _call("olb_set_active_planes", self.handle, int(z_first), int(z_last))

    def halo_bytes(self) -> int:
        """Bytes of one face's halo values (olb_halo_size)."""
        n, e = ctypes.c_int64(), ctypes.c_int()
        _call("olb_halo_size", self.handle, ctypes.byref(n), ctypes.byref(e))
        return n.value * e.value

    def halo_buffer(self):
        """A device buffer (torch uint8 tensor) for one face's halo values."""
        import torch

        return torch.empty(self.halo_bytes(), dtype=torch.uint8, device="cuda")

    def _halo_ptr(self, buf) -> int:
        # the C call takes a bare pointer and cannot see the buffer's size
        need = self.halo_bytes()
        if not getattr(buf, "is_cuda", False) or not buf.is_contiguous():
            raise ValueError("the halo buffer must be a contiguous CUDA tensor")
        if buf.numel() * buf.element_size() < need:
            raise ValueError(f"the halo buffer holds {buf.numel() * buf.element_size()} bytes, {need} needed")
        return buf.data_ptr()

    def halo_pack(self, face: int, buf):
        _call("olb_halo_pack", self.handle, int(face), self._halo_ptr(buf))

    def halo_unpack(self, face: int, buf):
        _call("olb_halo_unpack", self.handle, int(face), self._halo_ptr(buf))

    def synchronize(self):
        _call("olb_synchronize", self.handle)

    def counters(self) -> Tuple[int, int]:
        t, k = ctypes.c_int64(), ctypes.c_int64()
        _call("olb_counters", self.handle, ctypes.byref(t), ctypes.byref(k))
        return t.value, k.value


# --------------------------------------------------------------------------------------
# Advection-diffusion lattice (D2Q5 / D3Q7)
# --------------------------------------------------------------------------------------
D2Q5, D3Q7 = 2, 3


class AdeLattice:
    """A passive scalar on a D2Q5 / D3Q7 lattice (``olb_ade_*``): BGK towards the
    first-order equilibrium, advected by a prescribed velocity or by a fluid
    lattice's (``set_velocity_from``), with periodic axes, no-flux walls and Dirichlet
    cells (``set_material``)."""

    def __init__(self, descriptor: int, shape, dtype: str = "f64", stream=None):
        import torch

        nx, ny, nz = shape
        h = ctypes.c_void_p()
        _call("olb_ade_create", int(descriptor), int(nx), int(ny), int(nz), DTYPES[dtype], ctypes.byref(h))
        self.handle = h
        self.nx, self.ny, self.nz = nx, ny, nz
        self.cells = nx * ny * nz
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        _call("olb_ade_set_stream", self.handle, ctypes.c_void_p(self.stream.cuda_stream))

    def close(self):
        if self.handle is not None:
            load().olb_ade_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def set_tau(self, tau: float):
        _call("olb_ade_set_tau", self.handle, float(tau))

    def set_velocity(self, v=None, field=None):
        vv = None if v is None else (ctypes.c_double * 3)(*[float(a) for a in (list(v) + [0, 0, 0])[:3]])
        if field is not None:
            _check_array(field, "float64", 3 * self.cells, "velocity field")
        pf, kf = _ptr(field)
        _call("olb_ade_set_velocity", self.handle, vv, pf)

    def set_material(self, material, periodic: int = 0, wall_C=None):
        """Boundaries: material uint8 [nz, ny, nx] (1 bulk, 0 no-flux wall, 2..255
        Dirichlet with value wall_C[m]), the periodic axes, wall_C 256 values or None."""
        _check_array(material, "uint8", self.cells, "material")
        pm, km = _ptr(material)
        wc = None
        if wall_C is not None:
            wc = np.zeros(256)
            src = np.asarray(wall_C, np.float64).reshape(-1)
            wc[:src.size] = src
        _call("olb_ade_set_material", self.handle, pm, int(periodic), None if wc is None else wc.ctypes.data)

    def set_velocity_from(self, fluid: "Lattice"):
        """v = the fluid lattice's current velocity (computed on the device)."""
        _call("olb_ade_set_velocity_from", self.handle, fluid.handle)

    def init(self, C):
        _check_array(C, "float64", self.cells, "C")
        p, k = _ptr(C)
        _call("olb_ade_init", self.handle, p)

    def step(self, n: int = 1):
        _call("olb_ade_step", self.handle, int(n))

    def density(self, out=None):
        import torch

        if out is None:
            out = torch.empty((self.nz, self.ny, self.nx), dtype=torch.float64, device="cuda")
        _check_array(out, "float64", self.cells, "C")
        p, k = _ptr(out)
        _call("olb_ade_density", self.handle, p)
        return out


# --------------------------------------------------------------------------------------
# autograd: loss of a run as a function of (gamma, tau)
# --------------------------------------------------------------------------------------
def plane_velocity_loss(lattice: Lattice, gamma, tau, f0, n_steps: int, checkpoint_every: int,
                        objective):
    """Mean velocity component over a plane after ``n_steps`` steps from ``f0``, as a
    differentiable function of the porosity field ``gamma`` (float64 CUDA tensor
    [nz, ny, nx]) and ``tau`` (0-d float64 tensor).  The backward pass returns the
    gradients that ``olb_adjoint_run`` computed with its discrete adjoint."""
    import torch

    class _PlaneVelocityLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g, t):
            lattice.set_bgk(float(t))
            lattice.set_porosity(g.detach().contiguous())
            lattice.set_populations(f0)
            loss, dg, dtau = lattice.adjoint_run(n_steps, checkpoint_every, objective)
            ctx.save_for_backward(dg)
            ctx.dtau = dtau
            ctx.tau_meta = (t.dtype, t.device)
            return torch.tensor(loss, dtype=torch.float64, device=g.device)

        @staticmethod
        def backward(ctx, grad):
            (dg,) = ctx.saved_tensors
            dtype, device = ctx.tau_meta
            grad_tau = torch.tensor(float(grad) * ctx.dtau, dtype=dtype, device=device)
            return grad * dg.view_as(gamma), grad_tau

    return _PlaneVelocityLoss.apply(gamma, tau)


def velocity_misfit_loss(lattice: Lattice, gamma, tau, f0, n_steps: int, checkpoint_every: int,
                         u_target, region=None):
    """J = 1/2 sum over the fluid cells of ``region`` of |u - u*|^2 after ``n_steps``
    steps from ``f0`` (the objective of the guide's domain identification), as a
    differentiable function of ``gamma`` (float64 CUDA tensor [nz, ny, nx]) and
    ``tau`` (0-d float64 tensor); backward returns the gradients of
    ``olb_adjoint_run_misfit``.  Compose it with a projection gamma = p(alpha) and any
    torch optimiser."""
    import torch

    class _VelocityMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g, t):
            lattice.set_bgk(float(t))
            lattice.set_porosity(g.detach().contiguous())
            lattice.set_populations(f0)
            loss, dg, dtau = lattice.adjoint_run_misfit(n_steps, checkpoint_every, u_target, region)
            ctx.save_for_backward(dg)
            ctx.dtau = dtau
            ctx.tau_meta = (t.dtype, t.device)
            return torch.tensor(loss, dtype=torch.float64, device=g.device)

        @staticmethod
        def backward(ctx, grad):
            (dg,) = ctx.saved_tensors
            dtype, device = ctx.tau_meta
            grad_tau = torch.tensor(float(grad) * ctx.dtau, dtype=dtype, device=device)
            return grad * dg.view_as(gamma), grad_tau

    return _VelocityMisfit.apply(gamma, tau)


def force_misfit_loss(lattice: Lattice, force, f0, n_steps: int, checkpoint_every: int, u_target,
                      region=None):
    """J = 1/2 sum over the fluid cells of ``region`` of |u - u*|^2 after ``n_steps``
    steps from ``f0`` as a differentiable function of the per-cell force density
    ``force`` (float64 CUDA tensor [3, nz, ny, nx]): the objective and the control of
    the guide's force-field identification (testFlowOpti3d, adjoint variant).  The
    lattice's collision, tau and porosity stay as set; backward returns dJ/dF of
    ``olb_adjoint_gradients``."""
    import torch

    class _ForceMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, F):
            lattice.set_force_field(F.detach().contiguous())
            lattice.set_populations(f0)
            r = lattice.adjoint_gradients(n_steps, checkpoint_every, u_target=u_target, region=region,
                                          want=("dforce",))
            ctx.save_for_backward(r["dforce"])
            return torch.tensor(r["loss"], dtype=torch.float64, device=F.device)

        @staticmethod
        def backward(ctx, grad):
            (dF,) = ctx.saved_tensors
            return grad * dF.view_as(force)

    return _ForceMisfit.apply(force)
