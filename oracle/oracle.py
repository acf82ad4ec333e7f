"""Python binding of the FP64 CPU oracle (``olb_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The GPU library never
imports this module and this module never imports the GPU library.

Arrays follow the canonical layout of the method: populations ``f[q, nz, ny, nx]``
(x fastest), unshifted, float64; material ``uint8[nz, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "olb_oracle.cpp")
_LIB = os.path.join(_HERE, "libolb_oracle.so")

D2Q9, D3Q19 = 0, 1


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the oracle shared library next to its source (g++, FP contraction off)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    base = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(_LIB + ".tmp", _LIB)
            if verbose:
                print("built", _LIB, "openmp" if extra else "serial")
            return _LIB
    raise RuntimeError("oracle build failed:\n" + r.stderr)


class _Lattice(ctypes.Structure):
    _fields_ = [("descriptor", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("periodic", ctypes.c_uint32), ("collision", ctypes.c_int32),
                ("material", ctypes.c_void_p), ("wall_u", ctypes.c_void_p),
                ("tau", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("gamma", ctypes.c_void_p), ("magic", ctypes.c_double),
                ("force_field", ctypes.c_void_p)]


class _Objective(ctypes.Structure):
    _fields_ = [("plane_axis", ctypes.c_int32), ("plane_index", ctypes.c_int32),
                ("component", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("u_target", ctypes.c_void_p), ("region", ctypes.c_void_p)]


@dataclass
class Misfit:
    """Velocity-misfit objective J = 1/2 sum over the fluid cells of the region of
    |u - u*|^2 (the guide's optimisation examples).  u_target: [3, nz, ny, nx] (or
    [d, ...]); region: bool/uint8 [nz, ny, nx] or None (every fluid cell)."""
    u_target: np.ndarray
    region: Optional[np.ndarray] = None


def _objective(objective, shape):
    """ctypes objective and the arrays it points into (kept alive by the caller)."""
    if isinstance(objective, Misfit):
        n = int(np.prod(shape))
        ut = np.zeros((3, n))
        src = np.asarray(objective.u_target, np.float64).reshape(-1, n)
        ut[:src.shape[0]] = src
        reg = None if objective.region is None else np.ascontiguousarray(
            np.asarray(objective.region).reshape(n) != 0, np.uint8)
        obj = _Objective(0, 0, 0, 1, ut.ctypes.data, None if reg is None else reg.ctypes.data)
        return obj, (ut, reg)
    return _Objective(*objective), ()


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        P, I64, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        sig = {
            "olb_oracle_descriptor": [ctypes.c_int, P, P, P, P, P, P],
            "olb_oracle_equilibrium": [ctypes.c_int, D, P, P],
            "olb_oracle_collide_cell": [ctypes.c_int, P, D, D, P, P],
            "olb_oracle_collide_cell_trt": [ctypes.c_int, P, D, D, D, P, P],
            "olb_oracle_init_equilibrium": [P, P, P, P],
            "olb_oracle_collide": [P, P, P],
            "olb_oracle_stream": [P, P, P, P],
            "olb_oracle_step": [P, P, I64],
            "olb_oracle_moments": [P, P, P, P],
            "olb_oracle_diagnostics": [P, P, P],
            "olb_oracle_loss": [P, P, P, P],
            "olb_oracle_tangent": [P, P, I64, P, P, D, P, P, P],
            "olb_oracle_collide_tangent": [P, P, P, P, D, P, P],
            "olb_oracle_collide_adjoint": [P, P, P, P, P, P, P],
            "olb_oracle_stream_adjoint": [P, P, P, P],
            "olb_oracle_adjoint": [P, P, I64, P, P, P, P, P, P],
            "olb_oracle_ade_descriptor": [ctypes.c_int, P, P, P, P, P, P],
            "olb_oracle_ade_init": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P, P],
            "olb_oracle_ade_step": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, P, P, P, I64],
            "olb_oracle_ade_density": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P],
            "olb_oracle_ade_step_bc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint, P, P, D,
                                       P, P, P, I64],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (rc={rc})")


def descriptor(d: int):
    """(dim, q, c[q,3] int, opposite[q] int, w[q] float64, cs2) of a lattice."""
    c = np.zeros((19, 3), np.int32)
    opp = np.zeros(19, np.int32)
    w = np.zeros(19, np.float64)
    dim, q, cs2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().olb_oracle_descriptor(d, ctypes.byref(dim), ctypes.byref(q), _p(c), _p(opp),
                                       _p(w), ctypes.byref(cs2)), "descriptor")
    q = q.value
    return dim.value, q, c[:q].copy(), opp[:q].copy(), w[:q].copy(), cs2.value


def equilibrium(d: int, rho: float, u) -> np.ndarray:
    q = descriptor(d)[1]
    out = np.zeros(q)
    uu = np.zeros(3)
    uu[:len(u)] = u
    _check(lib().olb_oracle_equilibrium(d, float(rho), _p(uu), _p(out)), "equilibrium")
    return out


def collide_cell(d: int, f: np.ndarray, tau: float, gamma: float = 1.0, F=(0, 0, 0)) -> np.ndarray:
    f = np.ascontiguousarray(f, np.float64)
    FF = np.zeros(3)
    FF[:len(F)] = F
    out = np.zeros_like(f)
    _check(lib().olb_oracle_collide_cell(d, _p(f), float(gamma), float(tau), _p(FF), _p(out)),
           "collide_cell")
    return out


def collide_cell_trt(d: int, f: np.ndarray, tau: float, magic: float, gamma: float = 1.0,
                     F=(0, 0, 0)) -> np.ndarray:
    f = np.ascontiguousarray(f, np.float64)
    FF = np.zeros(3)
    FF[:len(F)] = F
    out = np.zeros_like(f)
    _check(lib().olb_oracle_collide_cell_trt(d, _p(f), float(gamma), float(tau), float(magic), _p(FF),
                                             _p(out)), "collide_cell_trt")
    return out


BGK, TRT = 0, 1


@dataclass
class Lattice:
    """A lattice description for the oracle.  ``material`` is uint8[nz, ny, nx];
    ``collision`` BGK or TRT (with ``magic`` = Lambda)."""
    descriptor: int
    material: np.ndarray
    tau: float
    periodic: int = 0
    force: tuple = (0.0, 0.0, 0.0)
    gamma: Optional[np.ndarray] = None
    wall_u: np.ndarray = field(default_factory=lambda: np.zeros((256, 3)))
    collision: int = BGK
    magic: float = 0.25
    force_field: Optional[np.ndarray] = None  # per-cell force density [3, nz, ny, nx]

    def __post_init__(self):
        self.material = np.ascontiguousarray(self.material, np.uint8)
        if self.material.ndim == 2:
            self.material = self.material[None]
        self.wall_u = np.ascontiguousarray(self.wall_u, np.float64).reshape(256, 3)
        if self.gamma is not None:
            self.gamma = np.ascontiguousarray(self.gamma, np.float64).reshape(self.material.shape)
        if self.force_field is not None:
            self.force_field = np.ascontiguousarray(self.force_field, np.float64).reshape((3,) + self.material.shape)
        self.q = descriptor(self.descriptor)[1]

    @property
    def shape(self):
        return self.material.shape  # (nz, ny, nx)

    @property
    def cells(self):
        return int(self.material.size)

    def _c(self) -> _Lattice:
        nz, ny, nx = self.material.shape
        F = (ctypes.c_double * 3)(*[float(v) for v in (list(self.force) + [0, 0, 0])[:3]])
        self._keep = _Lattice(self.descriptor, nx, ny, nz, self.periodic, int(self.collision),
                              self.material.ctypes.data, self.wall_u.ctypes.data,
                              float(self.tau), F, _p(self.gamma), float(self.magic), _p(self.force_field))
        return self._keep

    def _f(self, f: np.ndarray) -> np.ndarray:
        if f.dtype != np.float64 or not f.flags.c_contiguous or f.size != self.q * self.cells:
            raise ValueError("populations must be C-contiguous float64 [q, nz, ny, nx]")
        return f

    def zeros(self) -> np.ndarray:
        return np.zeros((self.q,) + self.shape)

    def init_equilibrium(self, rho: np.ndarray, u: np.ndarray) -> np.ndarray:
        rho = np.ascontiguousarray(rho, np.float64).reshape(self.shape)
        u = np.ascontiguousarray(u, np.float64).reshape((3,) + self.shape)
        f = self.zeros()
        _check(lib().olb_oracle_init_equilibrium(ctypes.byref(self._c()), _p(rho), _p(u), _p(f)),
               "init_equilibrium")
        return f

    def collide(self, f: np.ndarray) -> np.ndarray:
        out = np.empty_like(self._f(f))
        _check(lib().olb_oracle_collide(ctypes.byref(self._c()), _p(f), _p(out)), "collide")
        return out

    def stream(self, fs: np.ndarray, fpre: np.ndarray) -> np.ndarray:
        out = np.empty_like(self._f(fs))
        _check(lib().olb_oracle_stream(ctypes.byref(self._c()), _p(fs), _p(self._f(fpre)),
                                       _p(out)), "stream")
        return out

    def step(self, f: np.ndarray, n: int = 1) -> np.ndarray:
        """Advance ``f`` in place by ``n`` collide-and-stream steps; returns ``f``."""
        _check(lib().olb_oracle_step(ctypes.byref(self._c()), _p(self._f(f)), int(n)), "step")
        return f

    def moments(self, f: np.ndarray):
        rho = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        _check(lib().olb_oracle_moments(ctypes.byref(self._c()), _p(self._f(f)), _p(rho), _p(u)),
               "moments")
        return rho, u

    def diagnostics(self, f: np.ndarray) -> np.ndarray:
        out = np.zeros(7)
        _check(lib().olb_oracle_diagnostics(ctypes.byref(self._c()), _p(self._f(f)), _p(out)),
               "diagnostics")
        return out

    def loss(self, f: np.ndarray, objective) -> float:
        out = ctypes.c_double()
        obj, keep = _objective(objective, self.shape)
        _check(lib().olb_oracle_loss(ctypes.byref(self._c()), _p(self._f(f)), ctypes.byref(obj),
                                     ctypes.byref(out)), "loss")
        return out.value

    def tangent(self, f0: np.ndarray, n: int, objective, dgamma=None, dtau: float = 0.0, dforce=None):
        """(loss, directional derivative) along (dgamma per cell, dtau, dforce [3, nz, ny, nx])."""
        loss, dl = ctypes.c_double(), ctypes.c_double()
        obj, keep = _objective(objective, self.shape)
        dg = None if dgamma is None else np.ascontiguousarray(dgamma, np.float64)
        dF = None if dforce is None else np.ascontiguousarray(dforce, np.float64).reshape((3,) + self.shape)
        _check(lib().olb_oracle_tangent(ctypes.byref(self._c()), _p(self._f(f0)), int(n),
                                        ctypes.byref(obj), _p(dg), float(dtau),
                                        ctypes.byref(loss), ctypes.byref(dl), _p(dF)), "tangent")
        return loss.value, dl.value

    def collide_tangent(self, f, df, dgamma=None, dtau=0.0, dforce=None):
        out = np.zeros_like(self._f(f))
        dg = None if dgamma is None else np.ascontiguousarray(dgamma, np.float64)
        dF = None if dforce is None else np.ascontiguousarray(dforce, np.float64).reshape((3,) + self.shape)
        _check(lib().olb_oracle_collide_tangent(ctypes.byref(self._c()), _p(f),
                                                _p(self._f(np.ascontiguousarray(df))), _p(dg),
                                                float(dtau), _p(out), _p(dF)), "collide_tangent")
        return out

    def collide_adjoint(self, f, lams, want_dforce: bool = False):
        lam = np.zeros_like(self._f(f))
        dg = np.zeros(self.shape)
        dt = ctypes.c_double(0.0)
        dF = np.zeros((3,) + self.shape) if want_dforce else None
        _check(lib().olb_oracle_collide_adjoint(ctypes.byref(self._c()), _p(f),
                                                _p(self._f(np.ascontiguousarray(lams))), _p(lam),
                                                _p(dg), ctypes.byref(dt), _p(dF)), "collide_adjoint")
        if want_dforce:
            return lam, dg, dt.value, dF
        return lam, dg, dt.value

    def stream_adjoint(self, lam):
        lams = np.zeros_like(self._f(lam))
        direct = np.zeros(self.shape)
        _check(lib().olb_oracle_stream_adjoint(ctypes.byref(self._c()), _p(lam), _p(lams),
                                               _p(direct)), "stream_adjoint")
        return lams, direct

    def adjoint(self, f0: np.ndarray, n: int, objective, want_lambda0: bool = False,
                want_dforce: bool = False):
        """(loss, dL/dgamma [nz,ny,nx], dL/dtau[, dL/df0][, dL/dF [3,nz,ny,nx]]) of the
        objective after n steps; dL/dF is the gradient with respect to the force density
        of every cell."""
        loss, dtau = ctypes.c_double(), ctypes.c_double()
        dg = np.zeros(self.shape)
        lam0 = self.zeros() if want_lambda0 else None
        dF = np.zeros((3,) + self.shape) if want_dforce else None
        obj, keep = _objective(objective, self.shape)
        _check(lib().olb_oracle_adjoint(ctypes.byref(self._c()), _p(self._f(f0)), int(n),
                                        ctypes.byref(obj), ctypes.byref(loss), _p(dg),
                                        ctypes.byref(dtau), _p(lam0), _p(dF)), "adjoint")
        out = (loss.value, dg, dtau.value)
        if want_lambda0:
            out = out + (lam0,)
        if want_dforce:
            out = out + (dF,)
        return out


# ------------------------------------------------------------------------------------
# Advection-diffusion (D2Q5 = 0, D3Q7 = 1), fully periodic
# ------------------------------------------------------------------------------------
def ade_descriptor(d: int):
    """(dim, q, c[q,3], opposite[q], w[q], cs2) of D2Q5 (d = 0) or D3Q7 (d = 1)."""
    c = np.zeros((7, 3), np.int32)
    opp = np.zeros(7, np.int32)
    w = np.zeros(7, np.float64)
    dim, q, cs2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().olb_oracle_ade_descriptor(d, ctypes.byref(dim), ctypes.byref(q), _p(c), _p(opp), _p(w),
                                           ctypes.byref(cs2)), "ade_descriptor")
    q = q.value
    return dim.value, q, c[:q].copy(), opp[:q].copy(), w[:q].copy(), cs2.value


@dataclass
class AdeLattice:
    """Passive scalar on a periodic D2Q5 / D3Q7 lattice of shape (nz, ny, nx), BGK with
    relaxation time ``tau`` towards the first-order equilibrium, advected by ``v``
    (a uniform 3-vector or a [3, nz, ny, nx] field)."""
    descriptor: int
    shape: tuple
    tau: float
    v: object = (0.0, 0.0, 0.0)
    # boundaries (None: every cell bulk, every axis periodic): material uint8 [nz, ny, nx]
    # with 1 bulk, 0 no-flux wall, 2..255 Dirichlet cell of value wall_C[m]
    material: Optional[np.ndarray] = None
    wall_C: Optional[np.ndarray] = None
    periodic: int = 7

    def __post_init__(self):
        self.q = ade_descriptor(self.descriptor)[1]
        if self.material is not None:
            self.material = np.ascontiguousarray(self.material, np.uint8).reshape(tuple(self.shape))
        if self.wall_C is not None:
            wc = np.zeros(256)
            src = np.asarray(self.wall_C, np.float64).reshape(-1)
            wc[:src.size] = src
            self.wall_C = wc
        v = np.asarray(self.v, np.float64)
        if v.size == 3:
            self._vu, self._vf = np.ascontiguousarray(v.reshape(3)), None
        else:
            self._vu, self._vf = None, np.ascontiguousarray(v.reshape(3, -1))

    def _dims(self):
        nz, ny, nx = self.shape
        return nx, ny, nz

    def init(self, C: np.ndarray) -> np.ndarray:
        C = np.ascontiguousarray(C, np.float64).reshape(-1)
        g = np.zeros((self.q,) + tuple(self.shape))
        _check(lib().olb_oracle_ade_init(self.descriptor, *self._dims(), _p(C), _p(self._vf), _p(self._vu),
                                         _p(g)), "ade_init")
        return g

    def step(self, g: np.ndarray, n: int = 1) -> np.ndarray:
        if g.dtype != np.float64 or not g.flags.c_contiguous:
            raise ValueError("g must be C-contiguous float64 [q, nz, ny, nx]")
        if self.material is None and self.periodic == 7:
            _check(lib().olb_oracle_ade_step(self.descriptor, *self._dims(), float(self.tau), _p(self._vf),
                                             _p(self._vu), _p(g), int(n)), "ade_step")
        else:
            _check(lib().olb_oracle_ade_step_bc(self.descriptor, *self._dims(), int(self.periodic),
                                                _p(self.material), _p(self.wall_C), float(self.tau),
                                                _p(self._vf), _p(self._vu), _p(g), int(n)), "ade_step_bc")
        return g

    def density(self, g: np.ndarray) -> np.ndarray:
        C = np.zeros(tuple(self.shape))
        _check(lib().olb_oracle_ade_density(self.descriptor, *self._dims(), _p(np.ascontiguousarray(g)), _p(C)),
               "ade_density")
        return C


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv, verbose=True)
