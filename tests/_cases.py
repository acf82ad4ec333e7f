"""Shared set-up for the GPU parity tests: one lattice description, built both as
an oracle lattice and as a libolb lattice, fed the same seeded inputs."""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, Optional

import numpy as np

from paper_2307_11752_gb300 import inputs as I


@dataclass
class Case:
    d: int
    material: np.ndarray          # uint8 [nz, ny, nx]
    periodic: int
    tau: float
    force: tuple = (0.0, 0.0, 0.0)
    gamma: Optional[np.ndarray] = None
    walls: Dict[int, tuple] = field(default_factory=dict)
    rho: Optional[np.ndarray] = None
    u: Optional[np.ndarray] = None
    noise: Optional[np.ndarray] = None
    collision: str = "bgk"   # or "trt" with magic parameter `magic`
    magic: float = 0.25

    @property
    def shape(self):
        return self.material.shape

    @property
    def q(self):
        return 9 if self.d == 0 else 19

    def wall_table(self):
        wu = np.zeros((256, 3))
        for k, v in self.walls.items():
            wu[k] = v
        return wu

    def oracle(self, oracle):
        return oracle.Lattice(self.d, self.material, self.tau, periodic=self.periodic,
                              force=self.force, gamma=self.gamma, wall_u=self.wall_table(),
                              collision=oracle.TRT if self.collision == "trt" else oracle.BGK,
                              magic=self.magic)

    def oracle_state(self, lat):
        rho, u = (self.rho, self.u) if self.rho is not None else I.rest(self.shape)
        f = lat.init_equilibrium(rho, u)
        if self.noise is not None:
            f = f + np.where(self.material[None] == I.FLUID, self.noise, 0.0)
        return np.ascontiguousarray(f)

    def gpu(self, dtype="f64", scheme="pull"):
        from paper_2307_11752_gb300 import olb
        import torch

        nz, ny, nx = self.shape
        lat = olb.Lattice(self.d, (nx, ny, nz), dtype=dtype, scheme=scheme)
        lat.set_material(torch.from_numpy(self.material.reshape(-1).copy()).cuda(), self.periodic)
        for k, v in self.walls.items():
            lat.set_wall_velocity(k, v)
        if self.collision == "trt":
            lat.set_trt(self.tau, self.magic)
        else:
            lat.set_bgk(self.tau)
        lat.set_force(self.force)
        if self.gamma is not None:
            lat.set_porosity(torch.from_numpy(self.gamma.reshape(-1).copy()).cuda())
        rho, u = (self.rho, self.u) if self.rho is not None else I.rest(self.shape)
        lat.init_equilibrium(torch.from_numpy(np.ascontiguousarray(rho).reshape(-1)).cuda(),
                             torch.from_numpy(np.ascontiguousarray(u).reshape(-1)).cuda())
        if self.noise is not None:
            lat.perturb(torch.from_numpy(np.ascontiguousarray(self.noise).reshape(-1)).cuda())
        return lat


def rel_err(gpu, ref, mask=None) -> float:
    """max |gpu - ref| / max |ref| over (fluid) entries."""
    g = np.asarray(gpu)
    r = np.asarray(ref)
    if mask is not None:
        g = g[..., mask]
        r = r[..., mask]
    return float(np.max(np.abs(g - r)) / np.max(np.abs(r)))


def tgv2d_case(n=64, u0=0.01, tau=0.8):
    rho, u = I.tgv2d(n, u0)
    return Case(0, I.periodic_box(n, n, 1), 3, tau, rho=rho, u=u)


def tgv3d_case(n=32, u0=0.02, tau=0.6):
    rho, u = I.tgv3d(n, u0)
    return Case(1, I.periodic_box(n, n, n), 7, tau, rho=rho, u=u)


def cavity_case(nx=37, ny=29, nz=23, seed=1, lid=0.05, tau=None, d=1):
    m = I.cavity_box(nx, ny, nz if d == 1 else 1)
    q = 19 if d == 1 else 9
    if tau is None:
        tau = I.cavity_tau(min(nx, ny), 400.0, lid) if d == 1 else 0.6
        tau = max(tau, 0.52)
    return Case(d, m, 0, tau, walls={I.LID: (lid, 0.0, 0.0)},
                noise=I.population_noise(seed, q, m, 1e-6))


def porous_channel_case(nx=40, ny=14, nz=11, tau=0.8, seed=2, d=1, moving=False):
    m = I.channel(nx, ny, nz if d == 1 else 1)
    walls = {}
    if moving:
        m[:, -1, :] = I.LID
        walls[I.LID] = (0.02, 0.0, 0.01 if d == 1 else 0.0)
    q = 19 if d == 1 else 9
    F = (I.channel_force(ny, tau, 0.05), 0.0, 0.0)
    return Case(d, m, 1, tau, force=F, gamma=I.smoothed_porosity(seed, m), walls=walls,
                noise=I.population_noise(seed + 1, q, m, 1e-4))


def assert_cells_close(got, ref, rtol: float, floor: float):
    """Per-cell bound |got - ref| <= rtol |ref| + floor max|ref| at every cell (no
    norm over the field, so one badly wrong cell fails).  The floor only matters at
    cells whose own gradient is below floor/rtol of the largest one."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    bound = rtol * np.abs(ref) + floor * np.max(np.abs(ref))
    excess = np.abs(got - ref) - bound
    k = int(np.argmax(excess))
    assert excess.flat[k] <= 0, (f"cell {k}: got {got.flat[k]!r}, reference {ref.flat[k]!r}, "
                                 f"bound {bound.flat[k]:.3e}")
