"""Seeded synthetic workloads (geometry, initial fields, noise) for the BGK lattice.

This module holds no lattice Boltzmann arithmetic: it only builds the inputs that
both the GPU library and the CPU oracle receive -- material numbers, initial
density/velocity fields, perturbations and porosity fields -- as plain numpy
arrays in the canonical layout ``[..., nz, ny, nx]`` (x fastest).

Random numbers come from SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014; constants as in the
public reference implementation by S. Vigna), mapped to doubles in [0, 1) with
the top 53 bits.

Material numbers follow the guide's convention (section "Setting Material
Numbers"): 0 void, 1 fluid, 2 no-slip bounce-back wall; numbers >= 3 are used
here for moving walls whose velocity is set separately.
"""
from __future__ import annotations

import math

import numpy as np

FLUID, WALL, LID = 1, 2, 3
PERIODIC_X, PERIODIC_Y, PERIODIC_Z = 1, 2, 4

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream started at ``seed``."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, shape) -> np.ndarray:
    """U[0,1) doubles of the given shape from SplitMix64(seed)."""
    n = int(np.prod(shape))
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64).reshape(shape) * 2.0 ** -53


# --------------------------------------------------------------------------------------
# Geometries
# --------------------------------------------------------------------------------------
def periodic_box(nx: int, ny: int, nz: int = 1) -> np.ndarray:
    """All-fluid box (used with every axis periodic)."""
    return np.full((nz, ny, nx), FLUID, np.uint8)


def cavity(n: int, dim: int = 3) -> np.ndarray:
    """Lid-driven cubic (square) cavity of n cells per side: fluid inside, no-slip
    walls on the faces, the whole top plane y = n-1 (edges and corners included)
    is the moving lid (material 3)."""
    return cavity_box(n, n, n if dim == 3 else 1)


def cavity_box(nx: int, ny: int, nz: int) -> np.ndarray:
    """Box cavity of any size: fluid inside, no-slip walls on the faces, the whole
    top plane y = ny-1 is the moving lid (material 3).  nz == 1 gives the 2D cavity
    (walls on x and y only)."""
    m = np.full((nz, ny, nx), WALL, np.uint8)
    if nz > 1:
        m[1:-1, 1:-1, 1:-1] = FLUID
    else:
        m[:, 1:-1, 1:-1] = FLUID
    m[:, ny - 1, :] = LID
    return m


def channel(nx: int, ny: int, nz: int) -> np.ndarray:
    """Channel periodic in x with no-slip walls on the y and z boundary planes
    (for nz == 1 only the y planes are walls)."""
    m = np.full((nz, ny, nx), FLUID, np.uint8)
    m[:, 0, :] = WALL
    m[:, ny - 1, :] = WALL
    if nz > 1:
        m[0, :, :] = WALL
        m[nz - 1, :, :] = WALL
    return m


def plates(nx: int, ny: int, nz: int = 1, top: int = WALL) -> np.ndarray:
    """Flow between two plates y = 0 (wall) and y = ny-1 (``top`` material);
    periodic in x (and z)."""
    m = np.full((nz, ny, nx), FLUID, np.uint8)
    m[:, 0, :] = WALL
    m[:, ny - 1, :] = top
    return m


# --------------------------------------------------------------------------------------
# Initial fields
# --------------------------------------------------------------------------------------
def tgv2d(n: int, u0: float, nz: int = 1):
    """2D Taylor-Green vortex on an n x n periodic box (extruded along z when nz > 1),
    cell centres at integer coordinates, k = 2 pi / n:
    u = u0 sin kx cos ky, v = -u0 cos kx sin ky, p = -(u0^2/4)(cos 2kx + cos 2ky),
    rho = 1 + 3 p.  Returns (rho[nz,n,n], u[3,nz,n,n])."""
    k = 2.0 * math.pi / n
    x = np.arange(n, dtype=np.float64)
    X, Y = np.meshgrid(x, x, indexing="xy")  # X varies along the last axis
    ux = u0 * np.sin(k * X) * np.cos(k * Y)
    uy = -u0 * np.cos(k * X) * np.sin(k * Y)
    p = -(u0 * u0 / 4.0) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho = np.broadcast_to(1.0 + 3.0 * p, (nz, n, n)).copy()
    u = np.zeros((3, nz, n, n))
    u[0] = ux
    u[1] = uy
    return rho, u


def tgv2d_velocity(n: int, u0: float, nu: float, t: float, nz: int = 1) -> np.ndarray:
    """Exact Navier-Stokes solution of the 2D vortex at time t: the initial velocity
    times exp(-2 nu k^2 t)."""
    k = 2.0 * math.pi / n
    return tgv2d(n, u0, nz)[1] * math.exp(-2.0 * nu * k * k * t)


def tgv3d(n: int, u0: float, xp=np, **kw):
    """Classical 3D Taylor-Green vortex in a periodic n^3 box, k = 2 pi / n:
    u = u0 sin kx cos ky cos kz, v = -u0 cos kx sin ky cos kz, w = 0,
    p - p0 = (u0^2/16)(cos 2kx + cos 2ky)(cos 2kz + 2), rho = 1 + 3 (p - p0).
    ``xp`` is numpy (default) or torch (then ``kw`` may give ``device=``)."""
    k = 2.0 * math.pi / n
    x = xp.arange(n, dtype=xp.float64, **kw)
    Z, Y, X = xp.meshgrid(x, x, x, indexing="ij")
    ux = u0 * xp.sin(k * X) * xp.cos(k * Y) * xp.cos(k * Z)
    uy = -u0 * xp.cos(k * X) * xp.sin(k * Y) * xp.cos(k * Z)
    u = xp.stack([ux, uy, xp.zeros_like(ux)])
    p = (u0 * u0 / 16.0) * (xp.cos(2 * k * X) + xp.cos(2 * k * Y)) * (xp.cos(2 * k * Z) + 2.0)
    return 1.0 + 3.0 * p, u


def rest(shape):
    """rho = 1, u = 0 on every cell of ``shape`` = (nz, ny, nx)."""
    return np.ones(shape), np.zeros((3,) + tuple(shape))


def population_noise(seed: int, q: int, material: np.ndarray, amplitude: float = 1e-6):
    """amplitude * U(-1, 1) per population of every fluid cell, zero elsewhere;
    shape [q, nz, ny, nx]."""
    r = uniform(seed, (q,) + material.shape)
    return np.where(material[None] == FLUID, amplitude * (2.0 * r - 1.0), 0.0)


def smoothed_porosity(seed: int, material: np.ndarray, passes: int = 3) -> np.ndarray:
    """Seeded U(0,1) field smoothed by ``passes`` 3x3x3 box filters (periodic along
    x, edge-clamped along y and z), clamped to [0, 1]; non-fluid cells get 1."""
    g = uniform(seed, material.shape)
    nz = material.shape[0]
    for _ in range(passes):
        p = np.pad(g, ((1, 1), (1, 1), (0, 0)), mode="edge")
        p = np.concatenate([p[:, :, -1:], p, p[:, :, :1]], axis=2)
        acc = np.zeros_like(g)
        dzs = (-1, 0, 1) if nz > 1 else (0,)
        for dz in dzs:
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    acc += p[1 + dz:1 + dz + g.shape[0], 1 + dy:1 + dy + g.shape[1],
                             1 + dx:1 + dx + g.shape[2]]
        g = acc / (len(dzs) * 9)
    g = np.clip(g, 0.0, 1.0)
    return np.where(material == FLUID, g, 1.0)


def random_fluid_cells(seed: int, material: np.ndarray, count: int) -> np.ndarray:
    """``count`` distinct flat indices of fluid cells, drawn with SplitMix64."""
    fluid = np.flatnonzero(material.reshape(-1) == FLUID)
    keys = splitmix64(seed, fluid.size)
    return np.sort(fluid[np.argsort(keys, kind="stable")[:count]])


# --------------------------------------------------------------------------------------
# Parameters of the named workloads (lattice units)
# --------------------------------------------------------------------------------------
def viscosity(tau: float) -> float:
    """Lattice kinematic viscosity nu = (tau - 1/2) / 3."""
    return (tau - 0.5) / 3.0


def cavity_tau(n: int, reynolds: float = 400.0, lid_speed: float = 0.05) -> float:
    """tau giving Re = U L / nu with L = n - 2 fluid cells between the halfway walls."""
    nu = lid_speed * (n - 2) / reynolds
    return 3.0 * nu + 0.5


def channel_force(ny: int, tau: float, centre_speed: float = 0.05) -> float:
    """Body force F_x = 8 nu u_c / H^2, H = ny - 2 (the poiseuille2d recipe)."""
    h = ny - 2
    return 8.0 * viscosity(tau) * centre_speed / (h * h)
