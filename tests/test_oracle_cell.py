"""Single-cell brute-force pins of the oracle's equilibrium and collision.

The moments of the second-order equilibrium, the conservation laws of a BGK
collision, the relaxation of a non-equilibrium perturbation by (1 - omega), and
the moments of Guo's forcing term (Guo, Zheng, Shi 2002, the scheme of Eq. dF)
are computed here by direct sums over the populations the oracle returns.
"""
import numpy as np
import pytest

from paper_2307_11752_gb300 import inputs as I


def _random_states(d, n, seed):
    dim = 2 if d == 0 else 3
    r = I.uniform(seed, (n, 4))
    for k in range(n):
        rho = 0.9 + 0.2 * r[k, 0]
        u = np.zeros(3)
        u[:dim] = 0.1 * (2 * r[k, 1:1 + dim] - 1) / np.sqrt(dim)
        yield rho, u


@pytest.mark.parametrize("d", [0, 1])
def test_equilibrium_moments(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    for rho, u in _random_states(d, 20, 11 + d):
        feq = oracle.equilibrium(d, rho, u)
        assert abs(feq.sum() - rho) < 1e-15
        assert np.allclose(c.T @ feq, rho * u, rtol=0, atol=1e-16)
        P = (c.T * feq) @ c
        expect = rho * (cs2 * np.diag([1.0] * dim + [0.0] * (3 - dim)) + np.outer(u, u))
        assert np.allclose(P, expect, rtol=0, atol=2e-16)


@pytest.mark.parametrize("d", [0, 1])
def test_collision_conserves_mass_and_momentum(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    noise = I.uniform(5 + d, (20, q))
    for k, (rho, u) in enumerate(_random_states(d, 20, 21 + d)):
        f = oracle.equilibrium(d, rho, u) + 1e-3 * (noise[k] - 0.5)
        for tau in (0.51, 0.8, 1.0, 1.7):
            fs = oracle.collide_cell(d, f, tau)
            assert abs(fs.sum() - f.sum()) < 2e-15
            assert np.allclose(c.T @ fs, c.T @ f, rtol=0, atol=2e-16)


@pytest.mark.parametrize("d", [0, 1])
def test_bgk_relaxes_non_equilibrium_by_one_minus_omega(oracle, d):
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    # A perturbation with zero mass and zero momentum leaves rho and u unchanged,
    # so one BGK step must scale it by (1 - omega) exactly.
    M = np.vstack([np.ones(q), c.T[:dim]])
    delta = I.uniform(7 + d, q) - 0.5
    delta -= M.T @ np.linalg.lstsq(M.T, delta, rcond=None)[0]
    for rho, u in _random_states(d, 5, 31 + d):
        feq = oracle.equilibrium(d, rho, u)
        for tau in (0.6, 1.0, 1.9):
            fs = oracle.collide_cell(d, feq + 1e-3 * delta, tau)
            assert np.allclose(fs - feq, (1 - 1 / tau) * 1e-3 * delta, rtol=0, atol=5e-16)
        # (tolerances here and below are a few ulps of O(1) populations; a dropped
        # or mis-scaled term is off by 1e-6 or more)
        # tau = 1 lands exactly on the equilibrium
        assert np.allclose(oracle.collide_cell(d, feq + 1e-3 * delta, 1.0), feq, rtol=0,
                           atol=5e-16)


@pytest.mark.parametrize("d", [0, 1])
def test_guo_source_moments(oracle, d):
    """Guo's term has moments 0, (1 - omega/2) F and (1 - omega/2)(u F + F u);
    with u = (j + F/2)/rho the post-collision momentum is exactly j + F."""
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    rF = I.uniform(41 + d, 3) - 0.5
    F = np.zeros(3)
    F[:dim] = 1e-4 * rF[:dim]
    for rho, u0 in _random_states(d, 10, 51 + d):
        feq0 = oracle.equilibrium(d, rho, u0)
        j = c.T @ feq0
        u = (j + F / 2) / rho
        for tau in (0.55, 0.8, 1.4):
            om = 1 / tau
            fs = oracle.collide_cell(d, feq0, tau, F=F)
            unforced = (1 - om) * feq0 + om * oracle.equilibrium(d, rho, u)
            S = fs - unforced
            assert abs(S.sum()) < 1e-15
            assert np.allclose(c.T @ S, (1 - om / 2) * F, rtol=0, atol=1e-15)
            second = (c.T * S) @ c
            assert np.allclose(second, (1 - om / 2) * (np.outer(u, F) + np.outer(F, u)),
                               rtol=0, atol=1e-15)
            assert abs(fs.sum() - rho) < 1e-15
            assert np.allclose(c.T @ fs, j + F, rtol=0, atol=1e-15)


@pytest.mark.parametrize("d", [0, 1])
def test_porosity_zero_relaxes_to_rest(oracle, d):
    """gamma = 0 (solid in the porous model) relaxes towards w rho, the rest state."""
    dim, q, c, opp, w, cs2 = oracle.descriptor(d)
    for rho, u in _random_states(d, 5, 61 + d):
        f = oracle.equilibrium(d, rho, u)
        for tau in (0.7, 1.0):
            fs = oracle.collide_cell(d, f, tau, gamma=0.0)
            assert np.allclose(fs, (1 - 1 / tau) * f + (1 / tau) * w * rho, rtol=0, atol=5e-16)
