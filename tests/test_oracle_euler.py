"""Pins of the oracle's Euler fluxes and Riemann solvers (readings c7/c8 of the
numerical flux (F.n)* in Eq. 1): consistency, antisymmetry, the Roe property,
and complex-step derivatives against finite differences."""
import numpy as np
import pytest

from oracle.euler import (lax_friedrichs, roe, roe_dissipation, normal_flux,
                          physical_flux, pressure, riemann)

G = 1.4


def random_states(rng, k):
    rho = rng.uniform(0.5, 2.0, k)
    u = rng.uniform(-0.6, 0.6, (3, k))
    p = rng.uniform(0.5, 3.0, k)
    E = p / (G - 1) + 0.5 * rho * (u ** 2).sum(0)
    return np.stack([rho, rho * u[0], rho * u[1], rho * u[2], E])


def random_normal(rng):
    n = rng.normal(size=3)
    return n / np.linalg.norm(n)


def test_physical_flux_closed_form():
    U = np.array([2.0, 2.0, 4.0, -2.0, 20.0])  # rho=2, u=(1,2,-1), E=20
    p = 0.4 * (20.0 - 0.5 * (4 + 16 + 4) / 2.0)
    assert abs(pressure(U, G) - p) < 1e-14
    F = physical_flux(U, G)
    assert np.allclose(F[0], [2.0, 2.0 + p, 4.0, -2.0, (20 + p) * 1.0])
    assert np.allclose(F[1], [4.0, 4.0, 8.0 + p, -4.0, (20 + p) * 2.0])
    assert np.allclose(F[2], [-2.0, -2.0, -4.0, 2.0 + p, -(20 + p)])


@pytest.mark.parametrize("kind", ["lf", "roe"])
def test_consistency(kind):
    rng = np.random.default_rng(0)
    U = random_states(rng, 50)
    n = random_normal(rng)
    assert np.abs(riemann(kind, U, U, n, G) - normal_flux(U, n, G)).max() < 1e-13


@pytest.mark.parametrize("kind", ["lf", "roe"])
def test_antisymmetry(kind):
    rng = np.random.default_rng(1)
    UL, UR = random_states(rng, 50), random_states(rng, 50)
    n = random_normal(rng)
    a = riemann(kind, UL, UR, n, G)
    b = riemann(kind, UR, UL, -n, G)
    assert np.abs(a + b).max() < 1e-12


def test_roe_property():
    """With |lambda| replaced by lambda the Roe dissipation is F(R).n - F(L).n."""
    rng = np.random.default_rng(2)
    UL, UR = random_states(rng, 50), random_states(rng, 50)
    n = random_normal(rng)
    d = roe_dissipation(UL, UR, n, G, absfun=lambda x: x)
    assert np.abs(d - (normal_flux(UR, n, G) - normal_flux(UL, n, G))).max() < 1e-12


def test_roe_upwind_supersonic():
    """For a supersonic state pair all |lambda| = lambda and Roe = F(UL).n."""
    rng = np.random.default_rng(3)
    UL = random_states(rng, 20)
    UR = UL * (1 + 0.01 * rng.uniform(-1, 1, UL.shape))
    n = np.array([1.0, 0.0, 0.0])
    for U in (UL, UR):
        U[1] = U[0] * 3.0          # u = 3 > c everywhere
        U[4] = 1.5 / (G - 1) + 0.5 * U[1] ** 2 / U[0]
    assert np.abs(roe(UL, UR, n, G) - normal_flux(UL, n, G)).max() < 1e-11


@pytest.mark.parametrize("kind", ["lf", "roe"])
def test_complex_step_matches_fd(kind):
    rng = np.random.default_rng(4)
    UL, UR = random_states(rng, 10), random_states(rng, 10)
    n = random_normal(rng)
    v = rng.normal(size=UL.shape)
    h = 1e-30
    cs = riemann(kind, UL + 1j * h * v, UR, n, G).imag / h
    e = 1e-6
    fd = (riemann(kind, UL + e * v, UR, n, G) - riemann(kind, UL - e * v, UR, n, G)) / (2 * e)
    assert np.abs(cs - fd).max() < 1e-6 * np.abs(cs).max()
