"""Pins of the oracle's ionisation update (Sec. 4.1, Eq. 6-10), rate fits
and temperature update (Sec. 4.1, Eq. 12) against closed forms, textbook
values and limits."""
import math

import numpy as np
import pytest

import oracle


def test_photoionisation_only_closed_form():
    # alpha = C = 0: dy/dt = -Gamma y  ->  y(t) = y0 exp(-Gamma t)
    for G, dt, y0 in [(1e-12, 3e13, 0.9988), (3e-14, 1e12, 0.5), (1e-9, 1e13, 1.0)]:
        y1, yb = oracle.chem_cell(1e-3, G, 0.0, 0.0, dt, 5, y0)
        assert y1 == pytest.approx(y0 * math.exp(-G * dt), rel=1e-12, abs=1e-300)
        # <y> = y0 (1 - e^{-G dt}) / (G dt)
        assert yb == pytest.approx(y0 * -math.expm1(-G * dt) / (G * dt), rel=1e-12)


def test_photoionisation_equilibrium():
    # dt -> infinity: Gamma y = alpha n_H (1-y)^2 (pure H, n_e = n_H x)
    nH, alpha = 1e-3, 2.59e-13
    for G in (1e-12, 1e-14, 1e-16):
        y1, _ = oracle.chem_cell(nH, G, alpha, 0.0, 1e30, 200, 0.5)
        a = alpha * nH
        # a y^2 - (2a + G) y + a = 0, root in (0,1)
        y = 2 * a / ((2 * a + G) + math.sqrt((2 * a + G) ** 2 - 4 * a * a))
        assert y1 == pytest.approx(y, rel=1e-9)


def test_pure_recombination_converges_to_exact():
    # Gamma = 0: dx/dt = -alpha n_H x^2  ->  1/x - 1/x0 = alpha n_H t
    nH, alpha, x0 = 1e-3, 2.59e-13, 0.9
    T = 1.0 / (alpha * nH)  # one recombination time
    nsteps = 4000
    dt = T / nsteps
    y = 1 - x0
    for _ in range(nsteps):
        y, _ = oracle.chem_cell(nH, 0.0, alpha, 0.0, dt, 5, y)
    x_exact = x0 / (1 + alpha * nH * T * x0)
    assert 1 - y == pytest.approx(x_exact, rel=2e-4)


def test_alpha_B_textbook_values():
    # case-B recombination coefficient (Osterbrock & Ferland, Table 2.1)
    for T, ref in [(5000.0, 4.54e-13), (1e4, 2.59e-13), (2e4, 1.43e-13)]:
        assert oracle.alpha_B(T) == pytest.approx(ref, rel=0.015)


def test_collisional_ionisation_vs_independent_fit():
    # Hui & Gnedin (1997) against Voronov (1997): two independent published fits
    for T in (1.5e4, 2e4, 5e4, 1e5, 3e5, 1e6):
        U = 13.6 / (8.617333262e-5 * T)
        vor = 2.91e-8 * U ** 0.39 * math.exp(-U) / (0.232 + U)
        assert oracle.coll_ion(T) == pytest.approx(vor, rel=0.2)
    assert oracle.coll_ion(100.0) == 0.0


def test_compton_cooling_sign():
    z = 9.0
    Tc = 2.7255 * (1 + z)
    assert oracle.cooling(Tc, 1e-4, 0.0, 0.0, z) == pytest.approx(0.0, abs=1e-45)
    assert oracle.cooling(2 * Tc, 1e-4, 0.0, 0.0, z) > 0
    assert oracle.cooling(0.5 * Tc, 1e-4, 0.0, 0.0, z) < 0


def test_temperature_particle_number_term():
    # no heating or cooling (no electrons, z = -1 removes Compton): only
    # T n_tot is conserved, T1 = T0 (1 + x0)/(1 + x1)
    T1 = oracle.temperature(100.0, 1e-4, 0.0, 0.5, 0.0, 0.0, -1.0, 1e12)
    assert T1 == pytest.approx(100.0 / 1.5, rel=1e-14)


def test_temperature_pure_heating_linear():
    # heating only (tiny density makes two-body cooling negligible):
    # T1 = T0 + 2/(3 k n_tot) H dt
    kB = 1.380649e-16
    nH, xb = 1e-12, 0.5
    H = 1e-36
    dt = 3e12
    T1 = oracle.temperature(1e4, nH, xb, xb, xb, H, -1.0, dt)
    dT = 2.0 / (3.0 * kB * nH * (1 + xb)) * H * dt
    assert T1 == pytest.approx(1e4 + dT, rel=1e-6)


def test_temperature_relaxes_to_heating_equilibrium():
    # constant heating against cooling: after many cooling times T sits where
    # H = Lambda(T)
    nH, xb, z = 1e-3, 0.999, 0.0
    T_eq = 2.0e4
    lam = oracle.cooling(T_eq, nH * xb, nH * (1 - xb), nH * xb, z)
    T = 1e4
    for _ in range(50):
        T = oracle.temperature(T, nH, xb, xb, xb, lam, z, 3e15)
    assert T == pytest.approx(T_eq, rel=1e-2)


@pytest.mark.parametrize("nH,xb,T0,heat_ratio", [(1e-1, 0.99, 8e4, 0.3), (1.0, 0.9, 5e3, 2.0), (1e-3, 0.999, 2e4, 0.5)])
def test_temperature_follows_the_energy_equation(nH, xb, T0, heat_ratio):
    # Eq. 12 at fixed ionisation: 3/2 k_B n_tot dT/dt = H - Lambda(T), n_tot =
    # n_H (1 + x) (atoms and ions plus one electron per ion); the explicit
    # sub-steps follow an accurate solution of it (scipy's LSODA) within
    # their first-order accuracy over up to two cooling times (measured at
    # most 2 %)
    integrate = pytest.importorskip("scipy.integrate")
    kB, z = 1.380649e-16, 6.0
    ne, nHII, nHI, ntot = nH * xb, nH * xb, nH * (1 - xb), nH * (1 + xb)
    heat = heat_ratio * oracle.cooling(T0, ne, nHI, nHII, z)
    rhs = lambda t, T: [2.0 / (3.0 * kB * ntot) * (heat - oracle.cooling(T[0], ne, nHI, nHII, z))]
    tc = T0 / abs(rhs(0.0, [T0])[0])
    for f in (0.1, 0.5, 2.0):
        ref = integrate.solve_ivp(rhs, (0.0, f * tc), [T0], method="LSODA", rtol=1e-10, atol=1e-8).y[0, -1]
        assert oracle.temperature(T0, nH, xb, xb, xb, heat, z, f * tc) == pytest.approx(ref, rel=0.03)
