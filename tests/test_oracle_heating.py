"""Pins of the oracle's Generalized-mode thermal model (Sec. 4.2, Eq. 12 and
Eq. 22; Sec. 5.2): newly ionised gas enters at T_reion, then the ionised
part heats by the power-law photo-heating of Eq. 22 -- each case-A
recombination balanced by one photo-ionisation that brings the spectrum's
mean excess energy -- against the Eq. 12 cooling terms with n_HI from the
photo-ionisation-equilibrium law.

The pins: the Eq. 22 bracket is the mean excess energy per ionisation,
checked by quadrature over 1-4 Ryd; the case-A coefficient against the
textbook table (Osterbrock & Ferland, Table 2.1); the integration against
energy conservation and against the equilibrium where heating equals
cooling; the whole run against the behaviour Sec. 5.2 reports for Test 2
(a sphere larger than the isothermal one, no pre-heating ahead of the
front)."""
import dataclasses as dc
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
import workloads as W

RYD_ERG = 13.6 * 1.602176634e-12
KB = 1.380649e-16


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 2.0, 3.0])
def test_eq22_bracket_is_the_mean_excess_energy(alpha):
    # photons per unit frequency ~ nu^-alpha / nu, absorbed in proportion to
    # sigma ~ nu^-2.75, each leaving h nu - 1 Ryd as heat
    w = lambda e: e ** (-alpha - 1.0) * e ** -2.75
    num = integrate.quad(lambda e: w(e) * (e - 1.0), 1.0, 4.0, epsabs=0, epsrel=1e-13)[0]
    den = integrate.quad(w, 1.0, 4.0, epsabs=0, epsrel=1e-13)[0]
    assert oracle.pl_heat_per_ion(alpha) == pytest.approx(RYD_ERG * num / den, rel=1e-12)


def test_case_a_recombination_coefficient():
    # Osterbrock & Ferland (2006) Table 2.1; the Hui & Gnedin fit lies within 3.5 %
    for T, aA, aB in ((5e3, 6.82e-13, 4.54e-13), (1e4, 4.18e-13, 2.59e-13), (2e4, 2.51e-13, 1.43e-13)):
        assert oracle.alpha_A(T) == pytest.approx(aA, rel=0.035)
        assert oracle.alpha_B(T) == pytest.approx(aB, rel=0.01)
        assert oracle.alpha_A(T) > oracle.alpha_B(T)        # case A adds captures to the ground state


def _rates(T, nH, yion, chi, alpha_pl, z):
    nHII, nHI = nH * (1 - yion), nH * yion
    ne = nHII + chi * nH
    heat = oracle.pl_heat_per_ion(alpha_pl) * oracle.alpha_A(T) * ne * nHII
    return heat, oracle.cooling(T, ne, nHI, nHII, z)


@pytest.mark.parametrize("chi", [0.0, 0.08])
def test_short_step_conserves_energy(chi):
    # 3/2 k_B n_tot dT = (H - Lambda) dt, n_tot counting H atoms and ions,
    # helium atoms and free electrons (one per HII, one per HeII)
    nH, yion, T0, z = 1e-3, 1e-3, 2e4, 6.0
    dt = 1e9                     # << cooling time: one sub-step, exact to first order
    T1 = oracle.gen_temperature(T0, 1.0, 1.0, yion, nH, chi, 2e4, 1.5, z, dt)
    heat, cool = _rates(T0, nH, yion, chi, 1.5, z)
    n_particles = nH + chi * nH + (nH * (1 - yion) + chi * nH)
    assert 1.5 * KB * n_particles * (T1 - T0) == pytest.approx((heat - cool) * dt, rel=1e-6)


@pytest.mark.parametrize("nH,yion", [(1e-3, 1e-4), (1e-1, 3e-3), (1.0, 1e-2)])
def test_long_step_settles_where_heating_equals_cooling(nH, yion):
    z = 0.0
    Teq = optimize.brentq(lambda T: (lambda h, c: h - c)(*_rates(T, nH, yion, 0.0, 1.5, z)), 3e3, 2e5, xtol=1e-6)
    assert 1e4 < Teq < 1e5
    for T0 in (5e3, 8e4):
        for dt in (3e17 / nH, 3e22 / nH):          # tens of cooling times, and far longer
            T = oracle.gen_temperature(T0, 1.0, 1.0, yion, nH, 0.0, 2e4, 1.5, z, dt)
            assert T == pytest.approx(Teq, rel=1e-3)


@pytest.mark.parametrize("nH,T0", [(1e-3, 2e4), (1e-1, 8e4), (1.0, 5e3)])
def test_relaxation_follows_the_energy_equation(nH, T0):
    # within about one cooling time the sub-stepped temperature follows the
    # solution of 3/2 k_B n_tot dT/dt = H - Lambda to first-order accuracy
    yion, z = 1e-3, 6.0
    ntot = 2 * nH - nH * yion
    rhs = lambda t, T: [(lambda h, c: (h - c) / (1.5 * KB * ntot))(*_rates(T[0], nH, yion, 0.0, 1.5, z))]
    tc = 1.5 * KB * ntot * T0 / abs(rhs(0, [T0])[0] * 1.5 * KB * ntot)
    for dt in (0.1 * tc, 0.5 * tc, 2 * tc):
        ref = integrate.solve_ivp(rhs, (0, dt), [T0], method="LSODA", rtol=1e-10, atol=1e-6).y[0, -1]
        got = oracle.gen_temperature(T0, 1.0, 1.0, yion, nH, 0.0, 2e4, 1.5, z, dt)
        assert got == pytest.approx(ref, rel=0.02)


def test_newly_ionised_gas_enters_at_t_reion():
    # mass-weighted mix of the gas already ionised and the newly ionised gas at T_reion
    dt = 1.0                     # heating and cooling negligible
    assert oracle.gen_temperature(100.0, 0.0, 0.3, 1e-3, 1e-3, 0.0, 2.5e4, 1.5, 0.0, dt) == pytest.approx(2.5e4, rel=1e-9)
    assert oracle.gen_temperature(1e4, 0.5, 1.0, 1e-3, 1e-3, 0.0, 2e4, 1.5, 0.0, dt) == pytest.approx(1.5e4, rel=1e-9)
    assert oracle.gen_temperature(3e4, 0.8, 0.6, 1e-3, 1e-3, 0.0, 2e4, 1.5, 0.0, dt) == pytest.approx(3e4, rel=1e-9)


def test_stromgren_with_temperature():
    # Sec. 5.2 (Test 2): T_init = 100 K; the ionised gas is hotter than
    # 10^4 K, recombines more slowly, and the sphere ends larger than the
    # isothermal analytic one; the gas ahead of the screen is not heated
    p = W.stromgren(n=32, nsteps=200)
    p = dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                   options=dc.replace(p.options, gen_mode=True, gamma_iters=4, isothermal=False, rates=1,
                                      T_init=100.0, t_reion=2e4))
    o = oracle.OracleSim(p)
    for _ in range(p.nsteps):
        o.step(p.dt)
        b = o.budget()
        assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-11 * b[0]
    x, _ = o.gen_state()
    T = o.fields()["T"]
    nH, ndot, t = p.nH[0], p.source_ndot.sum(), p.nsteps * p.dt
    a = 2.59e-13
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    R = (3 * x.sum() / (4 * math.pi)) ** (1 / 3)
    assert 1.0 < R / (rS * (1 - math.exp(-t * a * nH)) ** (1 / 3)) < 1.15
    ion = x > 0.99
    assert np.all((T[ion] > 8e3) & (T[ion] < 6e4)) and np.median(T[ion]) > 1e4
    assert np.all(T[x == 0] == 100.0)
