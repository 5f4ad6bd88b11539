"""Pins of the oracle's Generalized Opacity mode (Sec. 4.2, Eq. 14-22;
Sec. 5.1): a cell is a highly ionised fraction x_ion whose opacity comes
from a sub-grid law and a neutral rest behind an infinitely thin moving
screen; with the photo-ionisation-equilibrium law (Eq. 20-22) the ionised
volume of an isothermal Stromgren sphere follows the analytic I-front law
(Eq. 21) to better than 1 % after two recombination times, as Sec. 5.1
reports, and photons are conserved.

The screens' shares of the photons reaching them are iterated with lambda
and Gamma (Sec. 4.2: "until self-consistent"); at the fixed point every
photon a screen absorbs ionises an atom, so the photons absorbed beyond the
atoms left (lost) vanish as passes are added."""
import dataclasses as dc
import math

import numpy as np
import pytest

import oracle
import workloads as W


def _gen_stromgren(nsteps, iters=4, n=32):
    p = W.stromgren(n=n, nsteps=nsteps)
    return dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                      options=dc.replace(p.options, gen_mode=True, gamma_iters=iters))


def test_stromgren_law_after_two_recombination_times():
    p = _gen_stromgren(380)
    o = oracle.OracleSim(p)
    nH, a, ndot = p.nH[0], p.options.alpha_B_const, p.source_ndot.sum()
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    trec = 1 / (a * nH)
    for s in range(p.nsteps):
        o.step(p.dt)
        t = (s + 1) * p.dt
        if t >= 2 * trec and (s + 1) % 20 == 0:
            x, _ = o.gen_state()
            R = (3 * x.sum() / (4 * math.pi)) ** (1 / 3)
            err = R / (rS * (1 - math.exp(-t / trec)) ** (1 / 3)) - 1
            assert abs(err) < 0.01
        b = o.budget()
        assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-11 * b[0]
    assert abs(err) < 0.005          # settled: measured 0.28 % below


def _lost_photons(iters, nsteps=40):
    """Photons absorbed in the run that ionised nothing, over those emitted:
    absorbed - (atoms ionised + recombinations in the ionised parts)."""
    p = _gen_stromgren(nsteps, iters=iters)
    o = oracle.OracleSim(p)
    V = p.dx_phys_cm ** 3
    x0, a0, lost = np.zeros(p.ncell), 0.0, 0.0
    for _ in range(p.nsteps):
        o.step(p.dt)
        x, _ = o.gen_state()
        b = o.budget()
        used = ((x - x0) * p.nH * V).sum() + (p.options.alpha_B_const * p.nH ** 2 * x0 * V * p.dt).sum()
        lost += (b[1] - a0) - used
        x0, a0 = x, b[1]
    return lost / b[0]


def test_screen_iteration_converges_to_no_loss():
    # measured: 8.7e-2 (2 passes), 8.2e-3 (3), 2.3e-3 (4), 1.7e-6 (5), 3.7e-8 (6); how
    # fast a cascade of newly reached screens settles depends on the random
    # spheres, the fixed point loses nothing
    loss = [_lost_photons(k) for k in (2, 3, 4, 5, 6)]
    assert all(b < 0.5 * a for a, b in zip(loss, loss[1:])), loss
    assert loss[0] > 1e-2 and loss[3] < 1e-5 and loss[4] < 1e-6 and min(loss) > -1e-10
    assert loss[4] < 1e-5 * loss[0]


def test_screen_and_ionised_part():
    p = _gen_stromgren(40)
    o = oracle.OracleSim(p)
    for _ in range(p.nsteps):
        o.step(p.dt)
    x, y = o.gen_state()
    f = o.fields()
    assert np.all((x >= 0) & (x <= 1)) and np.all((y >= 0) & (y <= 1))
    # the ionised fraction reported is the ionised volume less its residual HI
    assert np.allclose(f["x_HII"], x * (1 - y), atol=1e-12)
    # the ionised part is in photo-ionisation equilibrium: y = alpha n_H / Gamma (Eq. 22)
    lit = (x > 0.5) & (f["gamma_HI"] > 0) & (y < 1)
    assert lit.sum() > 100
    assert np.allclose(y[lit], np.minimum(1.0, p.options.alpha_B_const * p.nH[lit] / f["gamma_HI"][lit]), rtol=1e-12)
    # the neutral rest is sharp: beyond the front cells nothing is ionised
    assert (x == 0).sum() > 0.5 * x.size and ((x > 0) & (x < 1)).sum() < (x >= 1).sum() + 2000


def test_helium_ratio_slows_the_screen():
    # Eq. 18: the screen ionises (1 + chi) n_H atoms per unit volume
    res = []
    for chi in (0.0, 0.08):
        p = _gen_stromgren(30)
        p = dc.replace(p, options=dc.replace(p.options, chi=chi))
        o = oracle.OracleSim(p)
        for _ in range(p.nsteps):
            o.step(p.dt)
        res.append(o.gen_state()[0].sum())
    assert res[1] < res[0] * 0.97


def test_merging_keeps_the_stromgren_law():
    # Sec. 3.3 in Generalized mode: merging all but the 0.05 N_RT brightest
    # rays keeps the sphere on the analytic law after two recombination times
    # (within 1 %; measured 0.52 %, as without merging, with a tenth of the
    # ray-cell segments), photons conserved
    p = _gen_stromgren(380)
    p = dc.replace(p, options=dc.replace(p.options, merge=True, n_ex=0.05, l_merge=0))
    o = oracle.OracleSim(p)
    nH, a, ndot = p.nH[0], p.options.alpha_B_const, p.source_ndot.sum()
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    trec = 1 / (a * nH)
    for s in range(p.nsteps):
        o.step(p.dt)
        t = (s + 1) * p.dt
        if t >= 2 * trec:
            R = (3 * o.gen_state()[0].sum() / (4 * math.pi)) ** (1 / 3)
            assert abs(R / (rS * (1 - math.exp(-t / trec)) ** (1 / 3)) - 1) < 0.01
    b = o.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-11 * b[0]
    assert o.rays()["merged"].sum() > 100
