"""Generalized Opacity mode (Sec. 4.2, Eq. 14-22) on the GPU against the
oracle on identical seeded inputs, and against the analytic I-front law of
an isothermal Stromgren sphere (Sec. 5.1: better than 1 % after two
recombination times).

Each screen's share of the photons reaching it comes from the previous pass
of the step's iteration.  A screen first reached in the last pass absorbs
all that reaches it, and what exceeds its atoms ionises nothing; that loss
depends on single-precision rounding in a way no tolerance bounds, so it
must be iterated away: with 5 passes it is 2e-6 of the photons emitted and
the two implementations agree cell by cell over whole runs (measured: x_ion
within 7e-5, ionised volume within 2e-6, budget terms within 5e-7 of
emitted, Gamma of cells more than half ionised within 1e-3, T within
1.5e-4)."""
import dataclasses as dc
import math

import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from parity_util import BUDGET_RTOL, compare_fields

pytestmark = pytest.mark.gpu


def _gen_stromgren(nsteps, iters=5, n=32, **kw):
    p = W.stromgren(n=n, nsteps=nsteps)
    return dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                      options=dc.replace(p.options, gen_mode=True, gamma_iters=iters, **kw))


def _gamma_rel(gf, of, x):
    """Largest relative Gamma difference on cells more than half ionised
    (Gamma of the ionised part divides by x_ion)."""
    g, o = gf["gamma_HI"], of["gamma_HI"]
    big = (x >= 0.5) & (o >= 1e-8 * max(o.max(), 1e-300))
    return float(np.max(np.abs(g - o)[big] / o[big])) if big.any() else 0.0


def _run_gen_pair(prob, x_atol, vol_rtol, bud_rtol, g_rtol, T_rtol=None):
    g = F.Simulation(prob, ray_capacity=1 << 21, keep_diagnostics=True)
    o = oracle.OracleSim(prob)
    worst = dict(x=0.0, vol=0.0, bud=0.0, gam=0.0, T=0.0)
    for s in range(prob.nsteps):
        g.step(prob.dt)
        o.step(prob.dt)
        gb, ob = g.budget(), o.budget()
        for b in (gb, ob):
            assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        xg, (xo, _) = g.ionized_volume(), o.gen_state()
        gf, of = g.fields(), o.fields()
        assert np.all((xg >= 0) & (xg <= 1))
        worst["x"] = max(worst["x"], float(np.max(np.abs(xg - xo))))
        worst["vol"] = max(worst["vol"], abs(xg.sum() - xo.sum()) / max(xo.sum(), 1e-300))
        worst["bud"] = max(worst["bud"], float(np.max(np.abs(gb - ob))) / ob[0])
        worst["gam"] = max(worst["gam"], _gamma_rel(gf, of, xo))
        if T_rtol is not None:
            worst["T"] = max(worst["T"], float(np.max(np.abs(gf["T"] - of["T"]) / of["T"])))
        assert np.max(np.abs(gf["x_HII"] - of["x_HII"])) <= x_atol
        if o.counts()["near_threshold"] == 0:
            assert g.counts()["rays"] == o.counts()["rays"]
        assert worst["x"] <= x_atol and worst["vol"] <= vol_rtol and worst["bud"] <= bud_rtol, (s, worst)
        assert worst["gam"] <= g_rtol and (T_rtol is None or worst["T"] <= T_rtol), (s, worst)
    g.close()
    o.close()
    return worst


def test_generalized_stromgren_matches_oracle():
    _run_gen_pair(_gen_stromgren(40), x_atol=5e-4, vol_rtol=2e-5, bud_rtol=2e-6, g_rtol=5e-3)


def test_generalized_subgrid_law_matches_oracle():
    p = W.cosmo20k(n=24, nsteps=8, nsrc=40)
    p = dc.replace(p, options=dc.replace(p.options, gen_mode=True, gamma_iters=4, chi=0.08))
    _run_gen_pair(p, x_atol=1e-5, vol_rtol=1e-6, bud_rtol=1e-6, g_rtol=1e-4)


def test_generalized_stromgren_law():
    p = _gen_stromgren(380, iters=4)
    g = F.Simulation(p, ray_capacity=1 << 21)
    nH, a, ndot = p.nH[0], p.options.alpha_B_const, p.source_ndot.sum()
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    trec = 1 / (a * nH)
    for s in range(p.nsteps):
        g.step(p.dt)
        t = (s + 1) * p.dt
        if t >= 2 * trec and (s + 1) % 20 == 0:
            R = (3 * g.ionized_volume().sum() / (4 * math.pi)) ** (1 / 3)
            err = R / (rS * (1 - math.exp(-t / trec)) ** (1 / 3)) - 1
            assert abs(err) < 0.01
    assert abs(err) < 0.005
    b = g.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-6 * b[0]
    g.close()


def test_generalized_batch_member_equals_alone():
    steps = 10
    probs = [_gen_stromgren(steps, n=16, iters=4),
             dc.replace(W.stromgren(n=16, nsteps=steps), options=dc.replace(W.stromgren().options, gamma_iters=4))]
    B = F.Batch(max_sims=2, max_grid=16, nbins=1, ray_capacity=1 << 20, emitter_capacity=16, gen_capable=True)
    slots = [B.add(p) for p in probs]
    for _ in range(steps):
        B.step()
    B.sync()
    for s, p in zip(slots, probs):
        a = F.Simulation(p, ray_capacity=1 << 20)
        for _ in range(steps):
            a.step(p.dt)
        if p.options.gen_mode:
            xa, xb = a.ionized_volume(), B.ionized_volume(s)
            assert np.max(np.abs(xa - xb)) <= 1e-4 and abs(xa.sum() - xb.sum()) <= 1e-5 * xa.sum()
        else:
            compare_fields(B.fields(s), a.fields(), x_atol=1e-5, g_rtol=1e-4)
        assert np.allclose(B.budget(s), a.budget(), rtol=1e-5)
        a.close()
    B.close()


def _gen_stromgren_T(nsteps, n=32, iters=5):
    # Sec. 5.2 (Test 2): the Stromgren setup with T_init = 100 K and evolving
    # temperature; newly ionised gas at T_reion, Eq. 22 photo-heating
    return _gen_stromgren(nsteps, n=n, iters=iters, isothermal=False, rates=1, T_init=100.0, t_reion=2e4,
                          alpha_pl=1.5)


def test_generalized_temperature_matches_oracle():
    # cell by cell over the whole run, T to single-precision integration;
    # never-reached cells keep T_init exactly
    p = _gen_stromgren_T(40)
    _run_gen_pair(p, x_atol=5e-4, vol_rtol=2e-5, bud_rtol=2e-6, g_rtol=5e-3, T_rtol=1e-3)


def test_generalized_temperature_stromgren():
    # the behaviour Sec. 5.2 reports: the ionised gas is hotter than 10^4 K,
    # the sphere ends larger than the isothermal analytic one (by about 4 %
    # there), and the gas the screen has not reached stays at T_init
    p = _gen_stromgren_T(200, iters=4)
    g = F.Simulation(p, ray_capacity=1 << 21)
    for _ in range(p.nsteps):
        g.step(p.dt)
    x, T = g.ionized_volume(), g.fields()["T"]
    nH, ndot, t, a = p.nH[0], p.source_ndot.sum(), p.nsteps * p.dt, 2.59e-13
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    R = (3 * x.sum() / (4 * math.pi)) ** (1 / 3)
    assert 1.0 < R / (rS * (1 - math.exp(-t * a * nH)) ** (1 / 3)) < 1.15
    ion = x > 0.99
    assert np.all((T[ion] > 8e3) & (T[ion] < 6e4)) and np.median(T[ion]) > 1e4
    assert np.all(T[x == 0] == np.float32(100.0))
    g.close()


def test_generalized_temperature_ragged_grid():
    # a 24 x 16 x 9 grid with the source near a corner: the screens, the
    # temperature and the escapes through three faces, cell by cell
    p = W.stromgren(n=32, nsteps=20)
    nx, ny, nz = 24, 16, 9
    p = dc.replace(p, grid=(nx, ny, nz), nH=np.full(nx * ny * nz, 1e-3), source_cells=np.array([[1, 14, 4]], np.int32),
                   mfp=dc.replace(p.mfp, mode=3),
                   options=dc.replace(p.options, gen_mode=True, gamma_iters=5, isothermal=False, rates=1,
                                      T_init=100.0, t_reion=2e4))
    _run_gen_pair(p, x_atol=5e-4, vol_rtol=2e-5, bud_rtol=2e-6, g_rtol=5e-3, T_rtol=1e-3)


def test_generalized_subgrid_law_with_temperature():
    # the sub-grid opacity law with helium and evolving temperature
    p = W.cosmo20k(n=24, nsteps=8, nsrc=40)
    p = dc.replace(p, options=dc.replace(p.options, gen_mode=True, gamma_iters=4, chi=0.08, isothermal=False,
                                         T_init=100.0, t_reion=2e4))
    _run_gen_pair(p, x_atol=1e-4, vol_rtol=1e-5, bud_rtol=1e-6, g_rtol=1e-3, T_rtol=1e-3)


def _oracle_lost(p):
    """The oracle's photons absorbed that ionised nothing, over those emitted:
    absorbed - (atoms ionised + recombinations in the ionised parts)."""
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
    o.close()
    return lost / b[0]


def test_screen_excess_is_zero_in_standard_mode():
    p = W.stromgren(n=16, nsteps=6)
    g = F.Simulation(p, ray_capacity=1 << 20)
    for _ in range(p.nsteps):
        g.step(p.dt)
    assert g.screen_excess() == 0.0
    g.close()


def test_screen_excess_against_oracle_loss():
    # photons the screens absorbed beyond their cells' neutral atoms, on the
    # first 40 steps of the 32^3 sphere: with 4 passes a measurable part of
    # the oracle's photons that ionised nothing (absorbed minus ionisations
    # and recombinations), with 6 passes iterated away on both sides
    p = _gen_stromgren(40, iters=4)
    g = F.Simulation(p, ray_capacity=1 << 22)
    for _ in range(p.nsteps):
        g.step(p.dt)
    lg = g.screen_excess() / g.budget()[0]
    g.close()
    lo = _oracle_lost(p)
    assert 1e-3 < lo < 1e-2
    assert 0.5 * lo <= lg <= 1.05 * lo
    p6 = _gen_stromgren(40, iters=6)
    g = F.Simulation(p6, ray_capacity=1 << 22)
    for _ in range(p6.nsteps):
        g.step(p6.dt)
    assert 0.0 <= g.screen_excess() / g.budget()[0] < 1e-6
    g.close()
