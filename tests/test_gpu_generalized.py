"""Generalized Opacity mode (Sec. 4.2, Eq. 14-22) on the GPU against the
oracle on identical seeded inputs, and against the analytic I-front law of
an isothermal Stromgren sphere (Sec. 5.1: better than 1 % after two
recombination times).

The moving-screen update is sensitive: the screen's share of arriving
photons is estimated from the previous pass, and a relative change of 1e-7
in the input (the gap between single and double precision) moves either
implementation's own per-cell ionised fractions by 1e-3 to 2e-2 and its
global sums by up to ~1e-4 within a few steps (measured: oracle against
oracle and GPU against GPU with the source rate changed by 1e-6).  So the
runs are compared element by element on the first steps, and after that on
the global quantities -- ionised volume, absorbed photons, mean Gamma, ray
count -- within a few times that sensitivity."""
import dataclasses as dc
import math

import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from parity_util import BUDGET_RTOL, compare_fields

pytestmark = pytest.mark.gpu


def _gen_stromgren(nsteps, iters=3, n=32, **kw):
    p = W.stromgren(n=n, nsteps=nsteps)
    return dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                      options=dc.replace(p.options, gen_mode=True, gamma_iters=iters, **kw))


def _run_gen_pair(prob, exact_steps):
    g = F.Simulation(prob, ray_capacity=1 << 21, keep_diagnostics=True)
    o = oracle.OracleSim(prob)
    for s in range(prob.nsteps):
        g.step(prob.dt)
        o.step(prob.dt)
        gb, ob = g.budget(), o.budget()
        for b in (gb, ob):
            assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        assert abs(gb[0] - ob[0]) <= 1e-6 * ob[0]
        xg, (xo, _) = g.ionized_volume(), o.gen_state()
        gf, of = g.fields(), o.fields()
        if s < exact_steps:
            compare_fields(gf, of, x_atol=1e-5)
            assert np.max(np.abs(xg - xo)) < 1e-5
            assert g.counts()["rays"] == o.counts()["rays"]
            assert np.array_equal(g.segment_counts(), o.segment_counts())
        else:
            assert np.all((xg >= 0) & (xg <= 1))
            assert abs(xg.sum() - xo.sum()) <= 1e-3 * xo.sum()
            assert np.all(np.abs(gb - ob) <= 5e-4 * ob[0])
            assert abs(g.counts()["rays"] - o.counts()["rays"]) <= 0.02 * o.counts()["rays"] + 16
            if of["gamma_HI"].mean() > 0:
                assert abs(gf["gamma_HI"].mean() - of["gamma_HI"].mean()) <= 2e-3 * of["gamma_HI"].mean()
    g.close()
    o.close()


def test_generalized_stromgren_matches_oracle():
    _run_gen_pair(_gen_stromgren(40), exact_steps=2)


def test_generalized_subgrid_law_matches_oracle():
    p = W.cosmo20k(n=24, nsteps=8, nsrc=40)
    p = dc.replace(p, options=dc.replace(p.options, gen_mode=True, gamma_iters=3, chi=0.08))
    _run_gen_pair(p, exact_steps=1)


def test_generalized_stromgren_law():
    p = _gen_stromgren(380)
    g = F.Simulation(p, ray_capacity=1 << 21)
    nH, a, ndot = p.nH[0], p.options.alpha_B_const, p.source_ndot.sum()
    rS = (3 * ndot / (4 * math.pi * a * nH * nH)) ** (1 / 3) / p.dx_phys_cm
    trec = 1 / (a * nH)
    for s in range(p.nsteps):
        g.step(p.dt)
        t = (s + 1) * p.dt
        if t >= 2 * trec and (s + 1) % 20 == 0:
            R = (3 * g.ionized_volume().sum() / (4 * math.pi)) ** (1 / 3)
            assert abs(R / (rS * (1 - math.exp(-t / trec)) ** (1 / 3)) - 1) < 0.01
    b = g.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-6 * b[0]
    g.close()


def test_generalized_batch_member_equals_alone():
    steps = 10
    probs = [_gen_stromgren(steps, n=16),
             dc.replace(W.stromgren(n=16, nsteps=steps), options=dc.replace(W.stromgren().options, gamma_iters=3))]
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
            assert abs(xa.sum() - xb.sum()) <= 1e-3 * xa.sum()
        else:
            compare_fields(B.fields(s), a.fields(), x_atol=1e-5, g_rtol=1e-4)
        assert np.allclose(B.budget(s), a.budget(), rtol=5e-4)
        a.close()
    B.close()
