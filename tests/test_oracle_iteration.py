"""Pins of the oracle's Gamma - <n_HI> iteration (Sec. 4.1, Eq. 7-11) and the
lambda - Gamma iteration of the sub-grid opacity (Sec. 4.2, Eq. 14-17).

Sec. 4.1 states the property that fixes the iteration: without
recombinations it gives the exact n_HI however long the step.  At the fixed
point each cell's ionisations during the step equal the photons it
absorbed (Gamma from the time-averaged n_HI makes the absorbed photons and
the ionisation update consistent); a single pass with the start-of-step
opacity does not.
"""
import dataclasses as dc

import numpy as np
import pytest

import oracle
import workloads as W


def _no_recombination(iters, nsteps=6, dt_factor=20.0):
    p = W.stromgren(n=16, nsteps=nsteps)
    return dc.replace(p, options=dc.replace(p.options, alpha_B_const=0.0, gamma_iters=iters), dt=p.dt * dt_factor)


def _ionisations_over_absorbed(prob):
    """Per step: atoms ionised in the box / photons absorbed in the box."""
    o = oracle.OracleSim(prob)
    V = prob.dx_phys_cm ** 3
    out = []
    for _ in range(prob.nsteps):
        x0 = o.fields()["x_HII"].copy()
        a0 = o.budget()[1]
        o.step(prob.dt)
        x1 = o.fields()["x_HII"]
        out.append(((x1 - x0) * prob.nH).sum() * V / (o.budget()[1] - a0))
    return np.array(out)


def test_iteration_is_exact_without_recombinations():
    r1 = _ionisations_over_absorbed(_no_recombination(1))
    r16 = _ionisations_over_absorbed(_no_recombination(16))
    assert np.abs(r1[0] - 1.0) > 0.5                   # one pass wastes most absorbed photons
    assert np.all(np.abs(r16 - 1.0) < 1e-4), r16 - 1.0


def test_iteration_converges():
    # the state after one long step approaches its fixed point as passes are added
    ref = oracle.OracleSim(_no_recombination(40, nsteps=2))
    for _ in range(2):
        ref.step(ref_dt := _no_recombination(40).dt)
    xref = ref.fields()["x_HII"]
    errs = []
    for k in (2, 4, 8, 16):
        p = _no_recombination(k, nsteps=2)
        o = oracle.OracleSim(p)
        for _ in range(2):
            o.step(p.dt)
        errs.append(np.abs(o.fields()["x_HII"] - xref).max())
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5 * max(1.0, errs[0])
    assert ref_dt > 0


def test_single_pass_is_the_plain_step():
    p = W.stromgren(n=16, nsteps=4)
    a = oracle.OracleSim(p)
    b = oracle.OracleSim(dc.replace(p, options=dc.replace(p.options, gamma_iters=1)))
    for _ in range(p.nsteps):
        a.step(p.dt)
        b.step(p.dt)
    for k, v in a.fields().items():
        assert np.array_equal(v, b.fields()[k])


@pytest.mark.parametrize("iters", [2, 4])
def test_lambda_gamma_iteration_keeps_the_budget_and_settles(iters):
    # sub-grid law (lambda depends on Gamma): every pass conserves photons,
    # and successive iteration counts approach one answer
    base = W.cosmo20k(n=24, nsteps=6, nsrc=40)
    res = {}
    for k in (iters, 2 * iters, 4 * iters):
        p = dc.replace(base, options=dc.replace(base.options, gamma_iters=k))
        o = oracle.OracleSim(p)
        for _ in range(p.nsteps):
            o.step(p.dt)
            b = o.budget()
            assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-10 * b[0]
        res[k] = o.fields()
    gmax = res[4 * iters]["gamma_HI"].max()
    d1 = np.abs(res[iters]["gamma_HI"] - res[4 * iters]["gamma_HI"]).max()
    d2 = np.abs(res[2 * iters]["gamma_HI"] - res[4 * iters]["gamma_HI"]).max()
    assert 1e-3 * gmax < d1 and d2 < d1
