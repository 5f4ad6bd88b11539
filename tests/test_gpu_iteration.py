"""The Gamma - <n_HI> iteration (Sec. 4.1, Eq. 7-11) and the lambda - Gamma
iteration of the sub-grid law (Sec. 4.2) on the GPU against the oracle on
identical seeded inputs: every step's rays (ids and directions bit-exact),
segments, fields and budgets within the parity tolerances; without
recombinations the iterated step ionises as many atoms as it absorbs
photons (the exactness Sec. 4.1 states), to single-precision accuracy."""
import dataclasses as dc

import numpy as np
import pytest

import paper_2409_04521_gb300 as F
import workloads as W
from parity_util import run_pair

pytestmark = pytest.mark.gpu


def _no_recombination(iters, nsteps=6):
    p = W.stromgren(n=16, nsteps=nsteps)
    return dc.replace(p, options=dc.replace(p.options, alpha_B_const=0.0, gamma_iters=iters), dt=p.dt * 20)


def test_iterated_long_steps_match_oracle():
    run_pair(_no_recombination(6), check_every=1)


def test_iterated_subgrid_law_matches_oracle():
    p = W.cosmo20k(n=24, nsteps=6, nsrc=40)
    run_pair(dc.replace(p, options=dc.replace(p.options, gamma_iters=3)), check_every=2)


def test_iterated_temperature_run_matches_oracle():
    p = W.cosmo16(n=24, nsteps=6, nsrc=8)
    run_pair(dc.replace(p, options=dc.replace(p.options, gamma_iters=3)), check_every=3, T_rtol=2e-3)


def test_iteration_conserves_photons_without_recombinations():
    p = _no_recombination(16)
    g = F.Simulation(p, ray_capacity=1 << 20)
    V = p.dx_phys_cm ** 3
    for _ in range(p.nsteps):
        x0 = g.fields()["x_HII"].copy()
        a0 = g.budget()[1]
        g.step(p.dt)
        ion = ((g.fields()["x_HII"] - x0) * p.nH).sum() * V
        assert abs(ion / (g.budget()[1] - a0) - 1.0) < 1e-3
    g.close()
