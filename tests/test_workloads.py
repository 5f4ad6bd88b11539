"""Checks of the seeded input generators (not the method): density-field
statistics and spectrum tables against independent quadrature."""
import numpy as np
import pytest
from scipy import integrate

import workloads as W


def test_lognormal_field_statistics():
    d = W.lognormal_delta(48, 1.0, seed=3)
    assert d.shape == (48 ** 3,)
    assert np.all(d > 0)
    g = np.log(d)
    assert g.std() == pytest.approx(1.0, rel=1e-12)
    assert g.mean() == pytest.approx(-0.5, abs=1e-12)
    # seeded: identical on a second call, different for another seed
    assert np.array_equal(d, W.lognormal_delta(48, 1.0, seed=3))
    assert not np.array_equal(d, W.lognormal_delta(48, 1.0, seed=4))


def test_blackbody_bins_against_quad():
    edges = 13.6 * 2.0 ** (np.arange(5) / 2.0)
    sp = W.blackbody_bins(1e5, edges)
    kT = 8.617333262e-5 * 1e5
    n = lambda E: E * E / np.expm1(E / kT)
    tot = integrate.quad(n, edges[0], edges[-1], epsabs=0, epsrel=1e-12)[0]
    assert sp.frac.sum() == pytest.approx(1.0, abs=1e-15)
    for b in range(4):
        lo, hi = edges[b], edges[b + 1]
        nb = integrate.quad(n, lo, hi, epsrel=1e-12)[0]
        sb = integrate.quad(lambda E: W.sigma_HI(E) * n(E), lo, hi, epsrel=1e-12)[0] / nb
        assert sp.frac[b] == pytest.approx(nb / tot, rel=1e-9)
        assert sp.sigma_cm2[b] == pytest.approx(sb, rel=1e-9)
        assert W.sigma_HI(hi) < sp.sigma_cm2[b] < W.sigma_HI(lo)
        assert 0 < sp.eheat_erg[b] < (hi - 13.6) * W.EV


def test_configs_shapes():
    p = W.stromgren()
    assert p.grid == (32, 32, 32) and p.nsteps == 30 and len(p.source_ndot) == 1
    assert p.dx_phys_cm == pytest.approx(12 * W.KPC / 32)
    p = W.cosmo16(n=32, nsteps=3)
    assert len(p.source_ndot) == 16 and p.spectrum.nbins == 4
    assert np.all((p.source_ndot >= 1e51) & (p.source_ndot <= 1e52))
    assert W.mean_nH_comoving() == pytest.approx(1.894e-7, rel=2e-3)
