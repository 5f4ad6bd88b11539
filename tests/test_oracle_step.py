"""Pins of the oracle's whole step (emission, march, deposit, termination,
split, chemistry) against analytic solutions and brute force:

* the Stromgren I-front law (Sec. 5.1, Eq. 21-24),
* exact photon conservation (emitted = absorbed + escaped + in flight),
* pure-exponential attenuation for a constant mean free path (Eq. 13),
* the optically thin rate Gamma = Ndot sigma / (4 pi r^2) (Eq. 14 limit),
* exact long characteristics through a frozen inhomogeneous medium,
* the single-cell closed form of Eq. 17 and its reduction to Eq. 5.
"""
import dataclasses as dc
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

S = 2 ** 21


def retarded_radius(t, rS, trec, c_cells_per_s, dx):
    """Analytic R(t) of Eq. 21 evaluated at the retarded time t - R/c."""
    R = 0.0
    for _ in range(200):
        tr = max(t - R * dx / (c_cells_per_s * dx), 0.0)
        R = rS * (1 - math.exp(-tr / trec)) ** (1 / 3)
    return R


def test_stromgren_front_and_budget():
    prob = W.stromgren()
    sim = oracle.OracleSim(prob)
    dx = prob.dx_phys_cm
    nH, a, Nd = 1e-3, 2.59e-13, 3e48
    rS = (3 * Nd / (4 * math.pi * a * nH * nH)) ** (1 / 3) / dx   # Eq. 23 (n_H squared)
    trec = 1 / (a * nH)                                            # Eq. 24
    assert rS == pytest.approx(12.13, abs=0.01)
    Rprev = 0
    for s in range(prob.nsteps):
        sim.step(prob.dt)
        b = sim.budget()
        assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-12 * b[0]
        R = oracle.ifront_radius_cells(sim.fields()["x_HII"], prob.options.x_init)
        assert R >= Rprev
        Rprev = R
    t = prob.nsteps * prob.dt
    R_inst = rS * (1 - math.exp(-t / trec)) ** (1 / 3)             # Eq. 21
    R_ret = retarded_radius(t, rS, trec, 1.0 / prob.dt, dx)
    assert R_inst == pytest.approx(7.29, abs=0.01)
    assert abs(R - R_ret) < 1.0
    assert 0 < R_inst - R < 1.5


def _uniform(n, nH, ndot, nsteps, **opt):
    prob = W.stromgren(n=n, nsteps=nsteps)
    prob.nH = np.full(n ** 3, nH)
    prob.source_ndot = np.array([ndot])
    prob.options = dc.replace(prob.options, **opt)
    return prob


def test_constant_mfp_pure_exponential():
    # mode 1: kappa = 1/lambda everywhere, n_HI ~ 0: after j steps every ray
    # of a shell has been attenuated by exp(-j dx/lambda) and splits conserve
    # photons, so in flight = Ndot dt sum_j exp(-j dx / lambda)
    n, nsteps = 24, 9
    prob = _uniform(n, 1e-30, 1e50, nsteps)
    lam_cells = 3.7
    prob.mfp = W.Mfp(mode=1, lambda0_cm_comoving=lam_cells * prob.dx_phys_cm)
    sim = oracle.OracleSim(prob)
    for s in range(nsteps):
        sim.step(prob.dt)
        b = sim.budget()
        q = math.exp(-1 / lam_cells)
        expect = 1e50 * prob.dt * sum(q ** j for j in range(1, s + 2))
        assert b[3] == pytest.approx(expect, rel=1e-12)
        assert b[2] == 0.0


def test_optically_thin_rate_inverse_square():
    # Eq. 14 limit: in a transparent medium each shell of packets crosses a
    # cell once per step and Gamma -> Ndot sigma <1/(4 pi r^2)>.
    n, nsteps = 32, 15
    prob = _uniform(n, 1e-30, 1e50, nsteps)
    sim = oracle.OracleSim(prob)
    for _ in range(nsteps):
        sim.step(prob.dt)
    g = sim.fields()["gamma_HI"].reshape(n, n, n)
    c = np.array([16.5, 16.5, 16.5])
    k, j, i = np.indices((n, n, n))
    r = np.sqrt((i + 0.5 - c[0]) ** 2 + (j + 0.5 - c[1]) ** 2 + (k + 0.5 - c[2]) ** 2)
    dx = prob.dx_phys_cm
    sig = 6.3e-18
    ratio = g * 4 * math.pi * (r * dx) ** 2 / (1e50 * sig)
    for r0 in (4, 6, 8, 10, 12):
        shell = (r >= r0) & (r < r0 + 1)
        assert ratio[shell].mean() == pytest.approx(1.0, abs=0.04), r0


def exact_tau(p_start, d, steps, kap_cells, n):
    """Optical depth along the straight line p_start + t d, t in [0, steps],
    by exact rational cell crossings (a brute-force long characteristic)."""
    p0 = [int(x) for x in p_start]
    d = [int(x) for x in d]
    T = int(steps)
    ts = {Fraction(0), Fraction(T)}
    for a in range(3):
        if d[a] == 0:
            continue
        lo, hi = sorted((p0[a], p0[a] + T * d[a]))
        for m in range(-(-lo // S), hi // S + 1):
            t = Fraction(m * S - p0[a], d[a])
            if 0 < t < T:
                ts.add(t)
    ts = sorted(ts)
    tau = 0.0
    for t0, t1 in zip(ts[:-1], ts[1:]):
        tm = (t0 + t1) / 2
        c = [math.floor((p0[a] + tm * d[a]) / S) for a in range(3)]
        tau += kap_cells[c[2], c[1], c[0]] * float(t1 - t0)
    return tau


def test_long_characteristics_frozen_medium():
    # no splitting (l_max = l_src), no recombination, a faint source: the
    # medium stays frozen and each packet must carry N0 exp(-tau) with tau
    # the exact line integral from the source-cell centre.
    n, nsteps = 8, 3
    rng = np.random.default_rng(4)
    prob = W.stromgren(n=n, nsteps=nsteps)
    prob.source_cells = np.array([[3, 4, 2]], np.int32)
    prob.source_ndot = np.array([1e30])
    prob.nH = rng.uniform(0.2e-3, 3e-3, n ** 3)
    prob.options = dc.replace(prob.options, l_src=2, l_max=2, alpha_B_const=0.0)
    sim = oracle.OracleSim(prob)
    for _ in range(nsteps):
        sim.step(prob.dt)
    rays = sim.rays()
    kap = (prob.nH * (1 - prob.options.x_init) * 6.3e-18 * prob.dx_phys_cm).reshape(n, n, n)
    N0 = 1e30 * prob.dt / (12 * 16)
    c = (2 * prob.source_cells[0].astype(np.int64) + 1) * (S // 2)
    assert len(rays["level"]) > 50
    for i in range(len(rays["level"])):
        age = nsteps - rays["birth"][i]
        tau = exact_tau(c, rays["dir"][i], age, kap, [n] * 3)
        assert rays["N"][i, 0] == pytest.approx(N0 * math.exp(-tau), rel=1e-11)


def test_single_cell_closed_form_and_eq5_identity():
    # one cell, one step: every ray exits at the distance t_a = 0.5/|v_a|
    # (cells); absorbed = sum N0 (1 - exp(-kappa dx t_exit)) and escaped is
    # the rest.  With kappa = n_HI sigma, Eq. 17 reduces to Eq. 5:
    # Gamma n_HI V dt = absorbed photons.
    prob = W.stromgren(n=1, nsteps=1)
    prob.source_cells = np.array([[0, 0, 0]], np.int32)
    nH = 2e-3
    prob.nH = np.array([nH])
    prob.options = dc.replace(prob.options, seed=77)
    sim = oracle.OracleSim(prob)
    sim.step(prob.dt)
    R, Rq = oracle.rotation(77, 0, 0)
    dx = prob.dx_phys_cm
    nHI = nH * (1 - prob.options.x_init)
    kap = nHI * 6.3e-18
    N0 = 3e48 * prob.dt / 12
    absorbed = escaped = 0.0
    for p in range(12):
        d = oracle.direction(0, p, Rq).astype(float)
        t_exit = min(S / 2 / abs(da) for da in d if da != 0)
        absorbed += N0 * -math.expm1(-kap * dx * t_exit)
        escaped += N0 * math.exp(-kap * dx * t_exit)
    b = sim.budget()
    assert b[1] == pytest.approx(absorbed, rel=1e-13)
    assert b[2] == pytest.approx(escaped, rel=1e-13)
    gamma = sim.fields()["gamma_HI"][0]
    assert gamma * nHI * dx ** 3 * prob.dt == pytest.approx(absorbed, rel=1e-13)


def test_sources_in_one_cell_form_one_emitter():
    p1 = W.stromgren(n=12, nsteps=4)
    p1.source_cells = np.array([[5, 6, 7], [5, 6, 7]], np.int32)
    p1.source_ndot = np.array([1e48, 2e48])
    p2 = W.stromgren(n=12, nsteps=4)
    p2.source_cells = np.array([[5, 6, 7]], np.int32)
    p2.source_ndot = np.array([3e48])
    s1, s2 = oracle.OracleSim(p1), oracle.OracleSim(p2)
    assert s1.num_emitters() == 1
    for _ in range(4):
        s1.step(p1.dt)
        s2.step(p2.dt)
    assert np.allclose(s1.fields()["gamma_HI"], s2.fields()["gamma_HI"], rtol=1e-14, atol=0)


def test_escape_and_termination_budget():
    # small box: rays escape; dense gas: rays terminate.  Both keep the
    # budget exact.
    prob = _uniform(6, 5e-2, 3e48, 8)
    sim = oracle.OracleSim(prob)
    for _ in range(8):
        sim.step(prob.dt)
        b = sim.budget()
        assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-12 * b[0]
    prob = _uniform(6, 1e-6, 3e48, 8)
    sim = oracle.OracleSim(prob)
    for _ in range(8):
        sim.step(prob.dt)
    b = sim.budget()
    assert b[2] > 0.5 * b[0]
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-12 * b[0]
