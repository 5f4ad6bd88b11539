"""The two headline workloads at full size, in the launch configuration the
bench times (autotuned march variant): outputs the oracle can compute one by
one (sampled rays' directions from their ids, bit-exact; their geometry),
and properties that hold at any size (photon conservation, bounds, segment
accounting, attenuation-only photon contents)."""
import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from paper_2409_04521_gb300 import autotune

pytestmark = pytest.mark.gpu
S = 2 ** 21


def _run(prob, capacity):
    g = F.Simulation(prob, ray_capacity=capacity, keep_diagnostics=True)
    autotune.tune(g, prob, nsteps=min(prob.nsteps, 40))
    for _ in range(prob.nsteps):
        g.step(prob.dt)
    g.sync()
    return g


def _check(prob, g, nsample=3000, seed=0):
    c = g.counts()
    assert c["step"] == prob.nsteps and c["rays"] > 0
    b = g.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-6 * b[0]
    seg = g.segment_counts()
    assert seg.sum() == c["segments_last"]
    f = g.fields()
    assert np.all((f["x_HII"] >= 0) & (f["x_HII"] <= 1))
    assert np.all(f["gamma_HI"] >= 0) and np.all(f["T"] > 0) and np.all(f["n_HI"] >= 0)
    r = g.rays()
    n = len(r["level"])
    assert n == c["rays"]
    rng = np.random.default_rng(seed)
    idx = rng.choice(n, size=min(nsample, n), replace=False)
    # emitters in order of first appearance of their cell
    cells, first = [], {}
    for ijk in map(tuple, prob.source_cells):
        if ijk not in first:
            first[ijk] = len(cells)
            cells.append(ijk)
    ndot = np.zeros(len(cells))
    for ijk, nd in zip(map(tuple, prob.source_cells), prob.source_ndot):
        ndot[first[ijk]] += nd
    grid = np.array(prob.grid, np.int32)
    o = prob.options
    K = oracle.split_table(o.n_ray_min)
    for i in idx:
        e, bi, lv, px = int(r["emitter"][i]), int(r["birth"][i]), int(r["level"][i]), int(r["pixel"][i])
        _, Rq = oracle.rotation(o.seed, e, bi, o.rotate)
        assert np.array_equal(r["dir"][i], oracle.direction(lv, px, Rq))
        # the ray survived its last march: it did not leave the box (a child
        # made at the end of that march has not marched on its own yet)
        age = prob.nsteps - 1 - bi
        born_now = lv > o.l_src and age + 1 >= K[lv - 1] and age < K[lv - 1]
        if not born_now:
            p0 = (2 * np.array(cells[e], np.int64) + 1) * (S // 2) + age * r["dir"][i].astype(np.int64)
            _, _, esc = oracle.traverse(p0, r["dir"][i], grid)
            assert not esc
        # photons only decrease along a ray and it is above its termination threshold
        n0 = ndot[e] * prob.dt / (12 * 4 ** o.l_src) * 4.0 ** (-(lv - o.l_src))
        tot = r["N"][i].sum()
        assert tot <= n0 * (1 + 1e-5)
        assert tot >= o.eps_term * n0 * (1 - 1e-4)


def test_cosmo16_full_size():
    prob = W.cosmo16()
    g = _run(prob, 200_000_000)
    _check(prob, g)
    g.close()


def test_cosmo20k_full_size():
    prob = W.cosmo20k()
    g = _run(prob, 30_000_000)
    _check(prob, g)
    g.close()
