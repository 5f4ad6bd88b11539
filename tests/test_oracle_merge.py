"""Pins of the oracle's ray merging (Sec. 3.3, Eq. 4; Sec. 7.1).

The merge decides integers (exempt or not, which rays share a group) from
floating point, so its pixel function is pinned against an independent
double-precision ang2pix and against the exact pixel centres; the merge step
is checked against what the section fixes whatever the reading: photons
conserved, the N_ex*N_RT brightest rays untouched, one ray per (cell, merge
pixel) group, the ray-count ceiling of Eq. 4; and the global ionised fraction
and Gamma stay within the 1-2 % of the unmerged run that Sec. 7.1 reports.
"""
import dataclasses as dc
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W
from healpix_ref import ang2pix_nest

S = 2 ** 21


def _rot(seed, key, step):
    return oracle.rotation(seed, key, step)[1]


def test_merge_rotation_is_a_uniform_random_rotation():
    # drawn like an emitter's sphere (key 2^31 + cell): orthonormal to the
    # 2^-24 quantisation, proper, and uniform on SO(3) (E[R] = 0,
    # E[R_ij^2] = 1/3)
    Rs = np.array([oracle.merge_rotation(9, c, s) for c in range(2000) for s in (0, 7)], np.float64) / 2 ** 24
    for R in Rs[:200]:
        assert np.abs(R @ R.T - np.eye(3)).max() < 2e-7
        assert abs(np.linalg.det(R) - 1.0) < 3e-7
    n = len(Rs)
    assert np.all(np.abs(Rs.mean(0)) < 4.0 * np.sqrt(1.0 / 3.0 / n))
    assert np.all(np.abs((Rs ** 2).mean(0) - 1.0 / 3.0) < 4.0 * np.sqrt(4.0 / 45.0 / n))
    assert np.array_equal(oracle.merge_rotation(9, 5, 3, rotate=False), np.eye(3, dtype=np.int32) * 2 ** 24)
    # the emitters' generator with the key 2^31 + cell
    assert np.array_equal(oracle.merge_rotation(9, 5, 3), oracle.rotation(9, (1 << 31) + 5, 3)[1])
    # distinct cells and steps draw distinct spheres
    assert not np.array_equal(oracle.merge_rotation(9, 5, 3), oracle.merge_rotation(9, 6, 3))
    assert not np.array_equal(oracle.merge_rotation(9, 5, 3), oracle.merge_rotation(9, 5, 4))


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_merge_pixel_of_pixel_centres(level):
    # a rotated pixel centre falls in its own pixel on the same rotated sphere
    for k, (seed, key, step) in enumerate([(1, 0, 0), (7, (1 << 31) + 5, 3), (99, (1 << 31) + 4095, 40)]):
        Rq = _rot(seed, key, step)
        for p in range(12 * 4 ** level):
            d = oracle.direction(level, p, Rq)
            assert oracle.merge_pixel(level, Rq, d) == p


def test_merge_pixel_matches_independent_ang2pix():
    # random fixed-point directions on random spheres: the oracle's pixel
    # equals an independently written ang2pix of R^T d (tests/healpix_ref)
    # except within rounding distance of a pixel edge
    rng = np.random.default_rng(5)
    n = 6000
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    d = np.rint(v * (S - 1)).astype(np.int32)
    mism = 0
    for i in range(n):
        level = i % 5
        Rq = _rot(3, (1 << 31) + i, i % 17)
        u = Rq.astype(np.float64).T @ d[i].astype(np.float64)
        got = oracle.merge_pixel(level, Rq, d[i])
        ref = ang2pix_nest(level, u)
        if got != ref:
            mism += 1
            eps = 1e-9 * np.linalg.norm(u)
            near = {ang2pix_nest(level, u + eps * e) for e in np.vstack([np.eye(3), -np.eye(3)])}
            assert got in near, (i, level, got, ref)
    assert mism <= 2


def test_merge_pixel_nested_and_equal_area():
    # NESTED numbering: the level-(l+1) pixel of a direction lies inside its
    # level-l pixel (p_(l+1) >> 2 == p_l); equal-area pixels: uniform random
    # directions fill the 12*4^l pixels of a rotated sphere evenly (Poisson)
    rng = np.random.default_rng(8)
    n = 48000
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    d = np.rint(v * (S - 1)).astype(np.int32)
    Rq = _rot(4, (1 << 31) + 77, 5)
    level = 2
    npix = 12 * 4 ** level
    counts = np.zeros(npix, np.int64)
    for i in range(n):
        p = oracle.merge_pixel(level, Rq, d[i])
        counts[p] += 1
        if i % 40 == 0:
            assert oracle.merge_pixel(level + 1, Rq, d[i]) >> 2 == p
            assert oracle.merge_pixel(level - 1, Rq, d[i]) == p >> 2
    mu = n / npix
    assert np.all(np.abs(counts - mu) <= 5.0 * np.sqrt(mu))
    chi2 = float(((counts - mu) ** 2 / mu).sum())
    assert chi2 < npix + 5.0 * np.sqrt(2.0 * npix)


@pytest.mark.parametrize("lm,L", [(0, 0), (0, 1), (0, 3), (1, 1), (1, 2), (1, 4)])
def test_vertex_children(lm, L):
    rng = np.random.default_rng(lm * 10 + L)
    for pm in rng.choice(12 * 4 ** lm, size=4, replace=False):
        pm = int(pm)
        c1 = [oracle.vertex_child(lm, pm, L, 1, c) for c in range(4)]
        if L == lm:                                   # a true pixel: its NESTED children
            assert c1 == [4 * pm + c for c in range(4)]
        # the four level-(L+1) descendants of pm nearest to pm's centre
        depth = L + 1 - lm
        desc = range(pm << (2 * depth), (pm + 1) << (2 * depth))
        centre = oracle.pix2vec(lm, pm)
        ang = sorted((float(np.arccos(min(1.0, np.dot(centre, oracle.pix2vec(L + 1, q))))), q) for q in desc)
        assert sorted(c1) == sorted(q for _, q in ang[:4])
        if len(ang) > 4:
            assert ang[3][0] < ang[4][0] - 1e-9
        # deeper splits: distinct descendants of the four children
        c2 = [oracle.vertex_child(lm, pm, L, 2, c) for c in range(16)]
        assert len(set(c2)) == 16
        assert [q >> 2 for q in c2] == [c1[c >> 2] for c in range(16)]


def _problem(n=16, nsteps=8, nsrc=8, **kw):
    p = W.cosmo16(n=n, nsteps=nsteps, nsrc=nsrc)
    return dc.replace(p, options=dc.replace(p.options, **kw))


def _end_points(prob, r, step):
    """End point (fixed point) of each live ray after the march of `step`."""
    cells, first = [], {}
    for ijk in map(tuple, prob.source_cells):
        if ijk not in first:
            first[ijk] = len(cells)
            cells.append(ijk)
    out = np.zeros((len(r["level"]), 3), np.int64)
    for i in range(len(out)):
        d = r["dir"][i].astype(np.int64)
        if r["merged"][i]:
            out[i] = r["P"][i] + (step - r["birth"][i]) * d
        else:
            c = (2 * np.array(cells[r["emitter"][i]], np.int64) + 1) * (S // 2)
            out[i] = c + (step - r["birth"][i] + 1) * d
    return out


def _exact_mean(w, x):
    """Exact rational photon-weighted mean sum(w x) / sum(w) of doubles."""
    W = sum(Fraction(float(v)) for v in w)
    return sum(Fraction(float(v)) * Fraction(int(y)) for v, y in zip(w, x)) / W


def _rounded_once(got, exact):
    # rounded to nearest once: within half a unit of the exact mean (exact
    # halves may go either way)
    return abs(Fraction(int(got)) - exact) <= Fraction(1, 2)


def _key(r, i):
    return (int(r["emitter"][i]), int(r["birth"][i]), int(r["level"][i]), int(r["pixel"][i]), bool(r["vertex"][i]))


@pytest.mark.parametrize("n_ex,l_merge", [(1.0, 0), (2.0, 1)])
def test_merge_step_invariants(n_ex, l_merge):
    prob = _problem(merge=False, n_ex=n_ex, l_merge=l_merge)
    o = oracle.OracleSim(prob)
    for _ in range(prob.nsteps):
        o.step(prob.dt)
    step = prob.nsteps - 1
    pre = o.rays()
    b0 = o.budget()
    o.apply_merge(prob.dt)
    post = o.rays()
    b1 = o.budget()
    n, ncell = len(pre["level"]), prob.ncell
    K = math.floor(n_ex * ncell)
    assert K < n
    # photons per bin conserved, budget identity intact
    assert np.allclose(post["N"].sum(0), pre["N"].sum(0), rtol=1e-12)
    assert abs(b1[0] - b1[1] - b1[2] - b1[3]) <= 1e-11 * b1[0]
    assert b1[3] == pytest.approx(b0[3], rel=1e-12)
    # exempt: photon content at least the K-th largest (Sec. 3.3)
    T = pre["N"].sum(1)
    Tstar = np.sort(T)[::-1][K - 1]
    exempt = T >= Tstar
    assert exempt.sum() >= K
    post_keys = {_key(post, i): i for i in range(len(post["level"]))}
    for i in np.nonzero(exempt)[0]:
        j = post_keys[_key(pre, i)]
        assert np.array_equal(post["N"][j], pre["N"][i])
    # groups of the non-exempt rays by (end cell, merge pixel)
    ends = _end_points(prob, pre, step)
    grid = np.array(prob.grid)
    groups = {}
    kept = 0
    for i in np.nonzero(~exempt)[0]:
        c = ends[i] // S
        if np.any(c < 0) or np.any(c >= grid):
            kept += 1
            continue
        local = int((c[2] * grid[1] + c[1]) * grid[0] + c[0])
        Rq = oracle.merge_rotation(prob.options.seed, local, step)
        groups.setdefault((local, oracle.merge_pixel(l_merge, Rq, pre["dir"][i])), []).append(i)
    singles = sum(1 for g in groups.values() if len(g) == 1)
    multi = {k: g for k, g in groups.items() if len(g) > 1}
    assert multi, "no group merged"
    # Eq. 4: after the merge at most N_ex*N_RT (+ ties) + N_dir rays per cell
    assert len(post["level"]) == exempt.sum() + kept + len(groups)
    assert len(post["level"]) <= exempt.sum() + kept + 12 * 4 ** l_merge * ncell
    new = np.nonzero(post["merged"] & (post["birth"] == step))[0]
    assert len(new) == len(multi)
    for j in new:
        local = int(post["emitter"][j]) - (1 << 31)
        pm = int(post["pixel"][j])
        g = multi[(local, pm)]
        Rq = oracle.merge_rotation(prob.options.seed, local, step)
        assert np.array_equal(post["dir"][j], oracle.direction(l_merge, pm, Rq))
        assert np.allclose(post["N"][j], pre["N"][g].sum(0), rtol=1e-13)
        # Sec. 3.3: position, distance travelled and level are photon-
        # weighted averages of the constituents' (rounded once to the grid)
        w = T[g]
        cell = np.array([local % grid[0], (local // grid[0]) % grid[1], local // (grid[0] * grid[1])])
        assert np.all(post["P"][j] // S == cell)
        for a in range(3):
            assert _rounded_once(post["P"][j][a], _exact_mean(w, ends[g][:, a]))
        dist = np.where(pre["merged"][g], pre["A"][g] + step - pre["birth"][g], step - pre["birth"][g] + 1)
        assert _rounded_once(post["A"][j], _exact_mean(w, dist))
        lbar = _exact_mean(w, pre["level"][g])
        assert post["level"][j] >= l_merge and (post["level"][j] == l_merge or _rounded_once(post["level"][j], lbar))
        assert post["vertex"][j] == (post["level"][j] > l_merge)
    # every non-exempt ray alone in its group is kept unchanged
    for g in groups.values():
        if len(g) == 1:
            j = post_keys[_key(pre, g[0])]
            assert np.array_equal(post["N"][j], pre["N"][g[0]])
    assert singles + len(multi) == len(groups)


def test_merge_with_everything_exempt_changes_nothing():
    a = oracle.OracleSim(_problem(merge=False))
    b = oracle.OracleSim(_problem(merge=True, n_ex=1e9, l_merge=1))
    p = _problem()
    for _ in range(p.nsteps):
        a.step(p.dt)
        b.step(p.dt)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k])
    ra, rb = a.rays(), b.rays()
    assert np.array_equal(ra["pixel"], rb["pixel"]) and np.array_equal(ra["N"], rb["N"])


def test_merging_keeps_global_averages():
    # Sec. 7.1 (Test 4 with merging, N_ex = 16, 12 merge directions): the
    # volume- and mass-weighted ionised fraction and mean Gamma stay within
    # 1-2 % of the unmerged run at all times, at a fraction of its ray work
    p = W.cosmo16(n=24, nsteps=30, nsrc=16)

    def run(q):
        o = oracle.OracleSim(q)
        out = []
        for _ in range(q.nsteps):
            o.step(q.dt)
            f = o.fields()
            out.append((f["x_HII"].mean(), (f["x_HII"] * q.nH).sum() / q.nH.sum(), f["gamma_HI"].mean()))
        return np.array(out), o.counts()["segments_total"], o

    base, seg0, _ = run(p)
    merged, seg1, o = run(dc.replace(p, options=dc.replace(p.options, merge=True, l_merge=0, n_ex=16.0)))
    ratio = merged[3:] / base[3:]          # from the third step, when Gamma is non-zero everywhere lit
    assert np.all(np.abs(ratio - 1.0) <= 0.02), np.abs(ratio - 1.0).max(0)
    assert seg0 > 2.5 * seg1
    b = o.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= 1e-10 * b[0]
    r = o.rays()
    assert r["merged"].any() and r["vertex"].any()
