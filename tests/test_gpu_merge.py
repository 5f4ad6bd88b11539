"""Ray merging (Sec. 3.3, Eq. 4) on the GPU against the oracle on identical
seeded inputs.  The oracle merges by the section's definition in double
precision (content ranking, ang2pix on each cell's random sphere,
photon-weighted means rounded once); the GPU decides in single precision and
forms the means from exact integer sums of truncated weights.  Compared:
the merge-pixel decision (equal except within rounding of a pixel edge);
the merge step on the same rays (tests/merge_parity.py: identical groups,
merged ids, directions, photons, distances and levels, positions within the
stated bound, ambiguous rays counted and bounded); whole runs step by step,
the oracle merging the GPU's own rays after every march (each GPU step runs
in two stages and its marched rays are read back in between); the
ray-count ceiling of Eq. 4; batch members equal to the same simulation
alone."""
import dataclasses as dc

import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from merge_parity import compare_merge_step
from parity_util import BUDGET_RTOL, compare_fields, compare_rays

pytestmark = pytest.mark.gpu
S = 2 ** 21


def test_merge_pixel_probe_matches_oracle():
    # the GPU's single-precision decision equals the oracle's double-precision
    # ang2pix except within rounding of a pixel edge (a 4-unit nudge of the
    # direction reproduces it), and rotated pixel centres land in their pixel
    rng = np.random.default_rng(11)
    mism = total = 0
    for level in range(6):
        for key in (3, 70000, 5):
            Rq = oracle.merge_rotation(17, key, level + 3)
            v = rng.normal(size=(4000, 3))
            v /= np.linalg.norm(v, axis=1)[:, None]
            d = np.rint(v * (S - 1)).astype(np.int32)
            if level <= 3:      # and every rotated pixel centre
                d = np.vstack([d, [oracle.direction(level, p, Rq) for p in range(12 * 4 ** level)]])
            got = F.probe_merge_pixel(level, d, Rq)
            ref = np.array([oracle.merge_pixel(level, Rq, x) for x in d])
            for i in np.nonzero(got != ref)[0]:
                near = {oracle.merge_pixel(level, Rq, d[i] + s_ * e) for e in np.eye(3, dtype=np.int32)
                        for s_ in (-4, 4)}
                assert got[i] in near, (level, i, got[i], ref[i])
            if level <= 3:
                assert np.array_equal(got[4000:], np.arange(12 * 4 ** level))
            mism += int((got != ref).sum())
            total += len(d)
    assert mism <= 1e-3 * total, (mism, total)
    # one sphere per direction gives the same answers
    Rs = np.array([oracle.merge_rotation(5, c, 2) for c in range(64)], np.int32)
    d = np.rint(rng.normal(size=(64, 3)) * 2 ** 19).astype(np.int32)
    per = F.probe_merge_pixel(2, d, Rs)
    one = np.array([F.probe_merge_pixel(2, d[i:i + 1], Rs[i])[0] for i in range(64)])
    assert np.array_equal(per, one)


def _emitters(prob):
    cells, first = [], {}
    for ijk in map(tuple, prob.source_cells):
        if ijk not in first:
            first[ijk] = len(cells)
            cells.append(ijk)
    ndot = np.zeros(len(cells))
    for ijk, nd in zip(map(tuple, prob.source_cells), prob.source_ndot):
        ndot[first[ijk]] += nd
    return np.array(cells, np.int32), ndot


@pytest.mark.parametrize("n_ex,l_merge,with_merged", [(1.0, 0, False), (2.0, 1, True), (0.0, 0, True),
                                                      (0.5, 2, True)])
def test_merge_step_on_identical_rays(n_ex, l_merge, with_merged):
    # the same live rays (photons exact in single precision) merged by the GPU
    # kernels and by the oracle: identical groups and merged rays up to the
    # stated rounding (tests/merge_parity.py)
    prob = _prob(n_ex, l_merge, n=16, nsteps=8)
    plain = dc.replace(prob, options=dc.replace(prob.options, merge=False))
    dt, k = prob.dt, 6
    B = oracle.OracleSim(plain)
    if with_merged:                # a state that already holds merged rays and their children
        A = oracle.OracleSim(prob)
        for _ in range(k - 1):
            A.step(dt)
        B.set_rays(k - 2, A.rays())
        B.step(dt)
    else:
        for _ in range(k):
            B.step(dt)
    step = k - 1
    pre = B.rays()
    nref = 2.0 ** round(np.log2(pre["N"].max()))
    N32 = (pre["N"] / nref).astype(np.float32)
    thr32 = (pre["thr"] / nref).astype(np.float32)
    pre["N"], pre["thr"] = N32.astype(np.float64) * nref, thr32.astype(np.float64) * nref
    B.set_rays(step, pre)
    K = int(np.floor(n_ex * prob.ncell))
    cells, ndot = _emitters(prob)
    o = prob.options
    n0 = (ndot * dt / (12 * 4 ** o.l_src) / nref).astype(np.float32)
    gin = dict(pre, N=N32, thr=thr32)
    got = F.probe_merge(prob.grid, prob.spectrum.nbins, o.l_src, o.l_max, l_merge, K, o.seed, int(o.rotate), step,
                        o.eps_term, cells, n0, gin)
    got["N"] = got["N"] * nref
    got["thr"] = got["thr"] * nref
    B.apply_merge(dt, K)
    ref = B.rays()
    assert len(ref["level"]) < len(pre["level"])
    st = compare_merge_step(pre, got, B.rays(), prob, step, K, l_merge)
    assert st["merged"] > 0 and st["clean"] >= 0.8 * st["groups"], st
    assert (ref["birth"][ref["merged"]] == step).sum() > 0


def _step_local_run(prob, steps=None, capacity=1 << 22):
    """Run `prob` with merging on the GPU, each step in two stages: after the
    marches the GPU's rays are read back and the oracle merges those very
    rays; after the GPU's own merge the two results are compared.  Returns
    the per-step summaries and the GPU simulation (still open)."""
    steps = prob.nsteps if steps is None else steps
    g = F.Simulation(prob, ray_capacity=capacity)
    o = oracle.OracleSim(prob)
    K = int(np.floor(prob.options.n_ex * prob.ncell))
    out = []
    for s in range(steps):
        g.step_stage(prob.dt, 1)
        pre = g.rays()
        g.step_stage(prob.dt, 2)
        post = g.rays()
        o.set_rays(s, pre)
        o.apply_merge(prob.dt, K)
        st = compare_merge_step(pre, post, o.rays(), prob, s, K, prob.options.l_merge)
        b = g.budget()
        assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        out.append(st)
    o.close()
    return out, g


@pytest.mark.parametrize("n_ex,l_merge,seed", [(1.0, 0, 2), (2.0, 1, 4), (0.0, 0, 6)])
def test_merge_run_step_local(n_ex, l_merge, seed):
    # every step of a merging run: the GPU's merge of its own marched rays
    # equals the oracle's merge of the same rays (groups, merged rays)
    prob = _prob(n_ex, l_merge, seed=seed)
    stats, g = _step_local_run(prob)
    g.close()
    merged = sum(s["merged"] for s in stats)
    assert merged > 0
    assert sum(s["clean"] for s in stats) >= 0.8 * sum(s["groups"] for s in stats)


def _prob(n_ex, l_merge, n=16, nsteps=10, nsrc=8, seed=2):
    p = W.cosmo16(n=n, nsteps=nsteps, nsrc=nsrc, seed=seed)
    return dc.replace(p, options=dc.replace(p.options, merge=True, n_ex=n_ex, l_merge=l_merge))


def _table(r):
    key = np.stack([r["emitter"].astype(np.int64), r["birth"].astype(np.int64), r["level"].astype(np.int64),
                    r["pixel"].astype(np.int64), r["vertex"].astype(np.int64)], axis=1)
    order = np.lexsort(key.T[::-1])
    return key[order], {k: np.asarray(v)[order] for k, v in r.items()}


@pytest.mark.parametrize("n_ex,l_merge,seed", [(1.0, 0, 2), (2.0, 1, 4), (0.0, 0, 6)])
def test_merge_run_matches_oracle(n_ex, l_merge, seed):
    # Before the first step that merges, the two runs hold the same rays
    # element by element.  From then on each merge is compared step by step on
    # identical rays (test_merge_run_step_local); independent runs drift apart
    # (a ray within rounding of T_ref or of a pixel edge joins another group,
    # and merging amplifies it: the shot noise of Sec. 7.1), so the two whole
    # runs are compared on the quantities Sec. 7.1 validates merging with:
    # global ionised fraction and Gamma, ray count and photon budget.
    prob = _prob(n_ex, l_merge, seed=seed)
    g = F.Simulation(prob, ray_capacity=1 << 22)
    o = oracle.OracleSim(prob)
    n0_max = float(np.max(prob.source_ndot)) * prob.dt / 12
    first = None
    for s in range(prob.nsteps):
        g.step(prob.dt)
        o.step(prob.dt)
        gb, ob = g.budget(), o.budget()
        for b in (gb, ob):
            assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        assert abs(gb[0] - ob[0]) <= 1e-6 * ob[0]
        oc, gc = o.counts(), g.counts()
        gf, of = g.fields(), o.fields()
        orr = o.rays()
        if first is None and orr["merged"].any():
            first = s
        if first is None:
            compare_rays(g.rays(), orr, oc["near_threshold"], n0_max)
            compare_fields(gf, of)
            if oc["near_threshold"] == 0:
                assert gc["rays"] == oc["rays"]
                assert gc["segments_total"] == oc["segments_total"]
        else:
            assert abs(gc["rays"] - oc["rays"]) <= 0.02 * oc["rays"] + 16
            assert abs(gf["x_HII"].mean() - of["x_HII"].mean()) <= 0.01 * of["x_HII"].mean()
            assert abs(gf["gamma_HI"].mean() - of["gamma_HI"].mean()) <= 0.02 * of["gamma_HI"].mean()
            assert np.all(np.abs(gb - ob) <= 0.01 * ob[0])
    assert first is not None and first < prob.nsteps - 1
    g.close()
    o.close()


def test_merge_with_everything_exempt_equals_plain_run():
    p = _prob(1e9, 1)
    plain = dc.replace(p, options=dc.replace(p.options, merge=False))
    a = F.Simulation(p, ray_capacity=1 << 22)
    b = F.Simulation(plain, ray_capacity=1 << 22)
    for _ in range(p.nsteps):
        a.step(p.dt)
        b.step(p.dt)
    assert a.counts()["rays"] == b.counts()["rays"]
    assert a.counts()["segments_total"] == b.counts()["segments_total"]
    compare_fields(a.fields(), b.fields(), x_atol=1e-6, g_rtol=1e-5)
    assert not a.rays()["merged"].any()


def test_merge_ceiling_and_merged_geometry():
    # Eq. 4 after every merge: live rays <= floor(N_ex N_RT) (+ ties) + N_dir
    # per occupied cell; merged rays point along their merge pixel's centre
    prob = _prob(1.0, 1, n=24, nsteps=14, nsrc=16)
    g = F.Simulation(prob, ray_capacity=1 << 23)
    K = int(np.floor(prob.options.n_ex * prob.ncell))
    for s in range(prob.nsteps):
        g.step(prob.dt)
        c = g.counts()
        assert c["rays"] <= K + 48 * prob.ncell + 1024
    r = g.rays()
    m = np.nonzero(r["merged"] & (r["birth"] == prob.nsteps - 1) & ~r["vertex"] | (r["vertex"]))[0]
    assert len(m) > 0
    for i in m[:500]:
        if r["level"][i] != prob.options.l_merge and not r["vertex"][i]:
            continue
        local = int(r["emitter"][i]) - (1 << 31)
        Rq = oracle.merge_rotation(prob.options.seed, local, int(r["birth"][i]))
        assert np.array_equal(r["dir"][i], oracle.direction(prob.options.l_merge, int(r["pixel"][i]), Rq))
        cell = np.array([local % 24, (local // 24) % 24, local // 576])
        assert np.all(r["P"][i] // S == cell)
    b = g.budget()
    assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
    g.close()


def test_batch_members_with_merging_equal_alone():
    steps = 8
    probs = [_prob(1.0, l, n=n, nsteps=steps, nsrc=6, seed=20 + i)
             for i, (l, n) in enumerate([(0, 16), (1, 24), (0, 24)])]
    probs.append(dc.replace(probs[0], options=dc.replace(probs[0].options, merge=False)))
    B = F.Batch(max_sims=4, max_grid=24, nbins=4, ray_capacity=1 << 22, emitter_capacity=256, merge_l_max=1)
    slots = [B.add(p) for p in probs]
    for _ in range(steps):
        B.step()
    B.sync()
    for s, p in zip(slots, probs):
        a = F.Simulation(p, ray_capacity=1 << 22)
        for _ in range(steps):
            a.step(p.dt)
        bf, af = B.fields(s), a.fields()
        if not p.options.merge:
            compare_fields(bf, af, x_atol=1e-5, g_rtol=1e-4)
            assert B.counts(s)["rays"] == a.counts()["rays"]
            assert np.allclose(B.budget(s), a.budget(), rtol=1e-5)
        else:
            # two merging runs differ by rounding (the deposits are
            # single-precision reductions in any order), which moves rays
            # within rounding of T_ref or of a pixel edge into other groups:
            # compared on the quantities Sec. 7.1 validates merging with
            assert abs(bf["x_HII"].mean() - af["x_HII"].mean()) <= 0.01 * af["x_HII"].mean()
            assert abs(bf["gamma_HI"].mean() - af["gamma_HI"].mean()) <= 0.02 * af["gamma_HI"].mean()
            assert abs(B.counts(s)["rays"] - a.counts()["rays"]) <= 0.02 * a.counts()["rays"] + 16
            assert np.all(np.abs(B.budget(s) - a.budget()) <= 0.01 * a.budget()[0])
        a.close()
    B.close()


def test_merge_in_generalized_mode_matches_oracle():
    # merged rays and moving screens in the same march (Sec. 3.3 with
    # Sec. 4.2): cell by cell up to and including the first merge, then the
    # quantities Sec. 7.1 validates merging on -- ionised volume, mean Gamma,
    # ray count, photon budget -- (measured: volume within 4e-5, Gamma 7e-5,
    # budget 3e-5 of emitted, rays within 1)
    p = W.stromgren(n=32, nsteps=30)
    p = dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                   options=dc.replace(p.options, gen_mode=True, gamma_iters=5, merge=True, n_ex=0.05, l_merge=0))
    g = F.Simulation(p, ray_capacity=1 << 21)
    o = oracle.OracleSim(p)
    first = None
    for s in range(p.nsteps):
        g.step(p.dt)
        o.step(p.dt)
        gb, ob = g.budget(), o.budget()
        for b in (gb, ob):
            assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        xg, (xo, _) = g.ionized_volume(), o.gen_state()
        gf, of = g.fields(), o.fields()
        gc, oc = g.counts(), o.counts()
        if first is None:
            assert np.max(np.abs(xg - xo)) <= 5e-4
            if oc["near_threshold"] == 0:
                assert gc["rays"] == oc["rays"]
            if o.rays()["merged"].any():
                first = s
        assert abs(gc["rays"] - oc["rays"]) <= 0.02 * oc["rays"] + 16
        assert abs(xg.sum() - xo.sum()) <= 1e-3 * xo.sum()
        if of["gamma_HI"].mean() > 0:
            assert abs(gf["gamma_HI"].mean() - of["gamma_HI"].mean()) <= 1e-3 * of["gamma_HI"].mean()
        assert np.all(np.abs(gb - ob) <= 1e-3 * ob[0])
    assert first is not None and first < p.nsteps - 5
    assert g.rays()["merged"].sum() > 100
    g.close()
    o.close()


def test_merge_with_iteration_matches_oracle():
    # three passes of the Gamma - <n_HI> iteration and a merge after the last:
    # element by element up to the first merge, then Sec. 7.1's global criteria
    prob = _prob(1.0, 0, seed=2)
    prob = dc.replace(prob, options=dc.replace(prob.options, gamma_iters=3))
    g = F.Simulation(prob, ray_capacity=1 << 22)
    o = oracle.OracleSim(prob)
    n0_max = float(np.max(prob.source_ndot)) * prob.dt / 12
    first = None
    for s in range(prob.nsteps):
        g.step(prob.dt)
        o.step(prob.dt)
        gb, ob = g.budget(), o.budget()
        for b in (gb, ob):
            assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
        oc, gc = o.counts(), g.counts()
        gf, of = g.fields(), o.fields()
        orr = o.rays()
        if first is None and orr["merged"].any():
            first = s
        if first is None:
            compare_rays(g.rays(), orr, oc["near_threshold"], n0_max)
            compare_fields(gf, of)
        else:
            assert abs(gc["rays"] - oc["rays"]) <= 0.02 * oc["rays"] + 16
            assert abs(gf["x_HII"].mean() - of["x_HII"].mean()) <= 0.01 * of["x_HII"].mean()
            assert abs(gf["gamma_HI"].mean() - of["gamma_HI"].mean()) <= 0.02 * of["gamma_HI"].mean()
            assert np.all(np.abs(gb - ob) <= 0.01 * ob[0])
    assert first is not None and first < prob.nsteps - 1
    g.close()
    o.close()


@pytest.mark.parametrize("mode", ["generalized", "iteration"])
def test_merge_step_local_other_modes(mode):
    # each merge of a Generalized-mode run (merged rays and moving screens in
    # one march) and of a run with three passes of the Gamma - <n_HI>
    # iteration against the oracle's merge of the same rays
    if mode == "generalized":
        p = W.stromgren(n=32, nsteps=24)
        p = dc.replace(p, mfp=dc.replace(p.mfp, mode=3),
                       options=dc.replace(p.options, gen_mode=True, gamma_iters=5, merge=True, n_ex=0.05,
                                          l_merge=0))
    else:
        p = _prob(1.0, 0, seed=2)
        p = dc.replace(p, options=dc.replace(p.options, gamma_iters=3))
    stats, g = _step_local_run(p, capacity=1 << 21 if mode == "generalized" else 1 << 22)
    assert g.rays()["merged"].any()
    g.close()
    assert sum(s["merged"] for s in stats) > 0
    assert sum(s["clean"] for s in stats) >= 0.8 * sum(s["groups"] for s in stats)
