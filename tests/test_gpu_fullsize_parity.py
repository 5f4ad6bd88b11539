"""Oracle parity at the configurations' stated sizes (Sec. 5.4's Test 4 shape
at 128^3, Sec. 7.2's 200^3 cosmological shape with 2e4 sources, a 96^3
member of the uneven batch, a served request stream holding a 160^3
request), element by element: live rays (ids and directions bit-exact,
photons within 2e-4), ray-cell segments per cell (exact), Gamma_HI (1e-4
relative), x_HII (1e-3 absolute), T (2e-3 relative) and the photon budget,
over the first RT steps the oracle finishes in seconds to a minute.  The
march runs in every launch variant the autotuner may pick for the bench, so
whichever it times is covered.  Each comparison appends a row of max and
median errors per field to the file named by FLEXRT_ERRTABLE."""
import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from paper_2409_04521_gb300 import autotune, serve
from parity_util import (budget_checks, compare_fields, compare_rays, field_errors, record_errors)

pytestmark = pytest.mark.gpu


def _oracle_checkpoints(prob, checkpoints):
    o = oracle.OracleSim(prob)
    out = {}
    for s in range(1, max(checkpoints) + 1):
        o.step(prob.dt)
        if s in checkpoints:
            out[s] = dict(rays=o.rays(), fields=o.fields(), seg=o.segment_counts(), budget=o.budget(),
                          counts=o.counts())
    o.close()
    return out


def _n0_max(prob):
    return float(np.max(prob.source_ndot)) * prob.dt / (12 * 4 ** prob.options.l_src)


def _compare(name, prob, g, ref, step, variant, T_rtol=2e-3):
    oc, gc = ref["counts"], g.counts()
    budget_checks(g.budget(), ref["budget"])
    nd = compare_rays(g.rays(), ref["rays"], oc["near_threshold"], _n0_max(prob))
    if oc["near_threshold"] == 0:
        assert gc["rays"] == oc["rays"] and gc["segments_last"] == oc["segments_last"]
        assert gc["segments_total"] == oc["segments_total"]
        assert np.array_equal(g.segment_counts(), ref["seg"])
    gf = g.fields()
    compare_fields(gf, ref["fields"], T_rtol=T_rtol)
    record_errors(name, step, field_errors(gf, ref["fields"]), variant=list(variant), rays=gc["rays"],
                  straddles=oc["near_threshold"], rays_one_side=nd)


def _variant_run(name, prob, variants, checkpoints, capacity, last_only=()):
    ref = _oracle_checkpoints(prob, checkpoints)
    for v in variants:
        g = F.Simulation(prob, ray_capacity=capacity, keep_diagnostics=True)
        g.set_launch(*v)
        for s in range(1, max(checkpoints) + 1):
            g.step(prob.dt)
            if s in checkpoints and (v not in last_only or s == max(checkpoints)):
                _compare(name, prob, g, ref[s], s, v)
        g.close()


def test_cosmo16_full_size_matches_oracle():
    # 128^3, 16 sources, 4 bins, temperature evolution: the bench workload,
    # its first 15 RT steps, every launch of the march the autotuner can
    # choose (the non-default launch shapes at the last checkpoint)
    prob = W.cosmo16()
    shaped = [v for v in autotune.candidates() if v not in autotune.CANDIDATES]
    _variant_run("cosmo16 128^3", prob, autotune.CANDIDATES + shaped, (5, 10, 15), 40_000_000, last_only=shaped)


def test_cosmo20k_full_size_matches_oracle():
    # 200^3, 2e4 sources, sub-grid mean free path law, 3 bins: first 6 steps
    prob = W.cosmo20k()
    _variant_run("cosmo20k 200^3", prob, [(0, 2, 0), (0, 4, 0), (1, 3, 0), (0, 4, 0, 128, 128)], (3, 6),
                 30_000_000)


def test_batch64_member_96_matches_oracle():
    # a 96^3 member advanced inside a batch of uneven members (one set of
    # launches per step, replayed from a CUDA graph) against the oracle
    members = W.batch64(count=12, nsteps=12)
    big = [i for i, p in enumerate(members) if p.grid[0] == 96]
    assert big
    k = big[0]
    ref = _oracle_checkpoints(members[k], (6, 12))
    for v in [(0, 2, 0), (0, 4, 0), (0, 3, 2, 128, 2048)]:
        B = F.Batch(max_sims=16, max_grid=96, nbins=3, ray_capacity=1 << 24, emitter_capacity=1024,
                    keep_diagnostics=True)
        B.set_launch(*v)
        slots = [B.add(p) for p in members]
        for s in range(1, 13):
            B.step()
            if s in (6, 12):
                B.sync()
                view = _BatchMember(B, slots[k])
                _compare("batch64 member 96^3", members[k], view, ref[s], s, v)
        B.close()


class _BatchMember:
    """A batch member seen through the single-simulation getters."""

    def __init__(self, batch, slot):
        self.b, self.s = batch, slot

    def counts(self):
        return self.b.counts(self.s)

    def budget(self):
        return self.b.budget(self.s)

    def rays(self):
        return self.b.rays(self.s)

    def fields(self):
        return self.b.fields(self.s)

    def segment_counts(self):
        return self.b.segment_counts(self.s)


def test_served_stream_with_160_request_matches_oracle():
    # a short request stream served by continuous batching, one request at
    # 160^3 (the largest grid of the served config) with 50 steps: its
    # fields when it retires against the oracle after the same 50 steps
    reqs = [(0.0, W.batch_member(100_006, (160,), 50, shared_fields=True)),
            (0.001, W.batch_member(100_010, (32, 64), 50, shared_fields=True)),
            (0.002, W.batch_member(100_011, (96,), 60, shared_fields=True))]
    results, stats = serve.serve(reqs, hbm_budget_bytes=12e9, max_sims=8, max_grid=160, keep_fields=True)
    assert stats["requests"] == 3
    for r in results:
        prob = reqs[r.rid][1]
        if prob.grid[0] not in (160, 96):
            continue
        o = oracle.OracleSim(prob)
        for _ in range(prob.nsteps):
            o.step(prob.dt)
        of = o.fields()
        compare_fields(r.fields, of, T_rtol=2e-3)
        assert r.segments == o.counts()["segments_total"] or o.counts()["near_threshold"] > 0
        record_errors(f"served request {prob.grid[0]}^3", prob.nsteps, field_errors(r.fields, of))
        o.close()
