"""Batched and continuously batched simulations (flexrt_batch_*): every
member must give the same result as the same simulation run alone through
flexrt_create, within the stated tolerances, and match the oracle."""
import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F
import workloads as W
from parity_util import X_ATOL, GAMMA_RTOL, compare_fields

pytestmark = pytest.mark.gpu


def _members(n, steps, sizes=(16, 24, 32)):
    return [W.batch_member(s, sizes=sizes, nsteps=steps) for s in range(n)]


def _alone(prob, steps):
    s = F.Simulation(prob, ray_capacity=1 << 21)
    for _ in range(steps):
        s.step(prob.dt)
    out = (s.fields(), s.budget(), s.counts())
    s.close()
    return out


def _same(f_batch, b_batch, c_batch, ref):
    f, b, c = ref
    compare_fields(f_batch, f, x_atol=X_ATOL, g_rtol=GAMMA_RTOL)
    assert np.allclose(b_batch, b, rtol=1e-5, atol=1e-6 * b[0])
    assert c_batch["step"] == c["step"]
    assert abs(c_batch["segments_total"] - c["segments_total"]) <= 1e-6 * c["segments_total"] + 4


@pytest.mark.parametrize("use_graph", [True, False])
def test_members_equal_alone(use_graph):
    steps = 10
    probs = _members(5, steps)
    B = F.Batch(max_sims=8, max_grid=32, nbins=3, ray_capacity=1 << 22, emitter_capacity=1024,
                use_graph=use_graph)
    slots = [B.add(p) for p in probs]
    for _ in range(steps):
        B.step()
    B.sync()
    for s, p in zip(slots, probs):
        _same(B.fields(s), B.budget(s), B.counts(s), _alone(p, steps))
    B.close()


def test_member_matches_oracle():
    steps = 8
    probs = _members(3, steps)
    B = F.Batch(max_sims=4, max_grid=32, nbins=3, ray_capacity=1 << 22, emitter_capacity=256)
    slots = [B.add(p) for p in probs]
    for _ in range(steps):
        B.step()
    for s, p in zip(slots, probs):
        o = oracle.OracleSim(p)
        for _ in range(steps):
            o.step(p.dt)
        compare_fields(B.fields(s), o.fields())
        ob, gb = o.budget(), B.budget(s)
        assert np.all(np.abs(gb - ob) <= 1e-4 * ob[0])
        assert abs(gb[0] - gb[1] - gb[2] - gb[3]) <= 1e-6 * gb[0]
        rays = B.rays(s)
        assert len(rays["level"]) == B.counts(s)["rays"]
    B.close()


def test_continuous_admission_and_retirement():
    # members arrive at different steps, run their own number of steps, and
    # leave; freed slots, cells and emitters are reused by later members
    plan = [(0, 6), (0, 9), (2, 5), (3, 8), (7, 6), (9, 4)]   # (arrival step, steps)
    probs = [W.batch_member(20 + i, sizes=(16, 24), nsteps=n) for i, (_, n) in enumerate(plan)]
    B = F.Batch(max_sims=3, max_grid=24, nbins=3, ray_capacity=1 << 22,
                cell_capacity=2 * 24 ** 3 + 16 ** 3, emitter_capacity=128)
    slot_of, done_at, taken, results = {}, {}, {}, {}
    waiting = list(range(len(plan)))
    step = 0
    while len(results) < len(plan) and step < 200:
        for i in list(waiting):
            if plan[i][0] <= step:
                try:
                    slot_of[i] = B.add(probs[i])
                except F.FlexRTError as e:
                    assert e.status == 3      # full: wait for a retirement
                    continue
                taken[i] = 0
                waiting.remove(i)
        if not taken:
            step += 1
            continue
        B.step()
        step += 1
        for i in list(taken):
            taken[i] += 1
            if taken[i] == plan[i][1]:
                s = slot_of[i]
                results[i] = (B.fields(s), B.budget(s), B.counts(s))
                B.retire(s)
                del taken[i]
    assert len(results) == len(plan)
    for i, p in enumerate(probs):
        _same(*results[i], _alone(p, plan[i][1]))
    B.close()


def test_capacity_errors():
    B = F.Batch(max_sims=2, max_grid=16, nbins=3, ray_capacity=1 << 18, cell_capacity=2 * 16 ** 3,
                emitter_capacity=64)
    p = W.batch_member(1, sizes=(16,), nsteps=2)
    B.add(p)
    B.add(p)
    with pytest.raises(F.FlexRTError) as e:
        B.add(p)
    assert e.value.status == 3
    big = W.batch_member(2, sizes=(24,), nsteps=2)
    with pytest.raises(F.FlexRTError):
        B.add(big)                     # larger than max_grid
    B.close()


def test_served_results_equal_alone():
    # a short Poisson stream served by continuous batching: every request's
    # fields equal the same simulation run alone
    from paper_2409_04521_gb300 import serve
    reqs = W.request_stream(count=8, mean_gap_s=0.01, sizes=(16, 24, 32), steps=(3, 9), seed=11)
    results, stats = serve.serve(reqs, hbm_budget_bytes=2e9, max_sims=4, max_grid=32, emitter_capacity=512,
                                 keep_fields=True)
    assert stats["requests"] == len(reqs)
    for r in results:
        _, prob = reqs[r.rid]
        f, b, c = _alone(prob, prob.nsteps)
        compare_fields(r.fields, f)
        assert r.finished >= r.admitted >= r.arrival - 1e-9
