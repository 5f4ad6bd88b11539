"""Helpers for comparing the CUDA path with the oracle on identical inputs."""
import dataclasses as dc

import numpy as np

import oracle
import paper_2409_04521_gb300 as F

GAMMA_RTOL = 1e-4       # per-cell Gamma_HI, relative
GAMMA_FLOOR = 1e-8      # ... on cells with Gamma >= 1e-8 max Gamma; below, absolute 1e-12 max
X_ATOL = 1e-3           # x_HII absolute
BUDGET_RTOL = 1e-6      # photon conservation of each implementation
BUDGET_XTOL = 1e-4      # GPU budget terms against the oracle's, relative to emitted
RAY_RTOL = 2e-4         # photons carried by the same ray


def ray_table(r):
    key = np.stack([r["emitter"].astype(np.int64), r["birth"].astype(np.int64),
                    r["level"].astype(np.int64), r["pixel"].astype(np.int64)], axis=1)
    order = np.lexsort(key.T[::-1])
    return key[order], r["dir"][order], r["N"][order]


def compare_rays(go, oo, near_threshold, n0_max):
    gk, gd, gN = ray_table(go)
    ok, od, oN = ray_table(oo)
    if near_threshold == 0:
        assert gk.shape == ok.shape, (gk.shape, ok.shape)
        assert np.array_equal(gk, ok)
        assert np.array_equal(gd, od)
        scale = np.maximum(np.abs(oN), 1e-30)
        big = oN > 1e-9 * n0_max
        assert np.all(np.abs(gN - oN)[big] <= RAY_RTOL * scale[big])
        return 0
    # a termination decided within FP32 noise of the threshold: the ray (and
    # its children) exists on one side only and carries next to nothing
    gs = {tuple(k) for k in gk}
    os_ = {tuple(k) for k in ok}
    diff = gs ^ os_
    assert len(diff) <= 64 * near_threshold, len(diff)
    common = np.array(sorted(gs & os_), np.int64).reshape(-1, 4)
    gi = {tuple(k): i for i, k in enumerate(gk)}
    oi = {tuple(k): i for i, k in enumerate(ok)}
    for k in map(tuple, common):
        assert np.array_equal(gd[gi[k]], od[oi[k]])
    return len(diff)


def compare_fields(gf, of, x_atol=X_ATOL, g_rtol=GAMMA_RTOL, T_rtol=None):
    g, o = gf["gamma_HI"], of["gamma_HI"]
    gmax = max(o.max(), 1e-300)
    big = o >= GAMMA_FLOOR * gmax
    rel = np.abs(g - o)[big] / o[big]
    assert rel.size == 0 or rel.max() <= g_rtol, (rel.max(), int(np.argmax(rel)))
    assert np.all(np.abs(g - o)[~big] <= 1e-12 * gmax + GAMMA_FLOOR * gmax)
    assert np.max(np.abs(gf["x_HII"] - of["x_HII"])) <= x_atol
    if T_rtol is not None:
        assert np.max(np.abs(gf["T"] - of["T"]) / of["T"]) <= T_rtol
    return dict(gamma_rel_max=float(rel.max()) if rel.size else 0.0,
                x_abs_max=float(np.max(np.abs(gf["x_HII"] - of["x_HII"]))),
                T_rel_max=float(np.max(np.abs(gf["T"] - of["T"]) / of["T"])))


def budget_checks(gb, ob):
    for b in (gb, ob):
        assert abs(b[0] - b[1] - b[2] - b[3]) <= BUDGET_RTOL * b[0]
    assert np.all(np.abs(gb - ob) <= BUDGET_XTOL * ob[0])


def run_pair(prob, steps=None, capacity=1 << 22, check_every=1, T_rtol=None, x_atol=X_ATOL):
    """Run the same problem through the GPU and the oracle, comparing after
    every `check_every` steps.  Returns a summary dict."""
    steps = prob.nsteps if steps is None else steps
    g = F.Simulation(prob, ray_capacity=capacity, keep_diagnostics=True)
    o = oracle.OracleSim(prob)
    n0_max = float(np.max(prob.source_ndot)) * prob.dt / (12 * 4 ** prob.options.l_src) if len(prob.source_ndot) else 1.0
    summary = dict(steps=steps, straddles=0, max_diff_rays=0)
    for s in range(steps):
        g.step(prob.dt)
        o.step(prob.dt)
        if (s + 1) % check_every and s + 1 != steps:
            continue
        oc = o.counts()
        gc = g.counts()
        gb, ob = g.budget(), o.budget()
        budget_checks(gb, ob)
        nd = compare_rays(g.rays(), o.rays(), oc["near_threshold"], n0_max)
        summary["max_diff_rays"] = max(summary["max_diff_rays"], nd)
        if oc["near_threshold"] == 0:
            assert gc["rays"] == oc["rays"]
            assert gc["segments_last"] == oc["segments_last"]
            assert gc["segments_total"] == oc["segments_total"]
            assert np.array_equal(g.segment_counts(), o.segment_counts())
        summary["straddles"] = oc["near_threshold"]
        gf, of = g.fields(), o.fields()
        summary.update(compare_fields(gf, of, x_atol=x_atol, T_rtol=T_rtol))
        if s + 1 == steps:
            record_errors(f"{prob.name} {'x'.join(str(v) for v in prob.grid)}", steps, field_errors(gf, of),
                          gamma_iters=int(getattr(prob.options, "gamma_iters", 1)), rays=gc["rays"])
    summary["rays"] = g.counts()["rays"]
    summary["segments_total"] = g.counts()["segments_total"]
    g.close()
    o.close()
    return summary


def field_errors(gf, of):
    """Max and median error of the GPU's fields against the oracle's: Gamma_HI
    relative (cells with Gamma >= 1e-8 of the largest), x_HII absolute, T
    relative, n_HI relative (cells with n_HI >= 1e-8 of the largest)."""
    out = {}
    g, o = gf["gamma_HI"], of["gamma_HI"]
    big = o >= GAMMA_FLOOR * max(o.max(), 1e-300)
    rel = np.abs(g - o)[big] / o[big] if big.any() else np.zeros(1)
    out["gamma_rel"] = (float(rel.max()), float(np.median(rel)))
    ax = np.abs(gf["x_HII"] - of["x_HII"])
    out["x_abs"] = (float(ax.max()), float(np.median(ax)))
    rT = np.abs(gf["T"] - of["T"]) / of["T"]
    out["T_rel"] = (float(rT.max()), float(np.median(rT)))
    n, on = gf["n_HI"], of["n_HI"]
    bn = on >= 1e-8 * max(on.max(), 1e-300)
    rn = np.abs(n - on)[bn] / on[bn] if bn.any() else np.zeros(1)
    out["nHI_rel"] = (float(rn.max()), float(np.median(rn)))
    return out


def record_errors(config, step, errs, **extra):
    """Append one row of the per-field error table to the file named by
    FLEXRT_ERRTABLE (if set)."""
    import json
    import os
    path = os.environ.get("FLEXRT_ERRTABLE")
    if not path:
        return
    row = dict(config=config, step=step, **errs, **extra)
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")
