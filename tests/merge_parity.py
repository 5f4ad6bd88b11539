"""Step-local parity of ray merging (Sec. 3.3, Eq. 4): the GPU's merge of a
set of rays against the oracle's merge of the very same rays.

The oracle ranks rays by their double-precision photon content, decides each
ray's merge pixel by double-precision ang2pix and forms photon-weighted means
in double precision, rounded once.  The GPU ranks by the single-precision sum
of its single-precision bins, decides pixels in single precision and forms
the means as exact quotients of 64-bit integer sums of weights truncated to
2^-28 of the power of two above the group's brightest content.  So:

* a ray whose content lies within single-precision rounding of T_ref (the
  K-th largest) may be exempt on one side only, and a ray within rounding of
  a pixel edge may fall in a neighbouring pixel on the GPU -- both are
  counted, bounded, and the groups they touch are left out of the
  element-by-element comparison (like termination straddles);
* every other group must be the same set of rays on both sides, and its
  merged ray must have the same id and direction, photons and threshold
  within single-precision summation, position within 2 + n/64 units of
  2^-21 cell (n members: truncated weights, n/64; single- vs
  double-precision contents, 1/2; rounding, 1), and the same distance and
  level unless the exact mean sits within 1e-3 of a half-integer;
* every ray outside such groups (exempt, out of the box, alone in its group)
  is unchanged on both sides.
"""
import numpy as np

import oracle
import paper_2409_04521_gb300 as F

S = 2 ** 21


def emitter_cells(prob):
    cells, first = [], {}
    for ijk in map(tuple, prob.source_cells):
        if ijk not in first:
            first[ijk] = len(cells)
            cells.append(ijk)
    return np.array(cells, np.int64).reshape(-1, 3)


def end_points(r, ecells, step):
    """End point (2^-21 cell) of each ray after the march of `step`."""
    d = r["dir"].astype(np.int64)
    merged = np.asarray(r["merged"], bool)
    out = np.zeros((len(d), 3), np.int64)
    if (~merged).any():
        e = np.asarray(r["emitter"])[~merged].astype(np.int64)
        c = (2 * ecells[e] + 1) * (S // 2)
        out[~merged] = c + (step - r["birth"][~merged, None].astype(np.int64) + 1) * d[~merged]
    if merged.any():
        out[merged] = r["P"][merged] + (step - r["birth"][merged, None].astype(np.int64)) * d[merged]
    return out


def _keys(r):
    return [(int(r["emitter"][i]), int(r["birth"][i]), int(r["level"][i]), int(r["pixel"][i]),
             bool(r["vertex"][i])) for i in range(len(r["level"]))]


def compare_merge_step(pre, gpu, ora, prob, step, K, l_merge, max_ambiguous=0.01):
    """Compare the GPU's (gpu) and the oracle's (ora) merge of the rays `pre`
    as they stand after the march of `step`.  Returns a summary dict."""
    grid = np.array(prob.grid, np.int64)
    ndir = 12 * 4 ** l_merge
    seed = prob.options.seed
    n = len(pre["level"])
    T = pre["N"].sum(1)
    if K >= n:
        assert sorted(_keys(gpu)) == sorted(_keys(pre)) == sorted(_keys(ora))
        return dict(groups=0, clean=0, merged=0, ambiguous=0, ambiguous_rank=0, ambiguous_pixel=0, dirty=0,
                    dP_max=0, rays=n)
    Tref = np.sort(T)[::-1][K - 1] if K > 0 else np.inf
    amb_rank = np.zeros(n, bool) if K == 0 else np.abs(T - Tref) <= 1e-6 * Tref
    cand = (T < Tref) | amb_rank
    ends = end_points(pre, emitter_cells(prob), step)
    cell = ends // S
    inside = np.all((cell >= 0) & (cell < grid), axis=1)
    local = (cell[:, 2] * grid[1] + cell[:, 1]) * grid[0] + cell[:, 0]
    idx = np.nonzero(cand & inside)[0]
    rots = {}
    for loc in np.unique(local[idx]):
        rots[int(loc)] = oracle.merge_rotation(seed, int(loc), step)
    Rq = np.array([rots[int(local[i])] for i in idx], np.int32).reshape(-1, 3, 3)
    pix_o = np.array([oracle.merge_pixel(l_merge, Rq[k], pre["dir"][i]) for k, i in enumerate(idx)], np.int64)
    pix_g = F.probe_merge_pixel(l_merge, pre["dir"][idx], Rq).astype(np.int64) if len(idx) else pix_o
    amb_pix = pix_o != pix_g
    for k in np.nonzero(amb_pix)[0]:
        i = idx[k]
        near = {oracle.merge_pixel(l_merge, Rq[k], pre["dir"][i] + s * e)
                for e in np.eye(3, dtype=np.int32) for s in (-4, 4)}
        assert pix_g[k] in near, ("GPU merge pixel off a pixel edge", i, pix_o[k], pix_g[k])
    key_o = np.full(n, -1, np.int64)
    key_g = np.full(n, -1, np.int64)
    key_o[idx] = local[idx] * ndir + pix_o
    key_g[idx] = local[idx] * ndir + pix_g
    ambiguous = np.zeros(n, bool)
    ambiguous[idx[amb_pix]] = True
    ambiguous |= amb_rank
    dirty = set(key_o[ambiguous & (key_o >= 0)]) | set(key_g[ambiguous & (key_g >= 0)])
    certain = (T < Tref) & ~amb_rank & inside
    groups = {}
    for i in np.nonzero(certain)[0]:
        groups.setdefault(int(key_o[i]), []).append(int(i))
    clean = {k: g for k, g in groups.items() if k not in dirty}
    # pixel edges: a bounded fraction; contents within rounding of T_ref: as
    # many as there are (rays crossing fully ionised gas keep nearly equal
    # contents, and many can sit within 1e-6 of T_ref), each group they touch
    # left out
    assert amb_pix.sum() <= max_ambiguous * n + 4, (int(amb_pix.sum()), n)

    gk, ok = _keys(gpu), _keys(ora)
    gi = {k: i for i, k in enumerate(gk)}
    oi = {k: i for i, k in enumerate(ok)}
    # rays that stay as they were: exempt for sure, out of the box, alone in
    # a clean group
    stay = (~cand & ~amb_rank) | (cand & ~inside & ~amb_rank)
    for k, g in clean.items():
        if len(g) == 1:
            stay[g[0]] = True
    pk = _keys(pre)
    for i in np.nonzero(stay)[0]:
        a, b = gi[pk[i]], oi[pk[i]]
        assert np.array_equal(ora["N"][b], pre["N"][i]) and np.array_equal(gpu["N"][a], pre["N"][i])
        assert np.array_equal(gpu["dir"][a], pre["dir"][i]) and np.array_equal(ora["dir"][b], pre["dir"][i])
    # merged rays of clean groups: a ray made by this step's merge carries
    # emitter 2^31 + its cell, birth = this step and its merge pixel (it
    # splits only in a later march), so (cell, pixel) names it on both sides
    def made_here(r):
        return {(int(r["emitter"][i]) - (1 << 31), int(r["pixel"][i])): i
                for i in np.nonzero(np.asarray(r["merged"]) & (np.asarray(r["birth"]) == step))[0]}
    mg, mo = made_here(gpu), made_here(ora)
    nmerged, dPmax = 0, 0
    for key, g in clean.items():
        if len(g) < 2:
            continue
        a, b = mg[divmod(key, ndir)], mo[divmod(key, ndir)]
        w = T[g]
        m = len(g)
        assert np.array_equal(gpu["dir"][a], ora["dir"][b])
        assert np.allclose(gpu["N"][a], ora["N"][b], rtol=1e-5, atol=0)
        assert np.isclose(gpu["thr"][a], ora["thr"][b], rtol=1e-5)
        dP = np.abs(gpu["P"][a] - ora["P"][b]).max()
        assert dP <= 2 + m / 64.0, (key, m, gpu["P"][a], ora["P"][b])
        dPmax = max(dPmax, int(dP))
        dist = np.where(pre["merged"][g], pre["A"][g] + step - pre["birth"][g], step - pre["birth"][g] + 1)
        for got_g, got_o, x in ((gpu["A"][a], ora["A"][b], dist),
                                (gpu["level"][a], ora["level"][b], pre["level"][g])):
            mean = float((w * x).sum() / w.sum())
            if abs(mean - np.floor(mean) - 0.5) > 1e-3:
                assert got_g == got_o, (key, got_g, got_o, mean)
            else:
                assert abs(int(got_g) - int(got_o)) <= 1
        assert bool(gpu["vertex"][a]) == (gpu["level"][a] > l_merge)
        nmerged += 1
    # everything else: the ray counts differ by at most the dirty groups
    assert abs(len(gk) - len(ok)) <= len(dirty) + int(ambiguous.sum())
    return dict(groups=len(groups), clean=len(clean), merged=nmerged, ambiguous=int(ambiguous.sum()),
                ambiguous_rank=int(amb_rank.sum()), ambiguous_pixel=int(amb_pix.sum()), dirty=len(dirty),
                dP_max=dPmax, rays=n)
