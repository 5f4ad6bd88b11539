"""Pins of the oracle's split table (Sec. 3.2, Eq. 2) and one-step cell
traversal (Sec. 3.1) against the pixel-area definition and an exact
rational brute force."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle

S = 2 ** 21


def test_split_table_meaning():
    # Eq. 2: at r_split(l) one level-l pixel covers Delta x^2 / N_min of the
    # sphere of radius r_split: 4 pi r^2 / (12 4^l) = 1 / N_min (cells^2).
    for nmin in (2.0, 3.0, 5.5, 16.0):
        K = oracle.split_table(nmin)
        for l in range(13):
            area = lambda r: 4 * math.pi * r * r / (12 * 4 ** l)
            assert area(K[l]) >= 1 / nmin * (1 - 1e-12) or K[l] == 1
            if K[l] > 1:
                assert area(K[l] - 1) < 1 / nmin
    assert list(oracle.split_table(3.0)[:10]) == [1, 2, 3, 5, 10, 19, 37, 73, 145, 289]


def brute_force_traverse(p0, d, n):
    """Exact segment list: all face-crossing parameters t in (0,1) as
    Fractions, sorted; each piece takes the cell of its midpoint."""
    p0 = [int(x) for x in p0]
    d = [int(x) for x in d]
    ts = {Fraction(0), Fraction(1)}
    for a in range(3):
        if d[a] == 0:
            continue
        lo, hi = sorted((p0[a], p0[a] + d[a]))
        k0 = -(-lo // S)
        for k in range(k0, hi // S + 1):
            t = Fraction(k * S - p0[a], d[a])
            if 0 < t < 1:
                ts.add(t)
    ts = sorted(ts)
    cells, ds = [], []
    for t0, t1 in zip(ts[:-1], ts[1:]):
        tm = (t0 + t1) / 2
        c = [math.floor((p0[a] + tm * d[a]) / S) for a in range(3)]
        if any(c[a] < 0 or c[a] >= n[a] for a in range(3)):
            return cells, ds, True
        cells.append(c)
        ds.append(t1 - t0)
    # a ray ending exactly on the box face is still inside this step
    return cells, ds, False


def _check(p0, d, n):
    cells, ds, esc = oracle.traverse(p0, d, n)
    bc, bds, besc = brute_force_traverse(p0, d, n)
    # a ray starting outside the box (only possible on the far side of a face) escapes at once
    assert esc == besc, (p0, d)
    assert [list(c) for c in cells] == bc, (p0, d)
    for a, b in zip(ds, bds):
        assert a == pytest.approx(float(b), rel=2e-16, abs=1e-300)
    if not esc:
        assert sum(ds) == pytest.approx(1.0, abs=1e-15)


def test_traverse_random():
    rng = np.random.default_rng(11)
    n = [4, 5, 6]
    for _ in range(3000):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        d = np.rint(v * S).astype(np.int64)
        p0 = rng.integers(0, np.array(n) * S)
        _check(p0, d, n)


def test_traverse_faces_edges_and_ties():
    n = [4, 4, 4]
    rng = np.random.default_rng(3)
    cases = []
    # on faces / edges / corners, axis-aligned and diagonal directions
    for base in ([S, S, S], [2 * S, S + 5, S + S // 2], [S + 7, 2 * S, 3 * S - 1], [0, 0, 0], [4 * S - 1, S, S]):
        for d in ([S, 0, 0], [-S, 0, 0], [0, -S, 0], [S // 2, S // 2, 0], [-S // 2, S // 2, S // 3],
                  [1482910, 1482910, 0], [1210780, -1210780, 1210780], [-1210780, -1210780, -1210780],
                  [0, 0, 0], [S, S, S]):
            cases.append((base, d))
    # exact ties: start at a cell centre, equal per-axis distances to faces
    for _ in range(300):
        c = rng.integers(0, 4, 3) * S + S // 2
        m = int(rng.integers(1, S // 2))
        sg = rng.choice([-1, 1], 3)
        d = [int(sg[0] * m * 2), int(sg[1] * m * 2), int(sg[2] * rng.integers(0, 2 * m + 1))]
        cases.append((list(c), d))
    for p0, d in cases:
        _check(np.array(p0, np.int64), np.array(d, np.int64), n)


def test_traverse_outside_start_escapes():
    cells, ds, esc = oracle.traverse([4 * S, S, S], [S, 0, 0], [4, 4, 4])
    assert esc and len(cells) == 0
    cells, ds, esc = oracle.traverse([4 * S, S, S], [-S, 0, 0], [4, 4, 4])
    assert not esc and [list(c) for c in cells] == [[3, 1, 1]]


def test_at_most_four_segments():
    rng = np.random.default_rng(5)
    for _ in range(2000):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        d = np.rint(v * S).astype(np.int64)
        p0 = rng.integers(S, 3 * S, 3)
        cells, ds, esc = oracle.traverse(p0, d, [8, 8, 8])
        assert 1 <= len(cells) <= 4
