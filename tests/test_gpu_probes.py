"""Bit-exact parity of the device functions the step kernels use (HEALPix
vectors, sphere rotations, fixed-point directions, one-step traversal)
against the oracle, through the C-ABI probes."""
import numpy as np
import pytest

import oracle
import paper_2409_04521_gb300 as F

pytestmark = pytest.mark.gpu
S = 2 ** 21


def oracle_vq(level, p):
    return np.rint(oracle.pix2vec(level, p) * 2 ** 24).astype(np.int32)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5])
def test_pixvec_all_pixels(level):
    n = 12 * 4 ** level
    g = F.probe_pixvec(level, 0, n)
    o = np.array([oracle_vq(level, p) for p in range(n)])
    assert np.array_equal(g, o)


@pytest.mark.parametrize("level", [7, 9, 12])
def test_pixvec_sampled_deep_levels(level):
    n = 12 * 4 ** level
    rng = np.random.default_rng(level)
    for p0 in list(rng.integers(0, n - 64, 24)) + [0, n - 64]:
        g = F.probe_pixvec(level, int(p0), 64)
        o = np.array([oracle_vq(level, int(p0) + k) for k in range(64)])
        assert np.array_equal(g, o)


def test_rotations():
    for seed in (1, 2, 12345, 2 ** 63 + 7):
        for e in (0, 1, 5, 19999):
            for s in (0, 1, 99, 199):
                _, Rq = oracle.rotation(seed, e, s)
                assert np.array_equal(F.probe_rotation(seed, e, s), Rq)
    _, Rq = oracle.rotation(3, 0, 0, rotate=False)
    assert np.array_equal(F.probe_rotation(3, 0, 0, rotate=False), Rq)


@pytest.mark.parametrize("level", [0, 2, 5, 9])
def test_directions(level):
    n = 12 * 4 ** level
    rng = np.random.default_rng(100 + level)
    for e in range(3):
        _, Rq = oracle.rotation(9, e, 4)
        p0 = int(rng.integers(0, max(1, n - 256)))
        m = min(256, n)
        g = F.probe_direction(level, p0, m, Rq)
        o = np.array([oracle.direction(level, p0 + k, Rq) for k in range(m)])
        assert np.array_equal(g, o)


def _traverse_cases():
    rng = np.random.default_rng(8)
    p0, d = [], []
    for _ in range(20000):
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        d.append(np.rint(v * S).astype(np.int64))
        p0.append(rng.integers(-S, 7 * S, 3))
    # faces, edges, corners, axis-aligned and exactly tied diagonals
    for base in ([S, S, S], [2 * S, S + 5, S + S // 2], [0, 0, 0], [6 * S, 3 * S, 2 * S], [S + 7, 2 * S, 3 * S - 1]):
        for dd in ([S, 0, 0], [-S, 0, 0], [0, -S, 0], [0, 0, S], [S // 2, S // 2, 0], [-1210780, 1210780, -1210780],
                   [1482910, 1482910, 0], [0, 0, 0], [S, S, S], [-S, -S, -S]):
            p0.append(base)
            d.append(dd)
    for _ in range(2000):
        c = rng.integers(0, 6, 3) * S + S // 2
        m = int(rng.integers(1, S // 2))
        sg = rng.choice([-1, 1], 3)
        p0.append(c)
        d.append([sg[0] * 2 * m, sg[1] * 2 * m, sg[2] * int(rng.integers(0, 2 * m + 1))])
    return np.array(p0, np.int64), np.array(d, np.int64)


def test_traversal_cells_bit_exact():
    grid = (6, 5, 7)
    p0, d = _traverse_cases()
    d = np.clip(d, -S, S)
    cells, ds, nseg, esc = F.probe_traverse(p0, d, grid)
    for i in range(len(p0)):
        oc, ods, oesc = oracle.traverse(p0[i], d[i], grid)
        k = len(oc)
        assert nseg[i] == k, i
        assert bool(esc[i]) == oesc, i
        assert np.array_equal(cells[i, :k], oc), i
        # lengths: the exact fractions to a few single-precision ulp
        assert np.allclose(ds[i, :k], ods, rtol=6e-7, atol=0), (i, ds[i, :k], ods)


def test_rate_fits_match_oracle():
    # the chemistry kernel's single-precision fits (evaluated through log2 /
    # exp2 of sums) against the oracle's double-precision fits, 1 K to 1e9 K.
    # A rate of the form exp(-c lambda) (lambda = 2 T_HI / T) inherits
    # lambda's relative error times c lambda: the tolerance grows with lambda.
    T = np.geomspace(1.0, 1.0e9, 4001).astype(np.float32)
    g = F.probe_rates(T).astype(np.float64)
    Td = T.astype(np.float64)
    lam = 2 * 157807.0 / Td
    o = np.stack([[oracle.alpha_B(t), oracle.alpha_A(t), oracle.coll_ion(t), oracle.cooling(t, 1.0, 1.0, 1.0, -1.0)]
                  for t in Td])
    for k, name in enumerate(("alpha_B", "alpha_A", "C_HI", "cooling")):
        big = o[:, k] > 1e-35
        rel = np.abs(g[big, k] / o[big, k] - 1.0)
        tol = 3e-5 + 3e-6 * lam[big]
        assert np.all(rel <= tol), (name, float(rel.max()), float(Td[big][np.argmax(rel / tol)]))
        assert np.all(np.abs(g[~big, k]) <= 1e-34), name
    with pytest.raises(F.FlexRTError):
        F.probe_rates(np.array([0.5], np.float32))
