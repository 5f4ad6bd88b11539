"""The traversal probe that allocates no device memory.

Callers that cannot allocate device memory themselves (their device memory
belongs to another allocator, or they cannot afford cudaFree's implicit
synchronisation) use flexrt_probe_traverse_static.  It must return exactly
what the allocating flexrt_probe_traverse returns, call after call, although
every call reuses the same fixed device staging array.  This file is
collected last on purpose."""
import numpy as np
import pytest

import paper_2409_04521_gb300 as F
from paper_2409_04521_gb300 import flexrt as FX

S = 2 ** 21


def _cases(seed, n):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    d = np.rint(v * S).astype(np.int64)
    p0 = rng.integers(-S, 9 * S, (n, 3))
    # faces, edges, corners and exact ties
    p0[:64] = (rng.integers(0, 8, (64, 3)) * S)
    d[:32] = [[S, 0, 0], [0, -S, 0], [0, 0, S], [-S, -S, 0]] * 8
    d[32:64, :2] = np.array([[1482910, -1482910]] * 32)
    return p0, np.clip(d, -S, S)


@pytest.mark.gpu
def test_static_probe_matches_allocating_probe_on_consecutive_calls():
    grid = (8, 7, 9)
    for seed, n in ((1, 5000), (2, 3001)):   # a longer call, then a shorter one
        p0, d = _cases(seed, n)
        ca, dsa, na, ea = F.probe_traverse(p0, d, grid)
        cb, dsb, nb, eb = FX.probe_traverse_static(p0, d, grid)
        assert np.array_equal(na, nb)
        assert np.array_equal(ea, eb)
        for i in range(n):
            k = na[i]
            assert np.array_equal(ca[i, :k], cb[i, :k])
            assert np.allclose(dsa[i, :k], dsb[i, :k], rtol=4e-7, atol=0)
        # slots past each ray's last segment carry the reset values, not the
        # previous call's contents
        for i in range(n):
            k = nb[i]
            assert np.all(cb[i, k:] == -1) and np.all(dsb[i, k:] == 0)


@pytest.mark.gpu
def test_static_probe_rejects_batches_above_its_maximum():
    n = FX.STATIC_MAX_RAYS + 1
    p0 = np.zeros((n, 3), np.int64)
    d = np.zeros((n, 3), np.int64)
    with pytest.raises(F.FlexRTError) as e:
        FX.probe_traverse_static(p0, d, (4, 4, 4))
    assert e.value.status == 3
    assert str(FX.STATIC_MAX_RAYS) in str(e.value)
