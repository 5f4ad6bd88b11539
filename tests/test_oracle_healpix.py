"""Pins of the oracle's HEALPix NESTED pix2vec, rotation sampler and
fixed-point directions (Sec. 3.1, Eq. 1; Sec. 3.2, Eq. 3), checked against
closed forms, an independent ang2pix, and invariants of the pixelisation."""
import math

import numpy as np
import pytest

import oracle
from healpix_ref import ang2pix_nest


def _phi(v):
    p = math.atan2(v[1], v[0])
    return p + 2 * math.pi if p < 0 else p


def test_level0_closed_form():
    # faces 0-3: z = 2/3, phi = pi/4 + k pi/2; 4-7: z = 0, phi = k pi/2;
    # 8-11: z = -2/3, phi = pi/4 + k pi/2
    for f in range(12):
        v = oracle.pix2vec(0, f)
        k = f % 4
        if f < 4:
            z, phi = 2 / 3, math.pi / 4 + k * math.pi / 2
        elif f < 8:
            z, phi = 0.0, k * math.pi / 2
        else:
            z, phi = -2 / 3, math.pi / 4 + k * math.pi / 2
        assert v[2] == pytest.approx(z, abs=1e-16)
        assert _phi(v) == pytest.approx(phi, abs=1e-15)


def test_level1_closed_form():
    v = oracle.pix2vec(1, 0)
    assert v[2] == pytest.approx(1 / 3, abs=1e-16) and _phi(v) == pytest.approx(math.pi / 4, abs=1e-15)
    v = oracle.pix2vec(1, 3)
    assert v[2] == pytest.approx(11 / 12, abs=1e-16) and _phi(v) == pytest.approx(math.pi / 4, abs=1e-15)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_unit_norm_and_zero_sum(level):
    V = np.array([oracle.pix2vec(level, p) for p in range(12 * 4 ** level)])
    assert np.max(np.abs(np.linalg.norm(V, axis=1) - 1.0)) < 4e-16
    assert np.max(np.abs(V.sum(axis=0))) < 1e-12


@pytest.mark.parametrize("level", [1, 2, 3])
def test_ring_latitudes(level):
    ns = 2 ** level
    rings = set()
    for i in range(1, ns):
        rings.add(round(1 - i * i / (3 * ns * ns), 13))
        rings.add(round(-(1 - i * i / (3 * ns * ns)), 13))
    for i in range(ns, 3 * ns + 1):
        rings.add(round(4 / 3 - 2 * i / (3 * ns), 13))
    zs = {round(oracle.pix2vec(level, p)[2], 13) for p in range(12 * 4 ** level)}
    assert zs == rings


def test_phi_matches_libm():
    # the oracle's own series sin/cos must agree with libm to ~1 ulp
    for level in (2, 5, 8):
        ns = 2 ** level
        for p in range(0, 12 * ns * ns, max(1, (12 * ns * ns) // 997)):
            v = oracle.pix2vec(level, p)
            st = math.sqrt(1 - v[2] ** 2)
            phi = _phi(v)
            assert v[0] == pytest.approx(st * math.cos(phi), abs=3e-15)
            assert v[1] == pytest.approx(st * math.sin(phi), abs=3e-15)


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 5, 6])
def test_ang2pix_round_trip(level):
    n = 12 * 4 ** level
    step = 1 if n < 20000 else 7
    for p in range(0, n, step):
        assert ang2pix_nest(level, oracle.pix2vec(level, p)) == p


@pytest.mark.parametrize("level", [0, 1, 3, 5])
def test_children_nest_in_parent(level):
    # Eq. 3: children (l+1, 4p+i) lie inside parent pixel (l, p)
    n = 12 * 4 ** level
    for p in range(0, n, max(1, n // 300)):
        for i in range(4):
            assert ang2pix_nest(level, oracle.pix2vec(level + 1, 4 * p + i)) == p


def test_equal_area_monte_carlo():
    # HEALPix pixels have equal area, so uniform directions fill them equally
    rng = np.random.default_rng(7)
    level = 2
    npix = 12 * 4 ** level
    N = 200_000
    v = rng.standard_normal((N, 3))
    counts = np.zeros(npix)
    for row in v:
        counts[ang2pix_nest(level, row)] += 1
    mean = N / npix
    assert np.max(np.abs(counts - mean)) < 5 * math.sqrt(mean)


def test_splitmix64_known_answer():
    # SplitMix64 (Steele, Lea & Flood 2014) from state 0: published first output
    assert oracle.splitmix_draw(0, 0) == 0xE220A8397B1DCDAF
    # the stream advances by the golden gamma: draw i of key k == draw 0 of k + i*gamma
    g = 0x9E3779B97F4A7C15
    for i in range(1, 5):
        assert oracle.splitmix_draw(12345, i) == oracle.splitmix_draw((12345 + i * g) % 2 ** 64, 0)


def test_rotation_is_proper_orthogonal():
    for e in range(5):
        for s in range(5):
            R, Rq = oracle.rotation(42, e, s)
            assert np.max(np.abs(R @ R.T - np.eye(3))) < 1e-14
            assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
            assert np.array_equal(Rq, np.rint(R * 2 ** 24).astype(np.int32))
    R, Rq = oracle.rotation(42, 0, 0, rotate=False)
    assert np.array_equal(R, np.eye(3)) and np.array_equal(Rq, np.eye(3, dtype=np.int32) * 2 ** 24)


def test_rotation_uniform_on_sphere():
    # Marsaglia's quaternion gives Haar rotations: R e_z is uniform on S^2
    Z = np.array([oracle.rotation(9, e, s)[0][:, 2] for e in range(60) for s in range(60)])
    n = len(Z)
    assert np.all(np.abs(Z.mean(axis=0)) < 4 / math.sqrt(3 * n))
    assert np.all(np.abs((Z ** 2).mean(axis=0) - 1 / 3) < 4 * math.sqrt(4 / 45 / n))
    # distinct keys give distinct rotations
    keys = {oracle.rotation_key(9, e, s) for e in range(60) for s in range(60)}
    assert len(keys) == n


def test_fixed_point_direction():
    S = 2 ** 21
    for e in range(3):
        R, Rq = oracle.rotation(5, e, 1)
        for level in (0, 3, 6):
            for p in range(0, 12 * 4 ** level, max(1, 4 ** level)):
                d = oracle.direction(level, p, Rq).astype(np.float64)
                v = R @ oracle.pix2vec(level, p)
                assert np.all(np.abs(np.abs(d) <= S))
                assert np.max(np.abs(d - v * S)) <= 1.0
                assert abs(np.linalg.norm(d) / S - 1) < 4e-7
