"""Checkpoint and restart (flexrt_save_state / flexrt_load_state) and the cap
on a context's device allocations (flexrt_options.device_bytes_max).

A run's deposits are single-precision vector reductions whose order varies
from run to run, so two uninterrupted runs agree to rounding, not bit for
bit.  What a checkpoint must give: the state round-trips bit for bit; the
first step after a restore marches exactly the rays the saved context would
march (same ids, directions and photons, bit for bit); and a restored run
continues as an uninterrupted one, within the tolerance two uninterrupted
runs agree to.
"""
import dataclasses as dc

import numpy as np
import pytest

import paper_2409_04521_gb300 as F
import workloads as W
from parity_util import compare_fields, ray_table

pytestmark = pytest.mark.gpu


def _prob(**kw):
    p = W.cosmo16(n=24, nsteps=12, nsrc=8, seed=3)
    return dc.replace(p, options=dc.replace(p.options, **kw)) if kw else p


def _same_rays(a, b, exact=True):
    ka, da, Na = ray_table(a)
    kb, db, Nb = ray_table(b)
    assert np.array_equal(ka, kb) and np.array_equal(da, db)
    if exact:
        assert np.array_equal(Na, Nb)
    else:
        assert np.allclose(Na, Nb, rtol=1e-5, atol=1e-9 * max(Nb.max(), 1e-300))


@pytest.mark.parametrize("kw", [{}, dict(merge=True, n_ex=1.0, l_merge=0), dict(gamma_iters=3)])
def test_checkpoint_round_trip_and_resume(kw):
    prob = _prob(**kw)
    half = prob.nsteps // 2
    a = F.Simulation(prob, ray_capacity=1 << 21)
    b = F.Simulation(prob, ray_capacity=1 << 21)
    for _ in range(half):
        a.step(prob.dt)
        b.step(prob.dt)
    blob = b.save_state()
    c = F.Simulation(prob, ray_capacity=1 << 21)
    c.load_state(blob)
    assert np.array_equal(c.save_state(), blob)              # bit-exact round trip
    assert c.counts()["step"] == b.counts()["step"] == half
    assert np.array_equal(c.budget(), b.budget())
    # the next step marches the same rays through the same opacities
    b.step(prob.dt)
    c.step(prob.dt)
    if not kw:
        # one pass: the march reads only the restored state
        _same_rays(b.rays(), c.rays(), exact=True)
    elif not kw.get("merge"):
        # trial passes feed Gamma (single-precision reductions) back into the
        # opacity: equal to rounding
        _same_rays(b.rays(), c.rays(), exact=False)
    compare_fields(c.fields(), b.fields(), x_atol=1e-6, g_rtol=1e-5, T_rtol=1e-5)
    # and the resumed run follows the uninterrupted one
    a.step(prob.dt)
    for _ in range(half + 1, prob.nsteps):
        a.step(prob.dt)
        c.step(prob.dt)
    ca, cc = a.counts(), c.counts()
    assert cc["step"] == ca["step"] == prob.nsteps
    if not kw.get("merge"):
        assert cc["rays"] == ca["rays"] and cc["segments_total"] == ca["segments_total"]
        _same_rays(a.rays(), c.rays(), exact=False)
        compare_fields(c.fields(), a.fields(), x_atol=1e-4, g_rtol=1e-4, T_rtol=1e-3)
        assert np.allclose(c.budget(), a.budget(), rtol=1e-5)
    else:
        # merging runs, resumed or not, drift apart from rounding (rays
        # within rounding of T_ref or a pixel edge change groups): Sec. 7.1's
        # criteria
        fc, fa = c.fields(), a.fields()
        assert abs(cc["rays"] - ca["rays"]) <= 0.02 * ca["rays"] + 16
        assert abs(fc["x_HII"].mean() - fa["x_HII"].mean()) <= 0.01 * fa["x_HII"].mean()
        assert abs(fc["gamma_HI"].mean() - fa["gamma_HI"].mean()) <= 0.02 * fa["gamma_HI"].mean()
        assert np.all(np.abs(c.budget() - a.budget()) <= 0.01 * a.budget()[0])
    for s in (a, b, c):
        s.close()


def test_checkpoint_rejects_another_simulation():
    prob = _prob()
    other = W.cosmo16(n=16, nsteps=4, nsrc=4, seed=5)
    a = F.Simulation(prob, ray_capacity=1 << 20)
    o = F.Simulation(other, ray_capacity=1 << 20)
    o.step(other.dt)
    for _ in range(5):
        a.step(prob.dt)
    assert a.counts()["rays"] > 4096
    before = a.save_state()
    with pytest.raises(F.FlexRTError) as e:
        a.load_state(o.save_state())
    assert e.value.status == 1
    with pytest.raises(F.FlexRTError):
        a.load_state(before[:-4])
    bad = before.copy()
    bad[0] ^= 0xFF
    with pytest.raises(F.FlexRTError):
        a.load_state(bad)
    assert np.array_equal(a.save_state(), before)             # unchanged
    a.step(prob.dt)
    assert a.counts()["step"] == 6
    # a checkpoint with more live rays than the queue holds
    small = F.Simulation(prob, ray_capacity=1024)
    with pytest.raises(F.FlexRTError) as e:
        small.load_state(before)
    assert e.value.status == 3
    for s in (a, o, small):
        s.close()


def test_device_memory_cap():
    import torch
    prob = _prob()
    ok = F.Simulation(prob, ray_capacity=1 << 20)
    need = ok.device_bytes()
    assert need > 0
    ok.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for cap in (1, 1 << 16, need // 4, need - 1):
        with pytest.raises(F.FlexRTError) as e:
            F.Simulation(prob, ray_capacity=1 << 20, device_bytes_max=cap)
        assert e.value.status == 2                              # FLEXRT_E_OOM
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0            # nothing left allocated
    s = F.Simulation(prob, ray_capacity=1 << 20, device_bytes_max=need)
    assert s.device_bytes() <= need
    s.step(prob.dt)
    # growing the emitter tables beyond the cap fails and keeps the sources
    cells = np.argwhere(np.ones(prob.grid, bool))[:4000].astype(np.int32)
    with pytest.raises(F.FlexRTError) as e:
        s.add_sources(cells, np.full(len(cells), 1e50))
    assert e.value.status == 2
    s.step(prob.dt)
    assert s.counts()["step"] == 2
    s.close()
