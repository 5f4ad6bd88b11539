"""Autotuner for the fused march kernel's launch configuration.

For a given workload it runs the first RT steps of the simulation once per
candidate (deposit aggregation scheme, register budget, persistent blocks
per SM), then on the fastest of those once per launch shape (threads per
block, output run length of a warp in queue slots), times the march kernel
with CUDA events on the simulation's stream, and keeps the fastest.  Results are cached per workload signature
and device name in ``_build/tune_cache.json``.
"""
from __future__ import annotations

import hashlib
import json
import os
import threading

from . import build as _build
from . import flexrt as _f

CACHE = os.path.join(_build.BUILD, "tune_cache.json")
_lock = threading.Lock()

# Stage 1: (aggregation, register budget in resident blocks per SM, blocks
# per SM; 0 = occupancy limit) with the default launch shape.
BASES = [(a, m, 0) for a in (0, 1, 2) for m in (2, 3, 4)] + [(1, 3, 2), (2, 3, 2), (0, 3, 2)]
# Stage 2, on the best base: (threads per block, output run length in queue
# slots); (256, 512) is the default shape.
SHAPES = [(256, 512), (128, 512), (256, 128), (128, 128), (256, 2048), (128, 2048)]
CANDIDATES = [b + (256, 512) for b in BASES]


def candidates():
    """Every launch the two-stage search can return."""
    return [b + sh for b in BASES for sh in SHAPES]


def signature(prob, nsteps: int) -> str:
    h = hashlib.sha1()
    o = prob.options
    merge = (bool(getattr(o, "merge", False)), getattr(o, "l_merge", 0), getattr(o, "n_ex", 0.0))
    iters = int(getattr(o, "gamma_iters", 1))
    h.update(repr((tuple(prob.grid), prob.spectrum.nbins, len(prob.source_ndot), nsteps,
                   o.l_src, o.n_ray_min, prob.mfp.mode) + (merge if merge[0] else ())
                  + ((iters,) if iters > 1 else ())).encode())
    return h.hexdigest()[:16]


def _device_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "cuda"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, CACHE)


def time_variant(sim, prob, nsteps, variant):
    """March-kernel milliseconds over the first `nsteps` RT steps."""
    sim.set_launch(*variant)
    sim.reset()
    sim.profile(True)
    for _ in range(nsteps):
        sim.step(prob.dt)
    sim.sync()
    ms, launches, rays = sim.kernel_times()
    sim.profile(False)
    return float(ms["march"]), int(rays)


def tune(sim, prob, nsteps: int = None, candidates=None, use_cache: bool = True, verbose: bool = False):
    """Pick and apply the fastest march launch configuration for `prob` on
    the simulation `sim` (leaves `sim` reset).  Returns (variant, table)."""
    nsteps = prob.nsteps if nsteps is None else nsteps
    key = f"{_device_name()}|{signature(prob, nsteps)}"
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache and len(cache[key]["best"]) == 5:
        v = tuple(cache[key]["best"])
        sim.set_launch(*v)
        sim.reset()
        return v, cache[key]["table"]
    table = []

    def run(vs):
        for v in vs:
            try:
                ms, rays = time_variant(sim, prob, nsteps, v)
            except _f.FlexRTError:
                continue
            table.append([list(v), ms, rays])
            if verbose:
                print("variant", v, "march ms %.3f" % ms, flush=True)

    run(candidates or CANDIDATES)
    if not table:
        raise RuntimeError("no march variant could run")
    if candidates is None:
        b = tuple(min(table, key=lambda r: r[1])[0])[:3]
        run([b + sh for sh in SHAPES if sh != (256, 512)])
    best = tuple(min(table, key=lambda r: r[1])[0])
    sim.set_launch(*best)
    sim.reset()
    with _lock:
        cache = _load()
        cache[key] = {"best": list(best), "table": table}
        _store(cache)
    return best, table
