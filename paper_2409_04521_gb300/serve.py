"""Serving many simulations on one GPU by continuous batching.

Requests (a problem description with its own grid, sources, step length
and number of steps) arrive over time.  The server keeps one native batch
(flexrt_batch_*): between RT steps it admits arrived requests while slots,
cells, emitters and the ray-queue budget allow, advances every active
member by one step, and retires members that have taken their last step
(their fields go back to the host).  Each member's state stays on the
device from admission to retirement.

``serve_sequential`` runs the same requests one at a time through the
single-simulation path, for comparison on the same arrival stream.
"""
from __future__ import annotations

import dataclasses as dc
import time

import numpy as np

from .flexrt import Batch, FlexRTError, Simulation

CELL_BYTES = 8 + 8 + 4 + 4 + 4 + 8 + 16      # n_H, y, x, T, Gamma, kappa, deposits
EMITTER_BYTES = 16 + 4 + 8 + 4 + 4 + 8        # plus the rotation ring


@dc.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    steps: int
    segments: int
    fields: dict

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def ray_bytes(nbins: int) -> int:
    return 24 + 4 * nbins


def plan_capacity(hbm_budget_bytes: float, nbins: int, max_grid: int, queue_fraction: float = 0.7):
    """Split an HBM budget between the two ray queues and the cell arena."""
    q = hbm_budget_bytes * queue_fraction
    rays = int(q / (2 * ray_bytes(nbins)))
    cells = int(hbm_budget_bytes * (1 - queue_fraction) * 0.9 / CELL_BYTES)
    return rays, max(cells, max_grid ** 3)


def serve(requests, hbm_budget_bytes=150e9, max_sims=256, max_grid=160, nbins=3, emitter_capacity=65536,
          admit_queue_fraction=0.5, launch=None, clock=time.perf_counter, keep_fields=False, stream=None,
          batch=None, sleep=time.sleep):
    """Run `requests` = [(arrival_seconds, problem), ...] (sorted by arrival)
    through one continuously batched engine.  Returns (results, stats).
    `batch` replaces the engine (an object with the Batch methods)."""
    if batch is None:
        rays, cells = plan_capacity(hbm_budget_bytes, nbins, max_grid)
        B = Batch(max_sims=max_sims, max_grid=max_grid, nbins=nbins, ray_capacity=rays, cell_capacity=cells,
                  emitter_capacity=emitter_capacity, use_graph=True, stream=stream)
    else:
        B = batch
    if launch:
        B.set_launch(*launch)
    pending = list(enumerate(requests))
    active = {}          # slot -> [rid, arrival, admitted, steps_left, steps_total]
    results = []
    t0 = clock()
    steps = 0
    peak_active = 0
    while pending or active:
        now = clock() - t0
        # admission between steps
        while pending and pending[0][1][0] <= now:
            rid, (arr, prob) = pending[0]
            info = B.info()
            if info["queue_used"] > admit_queue_fraction * info["ray_capacity"]:
                break
            try:
                slot = B.add(prob)
            except FlexRTError as e:
                if e.status == 3:            # no slot, cells or emitters: wait
                    break
                raise
            active[slot] = [rid, arr, clock() - t0, prob.nsteps, prob.nsteps]
            pending.pop(0)
        if not active:
            # idle: wait for the next arrival
            wait = pending[0][1][0] - (clock() - t0)
            if wait > 0:
                sleep(min(wait, 0.01))
            continue
        peak_active = max(peak_active, len(active))
        B.step()
        steps += 1
        finished = [s for s, a in active.items() if a[3] == 1]
        for s in active:
            active[s][3] -= 1
        if finished:
            B.sync()
            for s in finished:
                rid, arr, adm, _, total = active.pop(s)
                f = B.fields(s) if keep_fields else {}
                c = B.counts(s)
                results.append(Result(rid, arr, adm, clock() - t0, total, c["segments_total"], f))
                B.retire(s)
    B.sync()
    wall = clock() - t0
    B.close()
    return results, summarize(results, wall, extra={"batch_steps": steps, "peak_active": peak_active})


def serve_sequential(requests, ray_capacity=None, launch=None, clock=time.perf_counter, keep_fields=False,
                     stream=None):
    """The same requests one at a time through flexrt_create / flexrt_step."""
    results = []
    t0 = clock()
    for rid, (arr, prob) in enumerate(requests):
        now = clock() - t0
        if arr > now:
            time.sleep(arr - now)
        adm = clock() - t0
        cap = ray_capacity or max(1 << 20, 64 * prob.ncell)
        s = Simulation(prob, ray_capacity=cap, stream=stream)
        if launch:
            s.set_launch(*launch)
        for _ in range(prob.nsteps):
            s.step(prob.dt)
        f = s.fields() if keep_fields else {}
        c = s.counts()
        s.close()
        results.append(Result(rid, arr, adm, clock() - t0, prob.nsteps, c["segments_total"], f))
    wall = clock() - t0
    return results, summarize(results, wall)


def summarize(results, wall, extra=None):
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    segs = sum(r.segments for r in results)
    out = {"requests": len(results), "wall_s": wall, "sims_per_hour": 3600.0 * len(results) / wall,
           "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
           "mean_s": float(lat.mean()), "segments_per_s": segs / wall}
    if extra:
        out.update(extra)
    return out
