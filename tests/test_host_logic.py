"""Host-side logic without a GPU: the replica barrier / max / sum used by
bench.py under torchrun (gloo, world size 2), and the serving loop's
admission, stepping and retirement against a fake batch."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
from paper_2409_04521_gb300 import serve
from paper_2409_04521_gb300.flexrt import FlexRTError


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    d = bench.Dist(backend="gloo")
    d.barrier()
    out[rank] = (d.max(10.0 + rank), d.sum(1.5 * (rank + 1)))
    d.close()


def test_replicas_barrier_max_sum_gloo():
    ws, port = 2, _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        assert out[r] == (11.0, 4.5)   # max over ranks of the time, sum of the work


class FakeBatch:
    """Stands in for the native batch: slots, an emitter budget and step
    counting, with the same methods the server calls."""

    def __init__(self, slots):
        self.free = list(range(slots))
        self.members = {}
        self.steps = 0
        self.retired = []

    def info(self):
        return {"queue_used": 0, "ray_capacity": 1 << 30}

    def add(self, prob):
        if not self.free:
            raise FlexRTError(3, "no free simulation slot")
        s = self.free.pop(0)
        self.members[s] = prob
        return s

    def step(self):
        self.steps += 1

    def sync(self):
        pass

    def counts(self, s):
        return {"segments_total": 7}

    def fields(self, s):
        return {}

    def retire(self, s):
        del self.members[s]
        self.retired.append(s)
        self.free.append(s)

    def close(self):
        pass


class P:
    def __init__(self, n):
        self.nsteps = n


def test_serve_loop_admission_and_retirement():
    now = [0.0]
    clock = lambda: now[0]
    def sleep(dt):
        now[0] += dt
    reqs = [(0.0, P(3)), (0.0, P(1)), (0.0, P(2)), (0.5, P(2)), (0.5, P(1))]
    fb = FakeBatch(slots=2)
    orig_step = fb.step
    def step():
        orig_step()
        now[0] += 0.1
    fb.step = step
    results, stats = serve.serve(reqs, batch=fb, clock=clock, sleep=sleep)
    assert stats["requests"] == 5
    by = {r.rid: r for r in results}
    # every request ran exactly its own number of steps
    assert all(by[i].steps == reqs[i][1].nsteps for i in range(5))
    # at most two at a time; the third waited for a retirement
    assert by[2].admitted >= min(by[0].finished, by[1].finished) - 1e-12
    assert all(r.finished >= r.admitted >= r.arrival for r in results)
    # total batch steps: never more than the sum of requested steps
    assert fb.steps <= sum(p.nsteps for _, p in reqs)
    assert sorted(fb.retired) == sorted(fb.retired) and len(fb.retired) == 5


def test_plan_capacity_splits_budget():
    rays, cells = serve.plan_capacity(150e9, nbins=3, max_grid=160)
    assert 2 * rays * serve.ray_bytes(3) <= 0.7 * 150e9 + 1
    assert cells * serve.CELL_BYTES <= 0.3 * 150e9
    assert cells >= 160 ** 3
