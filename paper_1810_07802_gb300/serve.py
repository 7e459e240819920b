"""Continuous-batching service for DUGKS solves (host-side scheduling only).

Requests arrive over time; each asks for a problem (parameters + initial
fields) advanced by a number of steps.  The server keeps every admitted
problem's state resident on the GPU, admits waiting requests in arrival order
whenever their device footprint (dugks_workspace_bytes) fits the budget and a
slot is free, advances all resident problems together with dugks_batch_step
(one launch per kernel variant per step, replayed from a CUDA graph), and
retires each problem when its steps are done, reading its macros back.  New
requests join the running batch between chunks of steps, so their work
overlaps on the device with the problems already in flight.

`SequentialServer` is the reference policy: one problem at a time, stepped by
per-step launches.  Both record, per request, its arrival, admission and
completion times; `summary` turns them into solves/s and p50/p99 latency.

The backends are injectable (solver_factory, batch_factory, footprint,
clock, sleep) so the policy itself is testable without a GPU.
"""
import collections
import time

import numpy as np


class Request:
    __slots__ = ("rid", "kind", "cfg", "fields", "steps", "arrival")

    def __init__(self, rid, kind, cfg, fields, steps, arrival):
        self.rid, self.kind, self.cfg, self.fields = rid, kind, cfg, fields
        self.steps, self.arrival = int(steps), float(arrival)


class Record:
    __slots__ = ("rid", "kind", "arrival", "admitted", "finished", "cells", "steps", "result", "error")

    def __init__(self, req):
        self.rid, self.kind, self.arrival = req.rid, req.kind, req.arrival
        self.cells = int(req.cfg["nx"]) * int(req.cfg["ny"])
        self.steps = req.steps
        self.admitted = self.finished = None
        self.result = None
        self.error = None   # set when the problem failed (e.g. a non-finite or non-physical step)

    @property
    def latency(self):
        return self.finished - self.arrival


def summary(records):
    """Throughput and latency of a finished run (times in seconds); failed
    requests are counted apart and left out of the latency figures."""
    failed = sum(1 for r in records if r.error is not None)
    records = [r for r in records if r.error is None]
    if not records:
        return {"solves": 0, "failed": failed}
    lat = np.array([r.latency for r in records])
    t0 = min(r.arrival for r in records)
    t1 = max(r.finished for r in records)
    updates = sum(r.cells * r.steps for r in records)
    return {"solves": len(records), "failed": failed, "solves_per_s": len(records) / (t1 - t0),
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "makespan_s": t1 - t0,
            "mlups": updates / (t1 - t0) / 1e6}


class AutotuneCache:
    """Step-kernel tile shape per problem shape (precision, model, y-boundary,
    nx, ny), measured once with dugks_autotune on the first problem of that
    shape and reused for every later one."""

    def __init__(self, trial_steps=10, tuner=None):
        if tuner is None:
            from . import solver as S

            tuner = S.autotune
        self.tuner, self.trial_steps = tuner, int(trial_steps)
        self.shapes = {}
        self.timings = {}

    @staticmethod
    def key(cfg):
        return (cfg.get("precision", "fp64"), cfg.get("model", "coupled"), cfg.get("bc_y", "periodic"),
                int(cfg["nx"]), int(cfg["ny"]))

    def __call__(self, cfg, fields):
        k = self.key(cfg)
        if k not in self.shapes:
            best, ms = self.tuner(cfg, trial_steps=self.trial_steps, **fields)
            self.shapes[k], self.timings[k] = int(best), ms
        return self.shapes[k]


class BatchingServer:
    """Continuous batching with admission by device-memory footprint.

    hbm_budget: bytes of solver workspaces that may be resident at once.
    max_members: slots (resident problems) at most.
    chunk: steps enqueued between scheduling decisions at most.
    tile_policy: None (the library's default tile shape) or a callable
      (cfg, fields) -> tile_shape, e.g. an AutotuneCache.
    persistent: advance the batch in persistent launches of up to 16 steps
      (dugks_batch_set_persistent) instead of one grid launch per step.
    """

    def __init__(self, hbm_budget, max_members=128, chunk=50, stream=None, solver_factory=None,
                 batch_factory=None, footprint=None, clock=time.perf_counter, sleep=time.sleep,
                 keep_results=True, tile_policy=None, persistent=False):
        if solver_factory is None:
            import torch

            from . import solver as S

            # solvers are created (and their macros read) on one stream, the
            # batch runs on another; the server synchronises between them
            self.create_stream = stream if stream is not None else torch.cuda.Stream()
            self.batch_stream = torch.cuda.Stream()
            solver_factory = lambda req: S.Solver(req.cfg, stream=self.create_stream, **req.fields)  # noqa: E731
            batch_factory = batch_factory or (lambda: S.Batch(stream=self.batch_stream, persistent=persistent))
            footprint = footprint or S.workspace_bytes
        self.hbm_budget = int(hbm_budget)
        self.max_members = int(max_members)
        self.chunk = int(chunk)
        self.make_solver, self.make_batch, self.footprint = solver_factory, batch_factory, footprint
        self.clock, self.sleep = clock, sleep
        self.keep_results = keep_results
        self.tile_policy = tile_policy

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        for r in reqs:
            if self.tile_policy is not None and "tile_shape" not in r.cfg:
                r.cfg = dict(r.cfg, tile_shape=int(self.tile_policy(r.cfg, r.fields)))
            if self.footprint(r.cfg) > self.hbm_budget:
                raise ValueError("request %d needs more device memory than the whole budget" % r.rid)
        pending = collections.deque(reqs)
        queue = collections.deque()
        active = []  # [req, record, solver, steps_left, bytes]
        used = 0
        done = []
        batch = self.make_batch()
        inflight = None
        t0 = self.clock()
        try:
            while pending or queue or active:
                now = self.clock() - t0
                while pending and pending[0].arrival <= now:
                    queue.append(pending.popleft())
                # admission in arrival order while memory and slots allow
                while queue and len(active) < self.max_members:
                    need = self.footprint(queue[0].cfg)
                    if used + need > self.hbm_budget:
                        break
                    req = queue.popleft()
                    rec = Record(req)
                    rec.admitted = self.clock() - t0
                    s = self.make_solver(req)
                    batch.add(s)
                    active.append([req, rec, s, req.steps, need, None])
                    used += need
                if not active:
                    if pending:
                        self.sleep(max(0.0, pending[0].arrival - (self.clock() - t0)))
                    continue
                k = min(self.chunk, min(a[3] for a in active))
                batch.step(k)
                mark = batch.mark()
                for a in active:
                    a[3] -= k
                finished = [a for a in active if a[3] == 0]
                if not finished:
                    # keep at most two chunks queued, so arrivals join soon
                    if inflight is not None:
                        inflight.synchronize()
                    inflight = mark
                else:
                    inflight = None
                    for a in self._sync_members(batch, active):
                        # a failed problem leaves the batch at once; the others go on
                        req, rec, s = a[0], a[1], a[2]
                        rec.finished = self.clock() - t0
                        rec.error = a[5]
                        batch.remove(s)
                        try:
                            s.close()
                        except Exception:
                            pass
                        used -= a[4]
                        active.remove(a)
                        done.append(rec)
                    finished = [a for a in active if a[3] == 0]
                    for a in finished:
                        req, rec, s = a[0], a[1], a[2]
                        res = s.macros()
                        rec.finished = self.clock() - t0
                        rec.result = res if self.keep_results else None
                        batch.remove(s)
                        s.close()
                        used -= a[4]
                        active.remove(a)
                        done.append(rec)
        finally:
            for a in active:
                try:
                    batch.remove(a[2])
                    a[2].close()
                except Exception:
                    pass
            batch.close()
        return sorted(done, key=lambda r: r.rid)

    @staticmethod
    def _sync_members(batch, active):
        """Waits for the batch; if that reports a failure, asks every member
        and returns those that failed, each with its error in slot 5."""
        try:
            batch.sync()
            return []
        except Exception as e:
            failed = []
            for a in active:
                try:
                    a[2].sync()
                except Exception as em:
                    a[5] = str(em)
                    failed.append(a)
            if not failed:
                raise e
            return failed


class SequentialServer:
    """One problem at a time in arrival order, stepped by per-step launches."""

    def __init__(self, stream=None, solver_factory=None, clock=time.perf_counter, sleep=time.sleep,
                 keep_results=True):
        if solver_factory is None:
            import torch

            from . import solver as S

            stream = stream if stream is not None else torch.cuda.Stream()
            solver_factory = lambda req: S.Solver(req.cfg, stream=stream, **req.fields)  # noqa: E731
        self.make_solver, self.clock, self.sleep = solver_factory, clock, sleep
        self.keep_results = keep_results

    def run(self, requests):
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        done = []
        t0 = self.clock()
        for req in reqs:
            wait = req.arrival - (self.clock() - t0)
            if wait > 0:
                self.sleep(wait)
            rec = Record(req)
            rec.admitted = self.clock() - t0
            s = self.make_solver(req)
            try:
                s.step(req.steps)
                res = s.macros()
                rec.result = res if self.keep_results else None
            except Exception as e:
                rec.error = str(e)
            rec.finished = self.clock() - t0
            try:
                s.close()
            except Exception:
                pass
            done.append(rec)
        return sorted(done, key=lambda r: r.rid)
