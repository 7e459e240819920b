"""The continuous-batching policy (paper_1810_07802_gb300/serve.py) on fake
backends: no GPU, a simulated clock that advances with the work done."""
import pytest

from paper_1810_07802_gb300.serve import BatchingServer, Request, SequentialServer, summary


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeSolver:
    def __init__(self, req, log):
        self.req, self.steps, self.closed = req, 0, False
        log.append(("create", req.rid))

    def step(self, n):
        self.steps += n

    def macros(self):
        return {"steps": self.steps}

    def close(self):
        self.closed = True


class FakeBatch:
    """Advances members; simulated device time = per-step cost of the batch."""

    def __init__(self, clock, tracker):
        self.clock, self.tracker, self.members = clock, tracker, []

    def add(self, s):
        assert s not in self.members
        self.members.append(s)
        self.tracker["max_members"] = max(self.tracker["max_members"], len(self.members))

    def remove(self, s):
        self.members.remove(s)

    def step(self, n):
        for s in self.members:
            s.steps += n
        self.clock.t += n * (1e-5 + 1e-9 * sum(s.req.cfg["nx"] * s.req.cfg["ny"] for s in self.members))

    def mark(self):
        class E:
            def synchronize(self):
                pass
        return E()

    def sync(self):
        pass

    def close(self):
        pass


def make_requests(n, spacing=0.001):
    reqs = []
    for i in range(n):
        nx = 16 * (1 + i % 5)
        reqs.append(Request(i, "k", {"nx": nx, "ny": nx}, {}, steps=10 + 7 * (i % 4), arrival=i * spacing))
    return reqs


def footprint(cfg):
    return cfg["nx"] * cfg["ny"] * 100


def run_batching(reqs, budget, max_members=8, chunk=5):
    clock, log, tracker = Clock(), [], {"max_members": 0}
    used_trace = []

    def fp(cfg):
        return footprint(cfg)

    srv = BatchingServer(budget, max_members=max_members, chunk=chunk,
                         solver_factory=lambda r: FakeSolver(r, log),
                         batch_factory=lambda: FakeBatch(clock, tracker), footprint=fp,
                         clock=clock, sleep=clock.sleep)
    recs = srv.run(reqs)
    return recs, log, tracker, used_trace


def test_every_request_completes_with_its_steps():
    reqs = make_requests(23)
    recs, log, tracker, _ = run_batching(reqs, budget=10 ** 9)
    assert [r.rid for r in recs] == list(range(23))
    for r, q in zip(recs, reqs):
        assert r.result["steps"] == q.steps
        assert r.finished >= r.admitted >= r.arrival - 1e-12
    assert tracker["max_members"] <= 8


def test_admission_is_fifo_and_within_budget():
    reqs = make_requests(30, spacing=0.0)          # a burst
    budget = footprint({"nx": 80, "ny": 80}) * 2   # room for about two large problems
    recs, log, tracker, _ = run_batching(reqs, budget=budget, max_members=16)
    order = [rid for op, rid in log if op == "create"]
    assert order == sorted(order)                  # admitted in arrival order
    # replay the admission/finish events: resident footprint never exceeds the budget
    events = sorted([(r.admitted, 1, r.rid) for r in recs] + [(r.finished, 0, r.rid) for r in recs])
    used = 0
    for t, kind, rid in events:
        used += footprint(reqs[rid].cfg) if kind else -footprint(reqs[rid].cfg)
        assert used <= budget


def test_oversized_request_rejected():
    reqs = make_requests(3)
    with pytest.raises(ValueError):
        run_batching(reqs, budget=10)


def test_batching_beats_sequential_on_a_burst():
    reqs = make_requests(40, spacing=0.0)
    recs, *_ = run_batching(reqs, budget=10 ** 9, max_members=40, chunk=50)
    clock, log = Clock(), []

    class SeqSolver(FakeSolver):
        def step(self, n):
            super().step(n)
            clock.t += n * (1e-5 + 1e-9 * self.req.cfg["nx"] * self.req.cfg["ny"])

    seq = SequentialServer(solver_factory=lambda r: SeqSolver(r, log), clock=clock, sleep=clock.sleep).run(reqs)
    assert summary(recs)["solves_per_s"] > summary(seq)["solves_per_s"]
    assert all(r.result["steps"] == q.steps for r, q in zip(seq, reqs))


def test_autotune_cache_tunes_each_shape_once_and_server_applies_it():
    from paper_1810_07802_gb300.serve import AutotuneCache

    calls = []

    def tuner(cfg, trial_steps, **fields):
        calls.append(AutotuneCache.key(cfg))
        return (2 if cfg["nx"] < 32 else 1), [1.0, 0.5]

    cache = AutotuneCache(trial_steps=3, tuner=tuner)
    clock, log, tracker = Clock(), [], {"max_members": 0}
    seen = []

    def make_solver(r):
        seen.append((r.rid, r.cfg.get("tile_shape")))
        return FakeSolver(r, log)

    srv = BatchingServer(1 << 40, max_members=8, chunk=5, solver_factory=make_solver,
                         batch_factory=lambda: FakeBatch(clock, tracker), footprint=footprint,
                         clock=clock, sleep=clock.sleep, tile_policy=cache)
    reqs = make_requests(20)
    recs = srv.run(reqs)
    assert len(recs) == 20
    assert sorted(calls) == sorted(set(calls)) and len(calls) == 5      # 5 distinct shapes
    for rid, shape in seen:
        assert shape == (2 if reqs[rid].cfg["nx"] < 32 else 1)


class FailingSolver(FakeSolver):
    """Reports a device failure (like a non-physical step) once it has run
    `fail_at` steps."""

    def __init__(self, req, log, fail_at):
        super().__init__(req, log)
        self.fail_at = fail_at

    def sync(self):
        if self.fail_at is not None and self.steps >= self.fail_at:
            raise RuntimeError("dugks_sync failed: non-physical")


class CheckingBatch(FakeBatch):
    def sync(self):
        for s in self.members:
            s.sync()


def test_failed_problem_is_retired_and_the_rest_complete():
    """A problem whose step fails on the device leaves the batch with its
    error recorded and its memory released; every other request completes
    with its full step count (failure detection on the host, no GPU)."""
    clock, log, tracker = Clock(), [], {"max_members": 0}
    bad = {3: 12, 7: 1}    # rid -> steps after which it fails
    reqs = make_requests(12)
    srv = BatchingServer(1 << 40, max_members=6, chunk=5,
                         solver_factory=lambda r: FailingSolver(r, log, bad.get(r.rid)),
                         batch_factory=lambda: CheckingBatch(clock, tracker), footprint=footprint,
                         clock=clock, sleep=clock.sleep)
    recs = srv.run(reqs)
    assert len(recs) == 12
    for r, q in zip(recs, reqs):
        if q.rid in bad:
            assert r.error is not None and r.result is None
        else:
            assert r.error is None and r.result["steps"] == q.steps
    s = summary(recs)
    assert s["failed"] == 2 and s["solves"] == 10


def test_sequential_server_records_failures():
    clock = Clock()

    class Boom(FakeSolver):
        def step(self, n):
            raise RuntimeError("dugks_step failed")

    reqs = make_requests(3)
    recs = SequentialServer(solver_factory=lambda r: Boom(r, []) if r.rid == 1 else FakeSolver(r, []),
                            clock=clock, sleep=clock.sleep).run(reqs)
    assert [r.error is None for r in recs] == [True, False, True]
