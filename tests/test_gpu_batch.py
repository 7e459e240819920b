"""Batches and the serving loop on the GPU.

A problem's result does not depend on what it is batched with: stepped in a
batch of one, in a mix of other sizes, precisions and models, or through the
continuous-batching server, it is bit-identical.  The batched kernel and the
single-problem kernel run the same tile code but are compiled separately
(constants from a device descriptor vs the parameter space), so the compiler
may fuse multiply-adds differently: the two paths agree to round-off, and
both agree with the oracle (test_gpu_parity).  A member large enough to fill
the GPU by itself (2048 tiles or more) is stepped by the single-problem kernel
inside the batch and is bit-identical to stepping it alone.  Batches advance
by default with one grid launch per step; the persistent mode advances up to
16 steps per launch, in which a tile waits only for its own member's previous
step.  Both are checked against the oracle and against each other."""
import numpy as np
import pytest

from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


def problems():
    out = []
    cfg, f = W.random_state(150, 70, seed=1)
    out.append((cfg, f))
    cfg, f = W.random_state(37, 29, seed=2, bc_y="wall")
    out.append((dict(cfg, precision="fp32", phi_ref=0.5), f))
    cfg, f = W.stationary_bubble(N=64, R=16.0, rho_ratio=10.0)
    out.append((dict(cfg, precision="fp32", phi_ref=0.5), f))
    cfg, f = W.layered_poiseuille(ny=64, nx=4, mu_ratio=100.0)
    out.append((cfg, f))
    cfg, f = W.translation_circle(L=40, R=10.0, U=0.02)
    out.append((cfg, f))
    cfg, f = W.spinodal(N=96)
    out.append((dict(cfg, precision="fp32"), f))
    # other compiled tile shapes form their own kernel groups
    cfg, f = W.layered_poiseuille(ny=128, nx=4, mu_ratio=100.0)
    out.append((dict(cfg, precision="fp32", phi_ref=0.5, tile_shape=4), f))
    cfg, f = W.random_state(33, 40, seed=3)
    out.append((dict(cfg, tile_shape=2), f))
    cfg, f = W.random_state(45, 21, seed=4)
    out.append((dict(cfg, recon="upwind"), f))
    cfg, f = W.random_state(38, 23, seed=6, bc_y="wall")
    out.append((dict(cfg, recon="upwind", precision="fp32", phi_ref=0.5), f))
    cfg, f = W.zalesak_disk(L=36, R=12.0, slot=3.0, U=0.04)
    r = np.random.default_rng(9)
    out.append((dict(cfg, velocity_field="sampled"),
                dict(f, ux0=0.02 * r.standard_normal((36, 36)), uy0=0.02 * r.standard_normal((36, 36)))))
    return out


def alone(S, cfg, f, steps, persistent=False):
    """The problem stepped by itself in a batch of one."""
    import torch

    st = torch.cuda.Stream()
    with S.Solver(cfg, stream=st, **f) as s:
        with S.Batch(stream=st, persistent=persistent) as b:
            b.add(s)
            b.step(steps)
            b.sync()
            b.remove(s)
        return s.macros(), s.get_state()


def single_path(S, cfg, f, steps):
    with S.Solver(cfg, **f) as s:
        s.step(steps)
        return s.macros()


def assert_round_off(cfg, m, m0, what=""):
    """Agreement of two compilations of the same arithmetic."""
    fp32 = cfg.get("precision", "fp64") == "fp32"
    for k in m:
        scale = max(1.0, np.abs(m0[k]).max())
        tol = (2e-6 if fp32 else 1e-12) * scale
        err = np.abs(m[k] - m0[k]).max()
        assert err <= tol, (what, k, err)


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_member_bit_identical_to_batch_of_one(S, persistent):
    import torch

    probs = problems()
    st = torch.cuda.Stream()
    solvers = [S.Solver(c, stream=st, **f) for c, f in probs]
    with S.Batch(stream=st, persistent=persistent) as b:
        for s in solvers:
            b.add(s)
        assert len(b) == len(solvers)
        b.step(3)
        b.step(4)
        b.sync()
    for s, (c, f) in zip(solvers, probs):
        assert s.step_count == 7
        m, state = s.macros(), s.get_state()
        m0, state0 = alone(S, c, f, 7, persistent)
        for k in m:
            assert np.array_equal(m[k], m0[k]), (c["nx"], c["ny"], k)
        assert np.array_equal(state, state0)
        assert_round_off(c, m, single_path(S, c, f, 7), (c["nx"], c["ny"]))
        s.close()


def test_large_members_take_the_single_problem_kernel(S):
    """FP64 512 x 512 (32 x 64 tiles of 16 x 8), FP32 1024 x 512 (32 x 64
    tiles of 32 x 8) and an upwind FP64 512 x 512 member sit at the 2048-tile
    threshold: inside a mixed batch each gives the bits of stepping it alone
    with dugks_step, across a membership change and an odd step count, while
    the small members keep the bits of their batch of one."""
    import torch

    big = []
    cfg, f = W.random_state(512, 512, seed=21)
    big.append((cfg, f))
    cfg, f = W.random_state(1024, 512, seed=22, rho_ratio=100.0)
    big.append((dict(cfg, precision="fp32", phi_ref=0.5), f))
    cfg, f = W.random_state(512, 512, seed=23)
    big.append((dict(cfg, recon="upwind"), f))
    small = problems()[:3]
    cfg, f = W.random_state(511, 512, seed=24)      # 2048 tiles of the last column ragged
    edge = (cfg, f)
    cfg, f = W.random_state(496, 512, seed=25)      # 31 x 64 = 1984 tiles: batched kernel
    below = (cfg, f)
    st = torch.cuda.Stream()
    everyone = big + small + [edge, below]
    solvers = [S.Solver(c, stream=st, **f) for c, f in everyone]
    with S.Batch(stream=st) as b:
        for s in solvers[:-1]:
            b.add(s)
        b.step(5)
        b.remove(solvers[0])
        b.add(solvers[-1])
        b.step(18)                  # one graph of 16 steps and two single steps
        b.sync()
    want = [5] + [23] * (len(everyone) - 2) + [18]
    for i, (s, (c, f), n) in enumerate(zip(solvers, everyone, want)):
        assert s.step_count == n
        m, state = s.macros(), s.get_state()
        if i < len(big) or i == len(big) + len(small):
            with S.Solver(c, **f) as ref:
                ref.step(n)
                m0, state0 = ref.macros(), ref.get_state()
        else:
            m0, state0 = alone(S, c, f, n)
        for k in m:
            assert np.array_equal(m[k], m0[k]), (i, k)
        assert np.array_equal(state, state0), i
        s.close()


def test_batch_membership_changes(S):
    import torch

    probs = problems()[:4]
    st = torch.cuda.Stream()
    solvers = [S.Solver(c, stream=st, **f) for c, f in probs]
    with S.Batch(stream=st) as b:
        b.add(solvers[0])
        b.add(solvers[1])
        b.step(2)
        b.add(solvers[2])
        b.step(3)
        b.remove(solvers[0])
        b.add(solvers[3])
        b.step(4)
        b.sync()
    want = [5, 9, 7, 4]
    for s, (c, f), n in zip(solvers, probs, want):
        assert s.step_count == n
        m0, _ = alone(S, c, f, n)
        m = s.macros()
        for k in m:
            assert np.array_equal(m[k], m0[k])
        s.close()


@pytest.mark.parametrize("persistent", [False, True])
def test_serving_results_identical_alone_and_in_the_mix(S, persistent):
    """Continuous batching (grid or persistent batch launches): each served
    result is bit-identical to the same problem in a batch of one of the same
    mode, and agrees to round-off with the one-at-a-time server."""
    from paper_1810_07802_gb300.serve import BatchingServer, Request, SequentialServer, summary

    trace = W.serving_trace(n=10, rate=400.0, seed=5, steps={"poiseuille": 30, "bubble": 20, "spinodal": 15})
    small = []
    for i, (kind, cfg, f, steps, t) in enumerate(trace):
        if cfg["nx"] * cfg["ny"] > 256 * 256:        # keep the test quick
            cfg, f = W.spinodal(N=128, seed=99 + i)
            cfg["precision"] = "fp32"
        small.append(Request(i, kind, cfg, f, steps, t))
    srv = BatchingServer(hbm_budget=8 << 30, max_members=6, chunk=8, persistent=persistent)
    recs = srv.run(small)
    assert len(recs) == len(small)
    for r, q in zip(recs, small):
        m0, _ = alone(S, q.cfg, q.fields, q.steps, persistent)
        for k in m0:
            assert np.array_equal(r.result[k], m0[k]), (q.rid, k)
    s = summary(recs)
    assert s["solves"] == len(small) and s["p99_ms"] >= s["p50_ms"] > 0
    seq = SequentialServer().run(small)
    for r, q in zip(seq, small):
        assert_round_off(q.cfg, r.result, recs[q.rid].result, q.rid)


def test_server_retires_a_failing_problem(S):
    """A request whose first step is non-physical (phi < -1/999 at density
    ratio 1000) fails in the batch; the server records its error and every
    other request completes bit-identical to its batch of one."""
    from paper_1810_07802_gb300.serve import BatchingServer, Request, summary

    reqs = []
    for i in range(5):
        cfg, f = W.random_state(40 + 3 * i, 30, seed=50 + i)
        reqs.append(Request(i, "ok", cfg, f, 12, 0.0))
    cfg, f = W.spinodal(N=32)
    f = dict(f, phi0=np.full((32, 32), -0.01))
    reqs.append(Request(5, "bad", cfg, f, 12, 0.0))
    recs = BatchingServer(hbm_budget=4 << 30, max_members=8, chunk=4).run(reqs)
    assert recs[5].error is not None and "NONPHYSICAL" in recs[5].error
    for r, q in zip(recs[:5], reqs[:5]):
        assert r.error is None
        m0, _ = alone(S, q.cfg, q.fields, q.steps)
        for k in m0:
            assert np.array_equal(r.result[k], m0[k]), (q.rid, k)
    s = summary(recs)
    assert s["failed"] == 1 and s["solves"] == 5


@pytest.mark.parametrize("persistent", [True, False])
def test_batch_members_match_the_oracle(S, persistent):
    """Every member of a mixed batch against the FP64 oracle directly (not
    through the single-problem kernel): two batched steps, a membership change,
    then 17 steps (one replay of the 16-step graph and one single step).  FP64
    members within 1e-10 on phi, p, u and the stored distributions; FP32
    members within the FP32 round-off bounds the single-problem tests use."""
    import torch

    from oracle.oracle import Oracle

    probs = problems()
    st = torch.cuda.Stream()
    solvers = [S.Solver(c, stream=st, **f) for c, f in probs]
    late = len(probs) - 1
    with S.Batch(stream=st, persistent=persistent) as b:
        for s in solvers[:late]:
            b.add(s)
        b.step(2)
        b.remove(solvers[0])
        b.add(solvers[late])
        b.step(17)
        b.sync()
    want = [2] + [19] * (late - 1) + [17]
    for s, (c, f), n in zip(solvers, probs, want):
        assert s.step_count == n
        o = Oracle({k: v for k, v in c.items() if k not in ("precision", "phi_ref", "p_ref", "tile_shape")}, **f)
        o.step(n)
        ref = o.macros()
        got = s.macros()
        what = "%dx%d %s %s" % (c["nx"], c["ny"], c.get("precision", "fp64"), c.get("model", "coupled"))
        if c.get("precision", "fp64") == "fp64":
            for k in ("phi", "p", "ux", "uy"):
                assert np.abs(got[k] - ref[k]).max() <= 1e-10, (what, k)
            for name, a, r in zip(("f", "g", "phiu"), s.distributions(), o.state()):
                assert np.abs(a - r).max() <= 1e-10, (what, name)
        else:
            assert np.abs(got["phi"] - ref["phi"]).max() <= 2e-5, what
            assert np.abs(got["ux"] - ref["ux"]).max() <= 1e-7, what
            assert np.abs(got["uy"] - ref["uy"]).max() <= 1e-7, what
            assert np.abs(got["p"] - ref["p"]).max() <= 1e-5, what
        s.close()


def _mix_run(S, persistent, steps):
    import torch

    probs = problems()
    # members of very different tile counts, so that small ones run ahead
    cfg, f = W.spinodal(N=480)
    probs.append((dict(cfg, precision="fp32"), f))
    cfg, f = W.random_state(20, 9, seed=12)
    probs.append((cfg, f))
    st = torch.cuda.Stream()
    solvers = [S.Solver(c, stream=st, **f) for c, f in probs]
    with S.Batch(stream=st, persistent=persistent) as b:
        for s in solvers:
            b.add(s)
        b.step(steps)
        b.sync()
    out = []
    for s, (c, f) in zip(solvers, probs):
        assert s.step_count == steps
        out.append((c, s.macros(), s.get_state()))
        s.close()
    return out


def test_persistent_and_grid_launches_agree(S):
    """37 steps (two 16-step launches and five single ones) of a mix of 13
    members from 1 to 900 tiles in both modes.  The two kernels run the same
    tile code with the same descriptor constants but are compiled separately,
    so they agree to round-off; the per-member queue order changes nothing
    else."""
    a = _mix_run(S, True, 37)
    b = _mix_run(S, False, 37)
    same = 0
    for (c, m, st), (_, m0, st0) in zip(a, b):
        assert_round_off(c, m, m0, ("modes", c["nx"], c["ny"]))
        same += int(np.array_equal(st, st0))
    print("\npersistent vs grid launches: %d of %d members bit-identical" % (same, len(a)), end="")


def test_persistent_wait_times_out_and_batches_still_run(S):
    """Failure detection without a fault: the persistent launch's wait for a
    member's previous step, run on a counter that nothing raises, gives up
    after its sleep budget (the kernel's own, about 2 s, and a short one); the
    host reads DUGKS_ERR_TIMEOUT and a persistent batch then still matches the
    oracle."""
    import time

    from oracle.oracle import Oracle

    t0 = time.perf_counter()
    assert S.check_batch_wait() == -6
    waited = time.perf_counter() - t0
    assert 1.0 < waited < 10.0, waited
    assert S.check_batch_wait(budget_ns=1000000) == -6
    cfg, f = W.random_state(40, 30, seed=8)
    import torch

    st = torch.cuda.Stream()
    with S.Solver(cfg, stream=st, **f) as s:
        with S.Batch(stream=st, persistent=True) as b:
            b.add(s)
            b.step(18)
            b.sync()
            b.remove(s)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(18)
    ref = o.macros()
    for k in ("phi", "p", "ux", "uy"):
        assert np.abs(got[k] - ref[k]).max() <= 1e-10, k
