"""Throughput benchmark of the coupled phase-field DUGKS step on GB300.

Workload: the spinodal-decomposition box (Sec. IV.C shape; 2048 x 2048
periodic cells, density ratio 1000, viscosity ratio 10, sigma = 1e-3, W = 4,
M = 0.02, phi = 0.5 + 0.01 (2U - 1) from SplitMix64), distributions stored in
FP32 as deviations from the rest state.  One "step" is one DUGKS time step of
the whole box (one fused kernel launch).  Metric: million lattice-cell
updates per second (MLUPS), whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on every host core (one process per core, each stepping its own
2048 x 32 periodic band of the same seeded field).  Under torchrun each rank runs an independent replica (weak scaling).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS_SIDE = 2048
FP32_BYTES_PER_CELL = 18 * 4 * 2 + 2 * 4 * 2   # read + write psi~ (18 FP32) and (phi u) history (2 FP32)
FP64_BYTES_PER_CELL = 18 * 8 * 2 + 2 * 8 * 2
REF_BAND_ROWS = 128
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "solo_step_kernel_fp32_spinodal2048.md")
PROFILE_SUMMARY_FP64 = os.path.join(ROOT, "profiles", "solo_step_kernel_fp64_spinodal2048.md")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1810_07802_gb300", "csrc", f)
                  for f in ("dugks_device.cuh", "dugks_launch.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-upwind", action="store_true")
    return ap.parse_args()


def workload(nx=N_CELLS_SIDE, ny=N_CELLS_SIDE, precision="fp32"):
    from paper_1810_07802_gb300 import workloads as W

    cfg, f = W.spinodal(N=N_CELLS_SIDE)
    if ny != N_CELLS_SIDE or nx != N_CELLS_SIDE:
        f = {k: (None if v is None else v[:ny, :nx].copy()) for k, v in f.items()}
        cfg.update(nx=nx, ny=ny)
    cfg["precision"] = precision
    return cfg, f


def config_dict(precision):
    return {"workload": "spinodal decomposition 2048x2048 periodic, rho ratio 1000, nu ratio 10, "
                        "sigma 1e-3, W 4, M 0.02, coupled A-C + hydrodynamic D2Q9 DUGKS",
            "nx": N_CELLS_SIDE, "ny": N_CELLS_SIDE, "precision": precision,
            "storage": "SoA [18][ny][pitch] deviations from the rest state" if precision == "fp32"
                       else "SoA [18][ny][pitch] FP64",
            "l2": "inputs larger than L2 (two 302 MB FP32 state buffers vs 129 MB L2)",
            "launches_per_step": 1}


# ------------------------------------------------------------------ helpers

def job_time_and_value(local_secs, units_per_rank, world, device="cuda"):
    """Whole-job timing of independent replicas: the slowest rank's time and
    the units all ranks processed divided by it (weak scaling, no data-path
    collective; the one all-reduce carries the timings)."""
    secs = float(local_secs)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([secs], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        secs = float(t.item())
    return secs, units_per_rank * world / secs


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is busy."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.rows = []
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def summary(self):
        rows = getattr(self, "rows", [])
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (the NVIDIA
    driver's libnvidia-ml, via ctypes; reads only) every `period` seconds from a thread
    while the GPU runs, so that even a few milliseconds of timed steps give
    many samples.  Falls back to ClockSampler (nvidia-smi) if NVML cannot be
    loaded.  The device is found by the PCI bus id torch reports."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, period=0.002):
        import threading

        self.index, self.period = index, period
        self.fallback = None
        self.rows = []
        self.recording = threading.Event()   # set only while timed steps run

    def record(self, on):
        if on:
            self.recording.set()
        else:
            self.recording.clear()

    def _open(self):
        import ctypes

        import torch

        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = getattr(props, "pci_bus_id", None)
        ok = False
        if bus is not None:
            busid = "%08x:%02x:%02x.0" % (getattr(props, "pci_domain_id", 0), bus, getattr(props, "pci_device_id", 0))
            ok = nv.nvmlDeviceGetHandleByPciBusId_v2(busid.encode(), ctypes.byref(h)) == 0
        if not ok and nv.nvmlDeviceGetHandleByIndex_v2(int(self.index), ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        return nv, h, reasons

    def _run(self):
        import ctypes

        nv, h, reasons = self.nv, self.h, self.reasons_fn
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
        while not self.stop.is_set():
            if self.recording.is_set() and nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(clk)) == 0 and \
                    reasons(h, ctypes.byref(rs)) == 0:
                self.rows.append((clk.value, mx.value, rs.value))
            time.sleep(self.period)

    def __enter__(self):
        import threading

        try:
            self.nv, self.h, self.reasons_fn = self._open()
        except (OSError, AttributeError):
            self.fallback = ClockSampler(self.index).__enter__()
            return self
        self.stop = threading.Event()
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()
        return self

    def __exit__(self, *exc):
        if self.fallback is not None:
            return self.fallback.__exit__(*exc)
        self.stop.set()
        self.thread.join(5)

    def summary(self):
        if self.fallback is not None:
            return dict(self.fallback.summary(), sampler="nvidia-smi -lms 100")
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0, "sampler": "nvml"}
        sm = [r[0] for r in self.rows]
        reasons = sorted({name for r in self.rows for bit, name in self.REASONS.items() if r[2] & bit})
        return {"sm_mhz": statistics.median(sm), "sm_min_mhz": min(sm), "sm_max_mhz": max(r[1] for r in self.rows),
                "reasons": reasons, "samples": len(self.rows), "sampler": "nvml every %g ms" % (self.period * 1e3)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


def kernel_source_hash():
    """Hash of the step kernel's code with comments and layout removed, so that
    a profile stays valid across comment-only edits."""
    import re

    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        text = open(p, encoding="utf-8").read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profile_values(summary=PROFILE_SUMMARY):
    """Key/value lines of a committed ncu summary of the step kernel, if it
    was taken from the current kernel source; else {}."""
    try:
        text = open(summary).read()
    except OSError:
        return {}
    vals = {}
    for line in text.splitlines():
        line = line.strip().lstrip("-* ")
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals if vals.get("kernel_source_sha256_16") == kernel_source_hash() else {}


def profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    (None if absent or taken from other kernel code)."""
    try:
        return float(profile_values()["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def profiled_warp_instructions():
    """Warp instructions per launch of the step kernel (ncu smsp__inst_executed)."""
    try:
        return float(profile_values()["smsp__inst_executed"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


def algorithmic_fp64_flops_per_cell():
    """The method's flops per coupled cell update: the distinct operations of
    one step of the FP64 oracle (oracle/count_flops.py wrote this number)."""
    try:
        with open(os.path.join(ROOT, "oracle", "flops_per_cell.json")) as fh:
            return float(json.load(fh)["coupled"]["distinct_flops_per_cell"])
    except (OSError, ValueError, KeyError):
        return None


def profiled_fp64_flops_per_cell():
    """Executed FP64 flops per cell update of the FP64 step kernel (ncu: DFMA
    counted twice, DADD and DMUL once)."""
    try:
        return float(profile_values(PROFILE_SUMMARY_FP64)["fp64_flops_per_cell"].split()[0])
    except (KeyError, ValueError, IndexError):
        return None


# ------------------------------------------------------------------ GPU arm

def time_steps(solver, stream, steps):
    import torch

    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    solver.step(steps)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


REPEATS = 5   # timed windows of K steps each; the reported time is their median


def run_gpu_measure(precision, steps, warmup, world, rank, recon="central", repeats=REPEATS, clock=None):
    """W untimed steps, then `repeats` windows of exactly K steps, each
    bracketed by a barrier and a synchronize and timed with CUDA events on
    the solver's stream (the slowest rank's time per window).  Returns the
    median window time and the per-window times."""
    import torch
    import torch.distributed as dist

    from paper_1810_07802_gb300 import solver as S

    cfg, f = workload(precision=precision)
    cfg["recon"] = recon
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = S.Solver(cfg, stream=stream, **f)
    s.step(warmup)
    s.sync()
    mass0 = s.reduce()[0]   # FP64 phi mass on the GPU (outside the timed region)
    windows = []
    for _ in range(repeats):
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clock is not None:
            clock.record(True)
        secs = time_steps(s, stream, steps)
        if clock is not None:
            clock.record(False)
        secs, _ = job_time_and_value(secs, 1, world)
        windows.append(secs)
    s.sync()   # raises if the device status word reports a non-finite or non-physical step
    mass1, resid_phi, resid_u, umax = s.reduce()
    s.close()
    cfg["_health"] = {"phi_mass_rel_drift": (mass1 - mass0) / mass0, "resid_phi": resid_phi, "resid_u": resid_u,
                      "umax": umax, "steps": steps * repeats}
    cfg["_windows_s"] = windows
    return statistics.median(windows), cfg


def run_e2e(steps, f_host=None):
    """Same metric through the public API with host buffers: dugks_create from
    pinned host fields (H2D), K steps, dugks_macros into pinned host arrays
    (D2H), all inside the timed region."""
    import numpy as np
    import torch

    from paper_1810_07802_gb300 import solver as S

    cfg, f = workload(precision="fp32")
    n = cfg["nx"] * cfg["ny"]
    pinned = {k: torch.empty((cfg["ny"], cfg["nx"]), dtype=torch.float64, pin_memory=True) for k in ("phi0",)}
    pinned["phi0"].numpy()[:] = f["phi0"]
    ws = torch.empty(S.workspace_bytes(cfg) + 256, dtype=torch.uint8, device="cuda")
    base = (ws.data_ptr() + 255) // 256 * 256
    ws_view = ws[base - ws.data_ptr():]
    stream = torch.cuda.Stream()
    outs = [torch.empty((cfg["ny"], cfg["nx"]), dtype=torch.float64, pin_memory=True) for _ in range(4)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = S.Solver(cfg, phi0=pinned["phi0"].numpy(), workspace=ws_view, stream=stream)
    s.step(steps)
    L = S.lib()
    ptrs = [o.numpy().ctypes.data_as(S._dp) for o in outs]
    code = L.dugks_macros(s.h, *ptrs, 0)
    t1 = time.perf_counter()
    s.close()
    if code != 0:
        raise S.DugksError(code, "dugks_macros")
    assert np.isfinite(outs[0].numpy()).all()
    mlups = n * steps / (t1 - t0) / 1e6
    h2d = n * 8 * 1          # phi0 (ux0, uy0, p0 are zero and not sent)
    d2h = n * 8 * 4          # phi, p, ux, uy
    return {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "steps": steps, "region": "dugks_create(host phi0) + dugks_step(K) + dugks_macros(host)"}


def run_serving(n=100, rate=50.0):
    """The serving mix (Poiseuille / bubble / spinodal requests, Poisson
    arrivals): continuous batching (FP32-shifted) against one solve at a time
    (FP32 and FP64), and the same requests as one burst."""
    import numpy as np

    from paper_1810_07802_gb300 import workloads as W
    from paper_1810_07802_gb300.serve import AutotuneCache, BatchingServer, Request, SequentialServer, summary

    def requests(precision, burst):
        tr = W.serving_trace(n=n, rate=rate, precision=precision, burst=burst)
        return [Request(i, k, c, f, st, t) for i, (k, c, f, st, t) in enumerate(tr)]

    def keep(d):
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in d.items()}

    budget = 64 << 30
    # untimed warm-up over the whole mix: the first burst served in a process
    # runs about 5 % slower than later ones, whatever the policy
    warm = requests("fp32", True)
    BatchingServer(budget, keep_results=False).run(warm)
    SequentialServer(keep_results=False).run(warm[:6])
    out = {"workload": "%d requests: layered Poiseuille (Ny 64-512, Nx 4, 400 steps), stationary bubbles "
                       "(N 64-512, ratio 10/100/1000, 100 steps), spinodal boxes (N 128-1024, 200 steps)" % n,
           "hbm_budget_bytes": budget}
    tuner = AutotuneCache(trial_steps=10)   # shapes are tuned before a run's clock starts
    t_tune = 0.0
    for label, burst in (("poisson_%g_per_s" % rate, False), ("burst", True)):
        r32, r64 = requests("fp32", burst), requests("fp64", burst)
        out[label] = {"batched_fp32": keep(summary(BatchingServer(budget, max_members=128, chunk=50,
                                                                  keep_results=False).run(r32))),
                      "sequential_fp32": keep(summary(SequentialServer(keep_results=False).run(r32))),
                      "sequential_fp64": keep(summary(SequentialServer(keep_results=False).run(r64)))}
        t0 = time.perf_counter()
        for r in requests("fp32", burst):
            tuner(r.cfg, r.fields)
        t_tune += time.perf_counter() - t0
        out[label]["batched_fp32_autotuned"] = keep(summary(BatchingServer(
            budget, max_members=128, chunk=50, keep_results=False, tile_policy=tuner).run(requests("fp32", burst))))
        out[label]["batched_fp32_persistent"] = keep(summary(BatchingServer(
            budget, max_members=128, chunk=50, keep_results=False, persistent=True).run(requests("fp32", burst))))
    # accuracy of the FP32 batched results against FP64 solves of the same requests (untimed sample)
    sample32 = requests("fp32", True)[:12]
    sample64 = requests("fp64", True)[:12]
    r32 = BatchingServer(budget, max_members=128, chunk=50).run(sample32)
    r64 = SequentialServer().run(sample64)
    worst = {}
    for a, b, q in zip(r32, r64, sample32):
        p32, p64 = a.result["phi"], b.result["phi"]
        l2 = float(np.sqrt(((p32 - p64) ** 2).sum() / (p64 ** 2).sum()))
        worst[q.kind] = max(worst.get(q.kind, 0.0), l2)
    out["fp32_vs_fp64"] = {"requests": len(sample32), "phi_l2_rel_max_by_kind": worst, "budget_phi_l2": 1e-4}
    chosen = {}
    for k, v in tuner.shapes.items():
        chosen["%s %dx%d" % (k[1], k[3], k[4])] = v
    out["autotune"] = {"shapes_tuned": len(tuner.shapes), "tuning_s": round(t_tune, 3), "tile_shape": chosen}
    return out


def cpu_baseline_sample(rows=REF_BAND_ROWS, steps=2):
    """The FP64 oracle, as it stands, on a 2048 x rows band of the workload."""
    from oracle.oracle import Oracle

    cfg, f = workload(ny=rows, precision="fp64")
    o = Oracle(cfg, **f)
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return N_CELLS_SIDE * rows * steps / dt / 1e6, dt, cfg


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_band_worker(band, rows, cmd_q, res_q, barrier):
    """One spawned process: the FP64 oracle on rows [band*rows, (band+1)*rows)
    of the workload, made periodic in y; steps on command, timed after a
    barrier shared with the other processes."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle.oracle import Oracle

    cfg, f = workload(precision="fp64")
    r0 = (band * rows) % N_CELLS_SIDE
    f = {k: (None if v is None else v[r0:r0 + rows, :].copy()) for k, v in f.items()}
    cfg.update(ny=rows)
    o = Oracle(cfg, **f)
    res_q.put((band, 0.0))
    while True:
        n = cmd_q.get()
        if n is None:
            break
        barrier.wait(timeout=900)
        t0 = time.perf_counter()
        o.step(n)
        res_q.put((band, time.perf_counter() - t0))


class OraclePool:
    """`procs` spawn-started processes, each stepping the unchanged FP64 oracle
    on its own 2048 x rows band of the workload, all started together by a
    barrier: the oracle's throughput on that many host cores.  Spawned, not
    forked, so it is safe after CUDA has been initialised."""

    def __init__(self, procs, rows):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.procs, self.rows = procs, rows
        self.barrier = ctx.Barrier(procs)
        self.res_q = ctx.Queue()
        self.cmd_qs = [ctx.Queue() for _ in range(procs)]
        self.ps = [ctx.Process(target=_oracle_band_worker, args=(b, rows, self.cmd_qs[b], self.res_q, self.barrier),
                               daemon=True) for b in range(procs)]
        for p in self.ps:
            p.start()
        for _ in range(procs):
            self.res_q.get(timeout=900)

    def step(self, n=1):
        """n oracle steps on every band; returns (cell updates, seconds of the slowest process)."""
        for q in self.cmd_qs:
            q.put(n)
        dts = [self.res_q.get(timeout=900)[1] for _ in range(self.procs)]
        return N_CELLS_SIDE * self.rows * n * self.procs, max(dts)

    def close(self):
        for q in self.cmd_qs:
            q.put(None)
        for p in self.ps:
            p.join(60)
            if p.is_alive():
                p.terminate()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def cpu_baseline_all_cores(rows=64, steps=10):
    """The oracle on every host core: one band per process (see OraclePool)."""
    cores = host_cores()
    with OraclePool(cores, rows) as pool:
        pool.step(1)                       # warm-up
        cells, dt = pool.step(steps)
    return cells / dt / 1e6, dt, cores


def ours(args):
    import torch

    rank, world, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1810_07802_gb300 import build, solver

    if not os.path.exists(build.LIB_PATH):
        build.build()
    solver.lib()
    dev_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if world == 1 else local

    with NvmlSampler(dev_index) as clk:
        secs, cfg = run_gpu_measure("fp32", args.steps, args.warmup, world, rank, clock=clk)
    clocks = clk.summary()
    cells = cfg["nx"] * cfg["ny"]
    value = cells * args.steps * world / secs / 1e6   # secs: the slowest rank's
    ms_step = secs / args.steps * 1e3

    peaks = measured_peaks()
    peak_gbs, peak_src = (peaks["hbm_gbs"], "measured") if peaks else (6800.0, "fallback")
    achieved = FP32_BYTES_PER_CELL * cells / (secs / args.steps) / 1e9
    traffic = profiled_traffic()
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak_gbs, "unit": "GB/s",
                "frac": round(achieved / peak_gbs, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": FP32_BYTES_PER_CELL * cells,
                "peak_source": peak_src, "kernel": "solo_step_kernel<float,32,8,coupled,periodic>"}

    extra = {}
    # second bound: instruction issue (4 schedulers per SM, one warp instruction per cycle each)
    winst = profiled_warp_instructions()
    if winst is not None:
        import torch

        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
        peak_issue = sms * 4 * mhz * 1e6
        ach_issue = winst / (secs / args.steps)
        extra["issue_roofline"] = {"bound": "issue", "achieved": round(ach_issue / 1e9, 1),
                                   "peak": round(peak_issue / 1e9, 1), "unit": "Gwarp-instr/s",
                                   "frac": round(ach_issue / peak_issue, 4),
                                   "warp_instructions_per_launch": winst,
                                   "peak_source": "%d SMs x 4 schedulers x %g MHz (sampled SM clock)" % (sms, mhz)}
    if not args.no_fp64:
        k64 = max(3, min(args.steps, 40))
        with NvmlSampler(dev_index) as clk64:
            secs64, _c64 = run_gpu_measure("fp64", k64, 3, world, rank, clock=clk64)
        ach64 = FP64_BYTES_PER_CELL * cells / (secs64 / k64) / 1e9
        extra["fp64"] = {"value": round(cells * k64 / secs64 / 1e6 * world, 1), "unit": "MLUPS", "steps": k64,
                         "ms_per_step": round(secs64 / k64 * 1e3, 4), "hbm_gbs": round(ach64, 1),
                         "hbm_frac": round(ach64 / peak_gbs, 4), "bound": "fp64 alu",
                         "window_ms": [round(w * 1e3, 4) for w in _c64["_windows_s"]],
                         "clocks": clk64.summary()}
        fpc = algorithmic_fp64_flops_per_cell()
        executed = profiled_fp64_flops_per_cell()
        if fpc is not None:
            import torch

            sms = torch.cuda.get_device_properties(0).multi_processor_count
            c64 = extra["fp64"]["clocks"]
            mhz = c64.get("sm_mhz") or c64.get("sm_max_mhz") or 2070.0
            peak64 = sms * 2 * 2 * mhz * 1e6          # 2 DFMA per cycle per SM, 2 flops each
            ach = fpc * cells / (secs64 / k64)
            extra["fp64"]["roofline"] = {"bound": "alu", "achieved": round(ach / 1e9, 1),
                                         "peak": round(peak64 / 1e9, 1), "unit": "GFLOP/s",
                                         "frac": round(ach / peak64, 4), "flops_per_cell": fpc,
                                         "flops_source": "distinct operations of one FP64 oracle step per cell "
                                                         "(oracle/count_flops.py)",
                                         "executed_flops_per_cell": executed,
                                         "executed_over_algorithmic": (round(executed / fpc, 4)
                                                                       if executed is not None else None),
                                         "peak_source": "%d SMs x 2 DFMA/cycle x 2 flops x %g MHz (sampled SM "
                                                        "clock)" % (sms, mhz)}
    if not args.no_upwind:
        # the upwind reconstruction (van Leer slopes) on the same workload, FP32-shifted
        ku = max(3, min(args.steps, 200))
        with NvmlSampler(dev_index) as clku:
            secsu, _cu = run_gpu_measure("fp32", ku, 3, world, rank, recon="upwind", clock=clku)
        achu = FP32_BYTES_PER_CELL * cells / (secsu / ku) / 1e9
        extra["upwind_fp32"] = {"value": round(cells * ku / secsu / 1e6 * world, 1), "unit": "MLUPS", "steps": ku,
                                "ms_per_step": round(secsu / ku * 1e3, 5), "hbm_gbs": round(achu, 1),
                                "hbm_frac": round(achu / peak_gbs, 4),
                                "kernel": "solo_step_kernel<float,32,8,coupled,periodic,upwind>",
                                "clocks": clku.summary()}

    line = {"metric": "coupled DUGKS MLUPS (spinodal 2048^2, FP32-shifted)", "value": round(value, 1),
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded SplitMix64 spinodal field)",
            "config": dict(config_dict("fp32"), parallelism="replicas" if world > 1 else "single GPU"),
            "health": cfg.get("_health"),
            "timing": {"windows": REPEATS, "steps_per_window": args.steps, "statistic": "median",
                       "window_ms": [round(w * 1e3, 4) for w in cfg["_windows_s"]],
                       "ms_x_median_sm_mhz_per_step": (round(ms_step * clocks["sm_mhz"], 1)
                                                       if clocks.get("sm_mhz") else None)},
            "roofline": roofline, "clocks": clocks, "gpu_launches": args.steps}
    if rank == 0:
        line["e2e"] = run_e2e(args.steps)
        if args.steps < 400:
            # the same path at a step count where create and read-back are amortised
            line["e2e"]["steady_state"] = run_e2e(400)
        if not args.no_serving:
            line["serving"] = run_serving()
        if not args.no_cpu_baseline:
            rows, nst = 64, 10
            v, dt, cores = cpu_baseline_all_cores(rows=rows, steps=nst)
            rows1, nst1 = 512, 4
            v1, dt1, _ = cpu_baseline_sample(rows=rows1, steps=nst1)
            line["cpu_baseline"] = {"value": round(v, 3), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                                    "sample": "%d FP64 steps of %d periodic 2048x%d bands of the same seeded field, "
                                              "one single-threaded C oracle process per host core, started together "
                                              "(%.1f s wall, slowest process)" % (nst, cores, rows, dt),
                                    "single_core": {"value": round(v1, 3), "unit": "MLUPS", "cores": 1,
                                                    "sample": "%d FP64 steps of a 2048x%d periodic band (%.1f s)"
                                                              % (nst1, rows1, dt1)}}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


def reference(args):
    rank, world, _ = dist_setup(args)
    if rank != 0:
        return
    cores = host_cores()
    rows = REF_BAND_ROWS // 4
    total_cells = 0
    t_total = 0.0
    with OraclePool(cores, rows) as pool:
        for _ in range(args.warmup):
            pool.step(1)
        for _ in range(args.steps):
            cells, dt = pool.step(1)
            total_cells += cells
            t_total += dt
    value = total_cells / t_total / 1e6
    line = {"metric": "coupled DUGKS MLUPS (spinodal 2048^2, FP32-shifted)", "value": round(value, 4),
            "unit": "MLUPS", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(t_total / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SplitMix64 spinodal field)",
            "config": config_dict("fp64"), "impl": "reference",
            "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": "each step: 1 FP64 step of each of %d periodic 2048x%d bands of the workload, "
                                       "one single-threaded C oracle process per host core, started together; "
                                       "step time = the slowest process" % (cores, rows)},
            "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        reference(a)
    else:
        ours(a)
