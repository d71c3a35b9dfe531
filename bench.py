"""Benchmark of the spectral flame step on GB300.

Workload (the large memory-bound configuration): one flame on a 4096 x 8192
(theta, phi) grid, FP32 FFTs and pointwise work with the FP64 mean mode and
time, seeded spectrum |k| <= 256 of amplitude 1e-3 (1+|k|)^-2, gamma = 0.8,
t0 = 200, dt = 1e-3.  A "step" is one explicit Euler step of the model
(passes A, B, C: the whole hot path).  Metric: grid-point updates per second
(N1 N2 per step) and the HBM roofline of the dominant pass.

--impl ours (default): the CUDA library through its C ABI.
--impl reference: the FP64 CPU oracle on the host cores, on a bounded
  sample of the same workload.

Multi-GPU: every rank steps its own independent flame (replicas, no
collective on the data path); value = all ranks' updates / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="flame-step-4096x8192-fp32mixed", n1=4096, n2=8192, prec="fp32", kmax=256,
                seed=0, gamma=0.8, t0=200.0, dt=1e-3)
L2_BYTES = 129 * 1024 * 1024


def workload_config(world):
    """The `config` object of the JSON line, the same for both arms."""
    w = WORKLOAD
    return {"workload": w["workload"], "grid": [w["n1"], w["n2"]], "kmax": w["kmax"],
            "l2": "inputs larger than L2: each step streams its 235 MB working set (state 33.5 MB, "
                  "uv 134 MB, gk 67 MB) through the 129 MB L2; flushed once before the timed steps",
            "parallelism": f"replicas{world}"}
FLUSH_BYTES = 512 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


PASS_NAMES = ("A", "B", "C", "CA")


def pass_bytes(n1, n2, K1, K2, esz):
    """Algorithmic HBM bytes of passes A, B, C and of the fused CA (pass C
    followed by the next step's pass A, which then reads no state): each
    array read or written once."""
    box = (2 * K1 + 1) * (K2 + 1) * esz
    col = n1 * (K2 + 1) * esz
    return [box + 2 * col, 2 * col + col, col + 2 * box, col + 2 * box + 2 * col]


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled through NVML every
    ~0.2 ms while the timed region runs.  The device is found by its UUID,
    so CUDA_VISIBLE_DEVICES renumbering does not matter.  Reads only: no
    setting of the GPU is changed."""

    # clock-event reason bits of NVML's public header
    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, device_index):
        self.samples, self.max_mhz, self.error = [], None, None
        self._stop = threading.Event()
        self._thread = None
        try:
            import ctypes
            import torch
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            uuid = getattr(torch.cuda.get_device_properties(device_index), "uuid", None)
            if uuid is None:
                raise RuntimeError("device UUID not exposed")
            self._h = ctypes.c_void_p()
            if nv.nvmlDeviceGetHandleByUUID(f"GPU-{uuid}".encode(), ctypes.byref(self._h)) != 0:
                raise RuntimeError("no NVML handle for the device")
            mx = ctypes.c_uint()
            if nv.nvmlDeviceGetMaxClockInfo(self._h, 1, ctypes.byref(mx)) == 0:  # 1 = SM clock
                self.max_mhz = float(mx.value)
            self._nv, self._ct = nv, ctypes
            self._reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                nv.nvmlDeviceGetCurrentClocksThrottleReasons
        except Exception as e:  # noqa: BLE001 - reported in the summary
            self._nv, self.error = None, f"{type(e).__name__}: {e}"

    def _poll(self):
        ct, nv = self._ct, self._nv
        clk, rs = ct.c_uint(), ct.c_ulonglong()
        while not self._stop.is_set():
            if nv.nvmlDeviceGetClockInfo(self._h, 1, ct.byref(clk)) == 0 and \
                    self._reasons(self._h, ct.byref(rs)) == 0:
                self.samples.append((float(clk.value), int(rs.value)))
            time.sleep(0.0002)

    def start(self):
        if self._nv is not None:
            self._thread = threading.Thread(target=self._poll, daemon=True)
            self._thread.start()
        return self

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join()

    def summary(self):
        """Median SM clock over the samples of the timed region and every
        clock-event reason seen active in them."""
        if not self.samples:
            why = self.error or "no samples in the timed region"
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [why], "samples": 0}
        seen = set()
        for _, bits in self.samples:
            seen.update(n for b, n in self.REASONS.items() if bits & b)
        return {"sm_mhz": statistics.median(c for c, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(seen), "samples": len(self.samples), "source": "nvml"}


def cpu_oracle_step_time(w, nsteps=1):
    """Seconds per oracle step (FP64 C oracle, OpenMP over rows/columns) on
    the full workload grid; returns (seconds per step, threads)."""
    from oracle import oracle
    from paper_0911_2889_gb300 import inputs
    oracle.build()
    p = oracle.Params(w["n1"], w["n2"], gamma=w["gamma"], t0=w["t0"], dt=w["dt"])
    st = inputs.spectrum_ic(w["n1"], w["n2"], w["kmax"], w["seed"])
    t0 = time.perf_counter()
    oracle.step(p, st, 0.0, w["t0"], nsteps)
    dt = (time.perf_counter() - t0) / nsteps
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dt, threads


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    pts = w["n1"] * w["n2"]
    for _ in range(args.warmup):
        cpu_oracle_step_time(w)
    times = []
    threads = 1
    for _ in range(args.steps):
        dt, threads = cpu_oracle_step_time(w)
        times.append(dt)
    sec = sum(times) / len(times)
    v = pts / sec
    line = {
        "impl": "reference", "metric": "grid_point_updates_per_s", "value": v, "unit": "points/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.gpus),
        "cpu_baseline": {"value": v, "unit": "points/s", "cores": threads, "kind": "oracle",
                         "sample": "one full FP64 oracle step of the 4096x8192 workload per timed step"},
        "e2e": {"value": v, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reduce_max(x, device="cpu"):
    """Max of a per-rank float over all ranks (identity without a process
    group); the device follows the backend (cuda for nccl, cpu for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, steps, world, max_ms):
    """Grid-point updates per second of all ranks together (replicas: every
    rank steps its own flame), timed by the slowest rank."""
    return points_per_rank * steps * world / (max_ms * 1e-3)


def _ev_time(fn, stream, reps=1):
    """Device time (ms) of fn() on `stream`, averaged over reps."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_batched(flame, inputs, nflames=256, steps=500, plain_steps=20):
    """Ensemble of uneven FP32 flames (grids uniform over 256x512, 512x1024,
    1024x2048, size seed 1234, spectrum seeds 1000+i), `steps` steps in one
    flame_step_batch call (grouped launches, replayed 8-step graphs), against
    the same flames stepped one by one (plain_steps steps each, graph-captured
    flame_step calls).  Effective GB/s counts the 3-pass algorithmic bytes of
    every flame's steps."""
    import torch
    grids = inputs.batch_grids(nflames)
    fl, ss, ms, ts = [], [], [], []
    for i, (n1, n2) in enumerate(grids):
        f = flame.Flame(n1, n2, prec="fp32", gamma=0.8, t0=200.0, dt=1e-3)
        st = inputs.spectrum_ic(n1, n2, inputs.batch_kmax(n1), 1000 + i, K1=f.K1, K2=f.K2)
        fl.append(f)
        ss.append(torch.from_numpy(flame.box_to_abi(st)).cuda().to(f.cdtype))
        ms.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
        ts.append(torch.full((1,), 200.0, dtype=torch.float64, device="cuda"))
    hs = [f.h for f in fl]
    s = torch.cuda.current_stream()
    flame.flame_step_batch(hs, ss, ms, ts, nsteps=steps)  # capture + warm-up
    torch.cuda.synchronize()
    t_batch = _ev_time(lambda: flame.flame_step_batch(hs, ss, ms, ts, nsteps=steps), s)
    for f, st, m, t in zip(fl, ss, ms, ts):
        f.step(st, m, t, plain_steps)  # capture each flame's graph
    torch.cuda.synchronize()
    t_plain = _ev_time(lambda: [f.step(st, m, t, plain_steps) for f, st, m, t in zip(fl, ss, ms, ts)], s)
    for f in fl:
        f.sync_status()
    pts_step = sum(n1 * n2 for n1, n2 in grids)
    bytes_step = sum(sum(pass_bytes(n1, n2, f.K1, f.K2, 8)) for (n1, n2), f in zip(grids, fl))
    for f in fl:
        f.close()
    rate = pts_step * steps / (t_batch * 1e-3)
    plain = pts_step * plain_steps / (t_plain * 1e-3)
    peak, kind = _peaks()
    gbs = bytes_step * steps / (t_batch * 1e-3) / 1e9
    return {"workload": f"ensemble-{nflames}-uneven-fp32mixed", "steps": steps,
            "value": rate, "unit": "points/s", "plain_value": plain, "plain_steps": plain_steps,
            "vs_plain": rate / plain, "ms_per_step": t_batch / steps,
            "effective_gbs": gbs, "frac_of_hbm": gbs / peak, "peak_kind": kind}


def passB_model_flops(n1, n2):
    """Model flops of one pass B launch (the row pass): per row, two
    half-length inverse complex FFTs (even and odd grid points) and one
    forward, 5 M log2 M each (M = N2/2), the odd points' pre-twiddle (6 M),
    g = u^2 + v^2 (3 per grid point: 6 M) and the real post-processing
    (10 per kept output, about 5 M)."""
    import math
    m = n2 // 2
    return n1 * (15.0 * m * math.log2(m) + 17.0 * m)


def step_model_flops(n1, n2):
    """Model flops of one step per grid point: three real 2-D transforms
    (two inverse, one forward) at 2.5 N log2 N each (N = N1 N2) and about 5
    pointwise flops (the product, the linear operator and the update)."""
    import math
    return 7.5 * math.log2(n1 * n2) + 5.0


def measure_trajectory(flame, inputs, n1, n2, prec, kmax, nsteps, fp64_peak=None):
    """A graph-captured nsteps-step flame_step call on one flame (seed 0,
    gamma 0.8, t0 200, dt 1e-3): grid-point updates per second; FP64 also
    against the measured FP64 FMA rate (model flops of step_model_flops)."""
    import torch
    s = torch.cuda.current_stream()
    f = flame.Flame(n1, n2, prec=prec, gamma=0.8, t0=200.0, dt=1e-3)
    st = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(n1, n2, kmax, 0, K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
    f.step(st, m, t, nsteps)  # capture the graphs
    torch.cuda.synchronize()
    ms = min(_ev_time(lambda: f.step(st, m, t, nsteps), s) for _ in range(3))
    f.sync_status()
    esz = 16 if prec == "fp64" else 8
    bytes_step = sum(pass_bytes(n1, n2, f.K1, f.K2, esz)[:3])
    f.close()
    out = {"workload": f"trajectory-{n1}x{n2}-{prec}-{nsteps}steps", "steps": nsteps,
           "value": n1 * n2 * nsteps / (ms * 1e-3), "unit": "points/s", "ms_per_step": ms / nsteps,
           "effective_gbs": bytes_step / (ms * 1e-3 / nsteps) / 1e9,
           "note": "graph-captured steps; the working set is L2-resident"}
    if prec == "fp64" and fp64_peak:
        fl_rate = step_model_flops(n1, n2) * n1 * n2 / (ms * 1e-3 / nsteps)
        out.update({"model_flops_per_point": step_model_flops(n1, n2), "achieved_gflops": fl_rate / 1e9,
                    "fp64_peak_gflops": fp64_peak / 1e9, "peak_kind": "measured (flame_fma_peak)",
                    "frac_of_fp64_peak": fl_rate / fp64_peak})
    return out


def measure_adjoint(flame, inputs, nsteps=200, ckpt=20, reps=2):
    """Gradient of the final area over nsteps FP32 steps on 512x1024 (|k| <= 64,
    seed 7), checkpoints every ckpt steps, against plain forward stepping."""
    import torch
    n1, n2 = 512, 1024
    f = flame.Flame(n1, n2, prec="fp32", gamma=0.8, t0=200.0, dt=1e-3)
    st0 = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(n1, n2, 64, 7, K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
    m0 = torch.zeros(1, dtype=torch.float64, device="cuda")
    t0 = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream()
    sT, mT, tT = st0.clone(), m0.clone(), t0.clone()
    f.step(sT, mT, tT, nsteps)
    _, lam, lam0 = f.area(sT, mT, tT, grad=True)
    f.adjoint(st0, m0, t0, nsteps, ckpt, lam, lam0)  # warm-up (allocates the checkpoint arena)
    torch.cuda.synchronize()
    t_adj = _ev_time(lambda: f.adjoint(st0, m0, t0, nsteps, ckpt, lam, lam0), s, reps)
    x, m, t = st0.clone(), m0.clone(), t0.clone()
    t_fwd = _ev_time(lambda: f.step(x, m, t, nsteps), s, reps)
    f.sync_status()
    f.close()
    pts = n1 * n2 * nsteps
    return {"workload": "adjoint-512x1024-200steps-ckpt20-fp32mixed", "value": pts / (t_adj * 1e-3),
            "unit": "points/s", "plain_value": pts / (t_fwd * 1e-3), "vs_plain": t_fwd / t_adj,
            "ms": t_adj, "note": "working set fits in L2"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_0911_2889_gb300 import flame, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = WORKLOAD
    n1, n2 = w["n1"], w["n2"]
    f = flame.Flame(n1, n2, gamma=w["gamma"], t0=w["t0"], dt=w["dt"], prec=w["prec"])
    st0 = inputs.spectrum_ic(n1, n2, w["kmax"], w["seed"] + rank, K1=f.K1, K2=f.K2)
    state = torch.from_numpy(flame.box_to_abi(st0)).cuda().to(f.cdtype)
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), w["t0"], dtype=torch.float64, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    esz = 8 if w["prec"] == "fp32" else 16
    pbytes = pass_bytes(n1, n2, f.K1, f.K2, esz)

    # Steps run back to back, pass by pass, exactly as flame_step enqueues
    # them: A, then (B, CA) for every step but the last and B, C for the last
    # when the column passes are fused (CA = pass C fused with the next
    # step's pass A), else A, B, C per step.  One event before every launch.
    fused = flame.flame_fused_steps(f.h)

    def sequence(nsteps):
        if fused:
            return [0] + [p for k in range(nsteps) for p in ((1, 3) if k + 1 < nsteps else (1, 2))]
        return [p for _ in range(nsteps) for p in (0, 1, 2)]

    def run_steps(nsteps, ev=None):
        seq = sequence(nsteps)
        for i, ps in enumerate(seq):
            if ev is not None:
                ev[i].record(stream)
            flame.flame_step_pass(f.h, ps, state, mean, t, stream)
        if ev is not None:
            ev[len(seq)].record(stream)
        return seq

    # The timed region: one flame_step(K) call, the call a user makes (K
    # steps as one captured CUDA graph; consecutive passes are programmatic
    # dependent launches), bracketed by events on the launching stream.
    f.step(state, mean, t, args.warmup, stream)  # warm-up (and graph capture of W steps)
    f.step(state, mean, t, args.steps, stream)   # capture the graph of K steps
    f.sync_status()
    torch.cuda.synchronize()
    t_a = torch.cuda.Event(enable_timing=True)
    t_b = torch.cuda.Event(enable_timing=True)
    flush.zero_()  # L2 starts cold; the steps then stream their working set (> L2) back to back
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    wall0 = time.perf_counter()
    t_a.record(stream)
    f.step(state, mean, t, args.steps, stream)
    t_b.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk.stop()
    total_ms = reduce_max(t_a.elapsed_time(t_b), device="cuda")
    # Per-kernel durations for the roofline: the same steps launched pass by
    # pass as flame_step enqueues them, one event before every launch.
    run_steps(args.warmup)
    seq = sequence(args.steps)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(seq) + 1)]
    flush.zero_()
    torch.cuda.synchronize()
    run_steps(args.steps, evs)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    f.sync_status()
    launch_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(len(seq))]
    passwise_ms = evs[0].elapsed_time(evs[-1])
    kinds = sorted(set(seq))
    kind_ms = {ps: [ms for ms, q in zip(launch_ms, seq) if q == ps] for ps in kinds}
    avg = {ps: sum(v) / len(v) for ps, v in kind_ms.items()}
    share = {ps: sum(v) for ps, v in kind_ms.items()}
    dom = max(kinds, key=lambda ps: share[ps])  # the kernel with the largest share of the timed region
    pts = n1 * n2
    value = whole_job_rate(pts, args.steps, world, total_ms)
    peak, peak_kind = _peaks()
    achieved = pbytes[dom] / (avg[dom] * 1e-3) / 1e9
    step_bytes = sum(pbytes[q] for q in seq) / args.steps

    # end to end through the public API with host buffers (pinned): one
    # flame_step_host call per step, its copies of the state, mean mode and
    # time in and out inside the timed region (the library overlaps them
    # with the step's first and last column passes)
    hs = state.cpu().pin_memory()
    hm = mean.cpu().pin_memory()
    ht = t.cpu().pin_memory()
    f.step_host(hs, hm, ht, 1, stream)  # first call: the handle's device copy and copy stream
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        e0.record(stream)
        f.step_host(hs, hm, ht, 1, stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        nk = k + 1
    e2e_value = pts * nk / (e2e_ms * 1e-3) * world
    io_bytes = state.numel() * state.element_size() + 16

    # DRAM bytes per launch of the dominant kernel from an ncu capture,
    # valid only for the kernel sources it was taken on
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            entry = json.load(open(prof)).get(f"{w['workload']}:pass{PASS_NAMES[dom]}")
            if entry and entry.get("step_sources_sha256") == kernel_sources_sha256():
                traffic = entry["dram_bytes_per_launch"]
        except (OSError, ValueError, KeyError):
            traffic = None

    batched = adjoint = traj64 = traj32 = None
    fp64_peak = None
    # the dominant pass against the FP32 FMA rate it is bound by on chip (the
    # HBM line above is the required roofline; this one says what binds it)
    roof_alu = None
    if PASS_NAMES[dom] == "B":
        fp32_peak = flame.flame_fma_peak("fp32")
        ach = passB_model_flops(n1, n2) / (avg[dom] * 1e-3) / 1e12
        roof_alu = {"bound": "alu", "kernel": "passB", "achieved": ach, "peak": fp32_peak / 1e12,
                    "peak_kind": "measured (flame_fma_peak, scalar FP32 FMA)", "unit": "TFLOP/s",
                    "frac": ach / (fp32_peak / 1e12), "model_flops": passB_model_flops(n1, n2)}
    if not args.no_extras:
        batched = measure_batched(flame, inputs)
        adjoint = measure_adjoint(flame, inputs)
        fp64_peak = flame.flame_fma_peak("fp64")
        traj64 = measure_trajectory(flame, inputs, 128, 256, "fp64", 16, 100, fp64_peak)
        traj32 = measure_trajectory(flame, inputs, 1024, 2048, "fp32", 256, 1000)

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            sec, threads = cpu_oracle_step_time(w)
            cpu = {"value": pts / sec, "unit": "points/s", "cores": threads, "kind": "oracle",
                   "sample": "one FP64 oracle step of the same 4096x8192 workload"}
        line = {
            "metric": "grid_point_updates_per_s", "value": value, "unit": "points/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(world),
            "fused_column_passes": fused,
            "roofline": {"bound": "hbm", "kernel": f"pass{PASS_NAMES[dom]}", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "alg_bytes": pbytes[dom], "avg_ms": avg[dom]},
            "roofline_alu": roof_alu,
            "passes_ms": {PASS_NAMES[ps]: avg[ps] for ps in kinds},
            "passwise_ms_per_step": passwise_ms / args.steps,
            "step_effective_gbs": step_bytes / (total_ms / args.steps * 1e-3) / 1e9,
            "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes},
            "gpu_launches": len(seq),
            "tuning": dict(zip(("passA", "passB"), flame.flame_tuning(f.h))),
            "clocks": clk.summary(),
            "wall_s": wall,
            "cpu_baseline": cpu,
            "batched": batched,
            "adjoint": adjoint,
            "fp64_128x256": traj64,
            "fp32_1024x2048": traj32,
        }
        print(json.dumps(line), flush=True)
    f.close()
    if world > 1:
        dist.destroy_process_group()


def run_suite(args):
    """Secondary configurations (one JSON line each): the FP64 128x256 and
    FP32 1024x2048 trajectories' step rates, the initial state from the
    paper's physical-space perturbation, and the 2-D real FFT pair sweep."""
    import torch

    from paper_0911_2889_gb300 import flame, inputs
    s = torch.cuda.current_stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peak, kind = _peaks()
    for (n1, n2, prec, kmax, nsteps) in ((128, 256, "fp64", 16, 100), (1024, 2048, "fp32", 256, 1000)):
        f = flame.Flame(n1, n2, prec=prec, gamma=0.8, t0=200.0, dt=1e-3)
        st = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(n1, n2, kmax, 0, K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
        m = torch.zeros(1, dtype=torch.float64, device="cuda")
        t = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
        f.step(st, m, t, nsteps)  # capture the graphs
        torch.cuda.synchronize()
        ms = _ev_time(lambda: f.step(st, m, t, nsteps), s)
        f.sync_status()
        esz = 16 if prec == "fp64" else 8
        gbs = sum(pass_bytes(n1, n2, f.K1, f.K2, esz)[:3]) / (ms * 1e-3 / nsteps) / 1e9  # passes A, B, C
        print(json.dumps({"suite": f"trajectory-{n1}x{n2}-{prec}", "steps": nsteps, "ms_per_step": ms / nsteps,
                          "points_per_s": n1 * n2 * nsteps / (ms * 1e-3), "effective_gbs": gbs,
                          "note": "graph-captured; L2-resident" if n1 * n2 <= 2 ** 21 else "graph-captured"}),
              flush=True)
        f.close()
    # the two-stage integrators (flame_step_heun, flame_step_if: two
    # right-hand-side evaluations per step, the stage update in pass C's
    # epilogue), graph-captured, steps back to back
    for name in ("heun", "if"):
        f = flame.Flame(4096, 8192, prec="fp32", gamma=0.8, t0=200.0, dt=1e-3)
        st = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(4096, 8192, 256, 0, K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
        m = torch.zeros(1, dtype=torch.float64, device="cuda")
        t = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
        fn = f.step_heun if name == "heun" else f.step_if
        nh = 10
        fn(st, m, t, nh)  # capture the graph
        torch.cuda.synchronize()
        ms = _ev_time(lambda: fn(st, m, t, nh), s)
        f.sync_status()
        print(json.dumps({"suite": f"{name}-step-4096x8192-fp32", "steps": nh, "ms_per_step": ms / nh,
                          "points_per_s": 4096 * 8192 * nh / (ms * 1e-3),
                          "note": "two right-hand-side evaluations per step; graph-captured, steps back to back"}),
              flush=True)
        f.close()
    # the per-step record of the diagnostics (t, Phi_0, <Phi_t>) and with
    # the surface area (the row pass's area variant: measured 0.363 ms per
    # step against 1.181 ms with the separate area kernels), against plain
    # steps
    f = flame.Flame(4096, 8192, prec="fp32", gamma=0.8, t0=200.0, dt=1e-3)
    st = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(4096, 8192, 256, 0, K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
    m = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), 200.0, dtype=torch.float64, device="cuda")
    nr = 20
    rec = torch.zeros((nr, 4), dtype=torch.float64, device="cuda")
    for mode in ("plain", "record", "record+area"):
        f.set_record(None if mode == "plain" else rec, with_area=mode == "record+area")
        f.step(st, m, t, nr)  # capture
        torch.cuda.synchronize()
        ms = _ev_time(lambda: f.step(st, m, t, nr), s)
        print(json.dumps({"suite": f"step-4096x8192-fp32-{mode}", "steps": nr, "ms_per_step": ms / nr,
                          "points_per_s": 4096 * 8192 * nr / (ms * 1e-3)}), flush=True)
    f.set_record(None)
    f.sync_status()
    f.close()
    for (n1, n2, prec) in ((128, 256, "fp64"), (4096, 8192, "fp32")):
        # flame_state_from_field: r2c (rows, columns) into the workspace, then
        # the retained modes.  Bytes: the field read; the N1 x (N2/2+1)
        # spectrum written by the row pass, read and written by the column
        # pass and read by the box extraction (4 x its size, an upper bound);
        # the box written
        f = flame.Flame(n1, n2, prec=prec)
        x = torch.from_numpy(inputs.physical_ic(n1, n2, 0)).cuda().to(f.rdtype)
        st, m = f.state_from_field(x)
        reps, tot = 5, 0.0
        for _ in range(reps):
            flush.zero_()
            tot += _ev_time(lambda: f.state_from_field(x), s)
        ms = tot / reps
        rsz = 4 if prec == "fp32" else 8
        spec = n1 * (n2 // 2 + 1) * 2 * rsz
        alg = n1 * n2 * rsz + 4 * spec + (2 * f.K1 + 1) * (f.K2 + 1) * 2 * rsz
        print(json.dumps({"suite": f"initial-state-from-field-{n1}x{n2}-{prec}", "ms": ms, "alg_bytes": alg,
                          "effective_gbs": alg / (ms * 1e-3) / 1e9,
                          "frac_of_hbm": alg / (ms * 1e-3) / 1e9 / peak, "peak_kind": kind}), flush=True)
        f.close()
    sizes = [(256, 256), (256, 512), (512, 512), (512, 1024), (1024, 1024), (1024, 2048), (2048, 2048),
             (2048, 4096), (4096, 4096), (4096, 8192)]
    for prec in ("fp32", "fp64"):
        for n1, n2 in sizes:
            f = flame.Flame(n1, n2, prec=prec)
            x = torch.from_numpy(inputs.real_field(n1, n2, 1)).cuda().to(f.rdtype)
            X = f.fft_r2c(x)
            y = f.fft_c2r(X)
            reps, tot = 5, 0.0
            for _ in range(reps):
                flush.zero_()
                tot += _ev_time(lambda: (f.fft_r2c(x, X), f.fft_c2r(X, y)), s)
            ms = tot / reps
            rsz = 4 if prec == "fp32" else 8
            alg = 8 * rsz * n1 * n2  # 32 B/pt FP32, 64 B/pt FP64 (4 passes, each read + write)
            gbs = alg / (ms * 1e-3) / 1e9
            print(json.dumps({"suite": f"fft-pair-{n1}x{n2}-{prec}", "ms": ms, "alg_bytes": alg,
                              "effective_gbs": gbs, "frac_of_hbm": gbs / peak, "peak_kind": kind}), flush=True)
            f.close()


# The sources the FP32 step kernels (passes A, B, C and the fused CA) are
# compiled from: their bodies, the line FFTs, the launch geometry, the
# descriptors, and the translation units that instantiate them.  Host code
# (flame_api.cu) and kernels off the step (adjoint, FP64, Heun, FFT pair)
# are not in it.
STEP_SOURCES = ("fft_engine.cuh", "flame_kernels.cuh", "flame_ops.cuh", "flame_internal.h",
                "flame_f32_a.cu", "flame_f32_b.cu", "flame_f32_c.cu")


def kernel_sources_sha256():
    """Hash of the step kernels' sources (STEP_SOURCES), to tell whether an
    ncu traffic figure was taken on the kernels that run now."""
    import hashlib
    d = os.path.join(ROOT, "paper_0911_2889_gb300", "csrc")
    h = hashlib.sha256()
    for name in STEP_SOURCES:
        h.update(name.encode())
        with open(os.path.join(d, name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def run_profile(args):
    """Deterministic launch sequence for ncu: two twiddle-table launches at
    creation, then `--profile N` plain steps (passes A, B, C each), nothing else."""
    import torch

    from paper_0911_2889_gb300 import flame, inputs
    w = WORKLOAD
    n1, n2 = args.grid if args.grid else (w["n1"], w["n2"])
    f = flame.Flame(n1, n2, gamma=w["gamma"], t0=w["t0"], dt=w["dt"], prec=args.prec)
    st = torch.from_numpy(flame.box_to_abi(inputs.spectrum_ic(n1, n2, w["kmax"], w["seed"], K1=f.K1, K2=f.K2))).cuda().to(f.cdtype)
    mean = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.full((1,), w["t0"], dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for _ in range(args.profile):
        f.step(st, mean, t, 1)
    torch.cuda.synchronize()
    f.sync_status()
    print(json.dumps({"profile_steps": args.profile, "grid": [n1, n2], "prec": args.prec}))
    f.close()


def run_profile_ensemble(args):
    """The ensemble of measure_batched for ncu or a quick timing: builds the
    256 flames, runs 8 warm-up steps and then `--profile-ensemble N` steps in
    one flame_step_batch call, and prints their event time per step."""
    import torch
    from paper_0911_2889_gb300 import flame, inputs
    grids = inputs.batch_grids(256)
    fl, ss, ms, ts = [], [], [], []
    for i, (n1, n2) in enumerate(grids):
        f = flame.Flame(n1, n2, prec="fp32", gamma=0.8, t0=200.0, dt=1e-3)
        st = inputs.spectrum_ic(n1, n2, inputs.batch_kmax(n1), 1000 + i, K1=f.K1, K2=f.K2)
        fl.append(f)
        ss.append(torch.from_numpy(flame.box_to_abi(st)).cuda().to(f.cdtype))
        ms.append(torch.zeros(1, dtype=torch.float64, device="cuda"))
        ts.append(torch.full((1,), 200.0, dtype=torch.float64, device="cuda"))
    hs = [f.h for f in fl]
    s = torch.cuda.current_stream()
    flame.flame_step_batch(hs, ss, ms, ts, nsteps=8)
    torch.cuda.synchronize()
    n = args.profile_ensemble
    ms_ = _ev_time(lambda: flame.flame_step_batch(hs, ss, ms, ts, nsteps=n), s)
    for f in fl:
        f.sync_status()
        f.close()
    classes = sorted({g: grids.count(g) for g in grids}.items())
    print(json.dumps({"profile_ensemble_steps": n, "ms_per_step": ms_ / n,
                      "classes": [[list(g), c] for g, c in classes]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the ensemble and adjoint measurements")
    ap.add_argument("--suite", action="store_true", help="print one line per secondary configuration and exit")
    ap.add_argument("--profile", type=int, default=0, help="run N plain steps for ncu and exit")
    ap.add_argument("--grid", type=int, nargs=2, default=None, help="grid for --profile")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"], help="precision for --profile")
    ap.add_argument("--profile-ensemble", type=int, default=0,
                    help="run the 256-flame ensemble for N batch steps (after 8 warm-up steps) and exit")
    args = ap.parse_args()
    if args.profile_ensemble:
        run_profile_ensemble(args)
    elif args.profile:
        run_profile(args)
    elif args.suite:
        run_suite(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
