"""Benchmark: FP64 stencil throughput on one GB300 (GStencil/s = point updates per second).

Headline workload (one "step", the JSON line's `value`): the Jacobi 2D 5-point star
and 9-point box stencils on 4096 x 4096 FP64 grids, seeded uniform [0, 1) inputs,
seeded positive weights normalised to sum 1, zero Dirichlet halo, T = 1000 time
steps each, run through the library's C ABI with its default (autotuned) kernel
choice. The paper's Table 1 lists Heat-2D and 2D9P on 8000^2 x 2000; this is the
same kind of workload at a size one step of which takes well under a second.

The line's `method_configs` object times the method's other kernels on their own
workloads, each in its own clocked window and beside the plain per-step kernel on
the same grid:
  heat1d      Jacobi 1D 3-point heat, N = 65536, T = 256 (temporally blocked kernel, tuned)
  gs2d        Gauss-Seidel 2D 5-point, 4096^2, T = 200 (wavefront kernel)
  gs1d        Gauss-Seidel 1D 3-point, N = 2^24, T = 200 (wavefront kernel)
  batch512    Jacobi 3D 7-point + Jacobi 3D 27-point + Gauss-Seidel 3D 7-point, 512^3 periodic,
              T = 100, in one stencil_run_batch call (one persistent launch in a CUDA graph)
  serving     the seeded serving mix at a stated arrival rate (continuous batching)

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-extra]
    python bench.py --source-hash     (the kernel-source hashes the DRAM traffic table is keyed on)

Prints one JSON line. --impl reference times the CPU oracle (the plain
definition in C, OpenMP over the host cores) on a bounded sample of the same
workload instead. Under torchrun (N > 1) every rank runs an independent
replica (the workload has no cross-grid exchange), timed between barriers;
rank 0 reports the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
PKG = os.path.join(ROOT, "paper_2010_04868_gb300")
CSRC = os.path.join(PKG, "csrc")

N_SIDE = 4096
T_STEPS = 1000
STENCILS = (("2d5p", 0, 5), ("2d9p", 1, 9))   # name, shape id, K
KERNEL_NAMES = {1: "plain", 2: "blocked", 3: "wavefront", 4: "diamond", 5: "stream"}
# the kernel source files each plan's code comes from (hashed to key the DRAM traffic table)
PLAN_SOURCES = {"plain": ("k_plain.cu", "common.cuh"), "blocked": ("k_blocked.cu", "common.cuh"),
                "stream": ("k_stream.cu", "common.cuh"),
                "diamond": ("k_diamond.cu", "common.cuh"), "wavefront": ("k_wavefront.cu", "common.cuh"),
                "batch": ("k_batch.cu", "k_plain.cu", "common.cuh")}
FALLBACK_HBM_GBS = 6800.0   # the profiling recipe's fallback copy bandwidth, used only without a measured one


# ------------------------------------------------------------------ measured peaks and traffic

def source_hash(files):
    """First 12 hex digits of the SHA-256 of the named csrc/ files, concatenated in order."""
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def traffic_table():
    """Rows of profiles/dram_traffic.md: {(workload, plan): (source hash, DRAM bytes per launch)}."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.md")
    rows = {}
    if not os.path.exists(path):
        return rows
    for ln in open(path):
        cells = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(cells) >= 4 and re.fullmatch(r"[0-9a-f]{12}", cells[2] or "") and cells[3].replace("_", "").isdigit():
            rows[(cells[0], cells[1])] = (cells[2], int(cells[3].replace("_", "")))
    return rows


def traffic_for(workload, plan_kernel, plan_key):
    """DRAM bytes per launch from an ncu capture of this plan's current source, else None."""
    row = traffic_table().get((workload, plan_key))
    if row is None or plan_kernel not in PLAN_SOURCES:
        return None
    return row[1] if row[0] == source_hash(PLAN_SOURCES[plan_kernel]) else None


def hbm_peak():
    """(GB/s, source) of the copy bandwidth the HBM fractions are taken against."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def fp64_probe():
    """Run the FP64 pipe micro-benchmark (built by build() next to its source) on this GPU."""
    exe = os.path.join(PKG, "peak", "fp64_peak")
    if not os.path.exists(exe):
        from paper_2010_04868_gb300 import build as _b
        exe = _b.build_probe()
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    for ln in out.stdout.splitlines():
        if ln.startswith("{") and "fp64_lane_ops_per_sm_clk" in ln:
            return json.loads(ln)
    raise RuntimeError("FP64 probe failed: %s %s" % (out.stdout[-300:], out.stderr[-300:]))


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


# ------------------------------------------------------------------ workload helpers

def workload_config(world):
    """The workload both arms (the library and the oracle) report on."""
    return {"workload": "Jacobi 2D 5-point star + 9-point box, 4096x4096 FP64, zero Dirichlet halo, "
                        "T=1000 each, autotuned kernel", "grids": "2 x 4096^2", "T": T_STEPS,
            "l2": "inputs (2 x 128 MiB grid + scratch) exceed L2; 512 MiB flush between steps",
            "parallelism": "replicas" if world > 1 else "single GPU"}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the method_configs sections")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=20.0, help="arrival rate (requests/s) of the serving section")
    ap.add_argument("--serve-slots", type=int, default=16)
    ap.add_argument("--source-hash", action="store_true")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate(total_ms, world, dist=None, device=None):
    """Max over ranks of the timed milliseconds (every rank must call it when world > 1)."""
    if world > 1:
        import torch
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())
    return float(total_ms)


def job_value(updates_per_rank_step, world, ms_per_step):
    """Whole-job throughput in GStencil/s: every rank processes its own replica in ms_per_step."""
    return world * updates_per_rank_step / (ms_per_step * 1e-3) / 1e9


def passes_of(plan, T):
    """Passes over the grid through HBM: every step for the plain kernel, every T_b steps for the
    blocked and split-tiled kernels, every 32-sweep block for the wavefront."""
    if plan["kernel"] in ("blocked", "diamond", "stream"):
        return -(-T // max(1, plan["tb"]))
    if plan["kernel"] == "wavefront":
        return -(-T // 32)
    return T


def weights(k):
    from paper_2010_04868_gb300 import inputs
    return inputs.normalized_weights(inputs.SEED_BASE + 100 + k, k)


def initial_grid():
    from paper_2010_04868_gb300 import inputs
    return inputs.grid(inputs.SEED_BASE + 2, (N_SIDE, N_SIDE))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.proc = None
        self.lines = []
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


class Roofs:
    """The two rooflines of this run: the FP64 pipe (probe, per SM clock) and HBM copy bandwidth."""

    def __init__(self, probe, nsm):
        self.ops_per_sm_clk = float(probe["fp64_lane_ops_per_sm_clk"])
        self.nsm = nsm
        self.hbm_gbs, self.hbm_src = hbm_peak()

    def fp64_peak(self, sm_mhz):
        return self.ops_per_sm_clk * self.nsm * (sm_mhz or 2070.0) * 1e6 / 1e9

    def figures(self, updates, k, ms, hbm_bytes, sm_mhz, tb_eff=1):
        """FP64 and HBM figures of a run: achieved rates, fractions, the binding roofline."""
        s = ms * 1e-3
        gst = updates / s / 1e9
        fp64 = updates * k / s / 1e9
        gbs = hbm_bytes / s / 1e9
        fp64_roof = self.fp64_peak(sm_mhz) / k
        hbm_roof = self.hbm_gbs * tb_eff / 16.0
        return {"gstencil_s": round(gst, 3), "fp64_gops": round(fp64, 1),
                "fp64_frac": round(fp64 / self.fp64_peak(sm_mhz), 4),
                "hbm_algorithmic_bytes": int(hbm_bytes), "hbm_gbs": round(gbs, 1),
                "hbm_frac": round(gbs / self.hbm_gbs, 4),
                "roofline_gstencil_s": {"fp64": round(fp64_roof, 2), "hbm_effective": round(hbm_roof, 1),
                                        "hbm_steps_per_pass": tb_eff,
                                        "binding": "fp64" if fp64_roof < hbm_roof else "hbm"}}


# ------------------------------------------------------------------ the headline workload

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2010_04868_gb300 import stencil as S

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    roofs = Roofs(fp64_probe(), nsm)

    u0_host = initial_grid()
    u0 = torch.from_numpy(u0_host).to(dev)
    work = {}
    for name, shape, k in STENCILS:
        st = S.Stencil(2, shape, 1, list(weights(k)), S.STENCIL_JACOBI)
        work[name] = dict(st=st, u=torch.empty_like(u0), scratch=torch.empty_like(u0), k=k)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)   # 512 MiB > L2

    nlaunch = {name: 0 for name, _, _ in STENCILS}

    def one_step(events=None):
        for name, _, _ in STENCILS:
            wk = work[name]
            if events is not None:
                events[name][0].record(stream)
            c0 = S.stencil_launch_count()
            wk["st"].run(wk["u"], T_STEPS, wk["scratch"])
            nlaunch[name] = S.stencil_launch_count() - c0
            if events is not None:
                events[name][1].record(stream)

    def reset():
        for name, _, _ in STENCILS:
            work[name]["u"].copy_(u0)
        flush.zero_()

    for _ in range(args.warmup):
        reset()
        one_step()
    torch.cuda.synchronize()
    for name, _, _ in STENCILS:
        rc = work[name]["st"].status()
        if rc != 0:
            raise RuntimeError("device status after warm-up: " + S.strerror(rc))

    plans = {}
    for name, _, _ in STENCILS:
        k, tb, tile = work[name]["st"].plan(work[name]["u"], T_STEPS)
        plans[name] = {"kernel": KERNEL_NAMES.get(k, str(k)), "tb": tb, "tile": list(tile)}

    sampler = ClockSampler(local).start()
    times = {name: 0.0 for name, _, _ in STENCILS}
    launches0 = S.stencil_launch_count()
    total_ms = 0.0
    for _ in range(args.steps):
        reset()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = {name: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for name, _, _ in STENCILS}
        one_step(ev)
        torch.cuda.synchronize()
        for name, _, _ in STENCILS:
            times[name] += ev[name][0].elapsed_time(ev[name][1])
        total_ms += ev[STENCILS[0][0]][0].elapsed_time(ev[STENCILS[-1][0]][1])
    launches = S.stencil_launch_count() - launches0
    clocks = sampler.stop()
    for name, _, _ in STENCILS:
        rc = work[name]["st"].status()
        if rc != 0:
            raise RuntimeError("device status after timing: " + S.strerror(rc))

    total_ms = aggregate(total_ms, world, dist, dev)
    updates_per_step = len(STENCILS) * N_SIDE * N_SIDE * T_STEPS
    ms_per_step = total_ms / args.steps
    value = job_value(updates_per_step, world, ms_per_step)

    # dominant kernel: the stencil with the larger share of the time
    dom = max(times, key=times.get)
    k_dom = work[dom]["k"]
    pd = plans[dom]
    launches_dom = max(1, nlaunch[dom])                      # kernel launches per run of the dominant stencil
    ops_per_launch = N_SIDE * N_SIDE * T_STEPS * k_dom / launches_dom   # FMA mode: K FP64 ops per update
    avg_launch_ms = times[dom] / args.steps / launches_dom
    achieved = ops_per_launch / (avg_launch_ms * 1e-3) / 1e9
    peak = roofs.fp64_peak(clocks.get("sm_mhz"))
    bytes_per_launch = 16 * N_SIDE * N_SIDE * passes_of(pd, T_STEPS) // launches_dom
    plan_key = "%s tb%d tile%s" % (pd["kernel"], pd["tb"], "x".join(str(t) for t in pd["tile"]))
    traffic = traffic_for("jacobi2d9" if dom == "2d9p" else "jacobi2d5", pd["kernel"], plan_key)
    roofline = {"bound": "alu",
                "kernel": "Jacobi 2D %dP %s (%d launches per run)" % (k_dom, pd["kernel"], launches_dom),
                "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": "Gop/s (FP64 lane operations)",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": "measured: FP64 probe in this run (%.4f lane-ops/SM/clk, best of its sweep) x %d SMs "
                               "x median SM clock of the timed region" % (roofs.ops_per_sm_clk, nsm),
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "hbm_gbs": round(bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9, 1),
                "hbm_frac": round(bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9 / roofs.hbm_gbs, 4),
                "hbm_peak_gbs": roofs.hbm_gbs, "hbm_peak_source": roofs.hbm_src,
                "traffic_source": "profiles/dram_traffic.md (ncu, same kernel source)" if traffic else
                                  "no ncu capture of this plan's current source"}

    per_stencil = {name: round(N_SIDE * N_SIDE * T_STEPS * args.steps / (times[name] * 1e-3) / 1e9, 3)
                   for name, _, _ in STENCILS}

    # the plain per-step kernel on the same grids, one run of each stencil, for comparison
    plain = {}
    for name, _, _ in STENCILS:
        wk = work[name]
        wk["st"].set_plan(S.STENCIL_KERNEL_PLAIN)
        wk["u"].copy_(u0)
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        wk["st"].run(wk["u"], T_STEPS, wk["scratch"])
        e1.record(stream)
        torch.cuda.synchronize()
        plain[name] = round(N_SIDE * N_SIDE * T_STEPS / (e0.elapsed_time(e1) * 1e-3) / 1e9, 3)
        wk["st"].set_plan(S.STENCIL_KERNEL_AUTO)

    # the streaming temporally blocked kernel (T_b = 2 and 4, default tiles) on the same grids
    blocked = {}
    for name, _, _ in STENCILS:
        wk = work[name]
        for tb in (2, 4):
            wk["st"].set_plan(S.STENCIL_KERNEL_STREAM, tb)
            wk["u"].copy_(u0)
            wk["st"].run(wk["u"], 8, wk["scratch"])
            wk["u"].copy_(u0)
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            wk["st"].run(wk["u"], T_STEPS, wk["scratch"])
            e1.record(stream)
            torch.cuda.synchronize()
            blocked["%s_tb%d" % (name, tb)] = round(N_SIDE * N_SIDE * T_STEPS / (e0.elapsed_time(e1) * 1e-3) / 1e9, 3)
        wk["st"].set_plan(S.STENCIL_KERNEL_AUTO)
        rc = wk["st"].status()
        if rc != 0:
            raise RuntimeError("device status after the streaming kernel: " + S.strerror(rc))

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(work, u0_host, stream, S)
    for name in work:
        work[name]["st"].close()
    del work, u0, flush
    torch.cuda.empty_cache()

    extra = None
    if not args.no_extra and rank == 0:
        extra = method_configs(args, roofs, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(budget_s=12.0)

    if rank == 0:
        line = {
            "metric": "FP64 GStencil/s", "value": round(value, 3), "unit": "GStencil/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 uniform [0,1), seeded normalised weights)",
            "config": workload_config(world),
            "per_stencil_gstencil_s": per_stencil, "plain_kernel_gstencil_s": plain,
            "stream_blocked_kernel_gstencil_s": blocked, "plans": plans,
            "roofline": roofline, "clocks": clocks, "gpu_launches": int(launches),
            "e2e": e2e, "cpu_baseline": cpu, "method_configs": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_e2e(work, u0_host, stream, S):
    """The same workload through stencil_run_host: pinned host grid in, result back, every step."""
    import ctypes

    import torch
    host = {name: torch.from_numpy(u0_host.copy()).pin_memory() for name in work}
    nbytes = u0_host.nbytes
    sptr = ctypes.c_void_p(stream.cuda_stream)

    def step():
        for name, wk in work.items():
            S.stencil_run_host(wk["st"].handle, ctypes.c_void_p(host[name].data_ptr()), (N_SIDE, N_SIDE),
                               ctypes.c_void_p(wk["u"].data_ptr()), ctypes.c_void_p(wk["scratch"].data_ptr()),
                               T_STEPS, sptr)

    step()
    torch.cuda.synchronize()
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    updates = len(work) * N_SIDE * N_SIDE * T_STEPS
    return {"value": round(updates / dt / 1e9, 3), "unit": "GStencil/s", "h2d_bytes_per_step": len(work) * nbytes,
            "d2h_bytes_per_step": len(work) * nbytes, "ms_per_step": round(dt * 1e3, 2)}


# ------------------------------------------------------------------ the method's other kernels

def _timed(fn, reset, reps, stream):
    """Mean CUDA-event milliseconds of fn over reps runs, reset() (outside the window) before each."""
    import torch
    tot = 0.0
    for _ in range(reps):
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps


def _plan_dict(st, u, T):
    k, tb, tile = st.plan(u, T)
    return {"kernel": KERNEL_NAMES.get(k, str(k)), "tb": tb, "tile": list(tile)}


def _single(name, workload, roofs, dev, reps, plain_T=None, plain_reps=1):
    """One workload of paper_2010_04868_gb300.workloads (the same seeded grid and weights as its ncu
    captures): the library's default plan against the plain per-step kernel, in one clocked window."""
    import torch

    from paper_2010_04868_gb300 import stencil as S
    from paper_2010_04868_gb300 import workloads as WL
    dim, shape, method, ext, T, bc, _ = WL.CONFIGS[name]
    stream = torch.cuda.current_stream()
    k = WL.k_points(dim, shape)
    u0 = torch.from_numpy(WL.config_grid(name)).to(dev)
    st = S.Stencil(dim, shape, 1, WL.config_weights(name), method, bc)
    u = torch.empty_like(u0)
    scratch = torch.empty_like(u0) if method == S.STENCIL_JACOBI else None
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)

    def reset():
        u.copy_(u0)
        flush.zero_()

    reset()
    st.run(u, T, scratch)                       # tuning (Jacobi) and warm-up outside the window
    torch.cuda.synchronize()
    plan = _plan_dict(st, u, T)
    sampler = ClockSampler(dev.index or 0).start()
    c0 = S.stencil_launch_count()
    ms = _timed(lambda: st.run(u, T, scratch), reset, reps, stream)
    launches = (S.stencil_launch_count() - c0) // reps
    rc = st.status()
    st.set_plan(S.STENCIL_KERNEL_PLAIN)
    pT = plain_T or T
    if pT == T:
        reset()
        st.run(u, 1, scratch)                   # first launch of the plain kernel outside the window
    ms_plain = _timed(lambda: st.run(u, pT, scratch), reset, plain_reps, stream) * T / pT
    clocks = sampler.stop()
    rc = rc or st.status()
    st.close()
    if rc != 0:
        raise RuntimeError("%s: %s" % (name, S.strerror(rc)))
    npts = 1
    for e in ext:
        npts *= e
    passes = passes_of(plan, T)
    tb_eff = T / passes
    out = {"workload": workload, "plan": plan, "ms": round(ms, 3), "launches_per_run": launches, "reps": reps}
    out.update(roofs.figures(npts * T, k, ms, 16 * npts * passes, clocks.get("sm_mhz"), round(tb_eff, 2)))
    plain_fig = roofs.figures(npts * T, k, ms_plain, 16 * npts * T, clocks.get("sm_mhz"))
    out["plain"] = {"ms": round(ms_plain, 3), "gstencil_s": plain_fig["gstencil_s"],
                    "fp64_frac": plain_fig["fp64_frac"], "hbm_gbs": plain_fig["hbm_gbs"],
                    "hbm_frac": plain_fig["hbm_frac"],
                    "timed": ("full T=%d" % T) if pT == T else ("%d of the %d steps, scaled to T (each step of the "
                                                                 "plain kernel does the same work)" % (pT, T))}
    out["speedup_vs_plain"] = round(ms_plain / ms, 3)
    plan_key = "%s tb%d tile%s" % (plan["kernel"], plan["tb"], "x".join(str(t) for t in plan["tile"]))
    tr = traffic_for(name, plan["kernel"], plan_key)
    out["traffic_per_launch"] = tr
    out["clocks"] = clocks
    del u0, u, scratch, flush
    torch.cuda.empty_cache()
    return out


def _batch512(roofs, dev, reps):
    """The three 512^3 periodic problems in one stencil_run_batch call, against separate tuned and plain runs."""
    import ctypes

    import torch

    from paper_2010_04868_gb300 import stencil as S
    from paper_2010_04868_gb300 import workloads as WL
    stream = torch.cuda.current_stream()
    names = ("jacobi3d7", "jacobi3d27", "gs3d7")
    T = WL.CONFIGS[names[0]][4]
    # one seeded 512^3 grid (that of the 7-point Jacobi workload) is the input of all three problems
    u0 = torch.from_numpy(WL.config_grid(names[0])).to(dev)
    sts, us, scs, ks = [], [], [], []
    for n in names:
        dim, shape, method, ext, _, bc, _ = WL.CONFIGS[n]
        sts.append(S.Stencil(dim, shape, 1, WL.config_weights(n), method, bc))
        us.append(torch.empty_like(u0))
        scs.append(torch.empty_like(u0) if method == S.STENCIL_JACOBI else None)
        ks.append(WL.k_points(dim, shape))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float64, device=dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)
    grids = [st.grid(u, sc) for st, u, sc in zip(sts, us, scs)]

    def reset():
        for u in us:
            u.copy_(u0)
        flush.zero_()

    def batch():
        S.stencil_run_batch([s.handle for s in sts], grids, [T] * 3, sptr)

    def separate():
        for st, u, sc in zip(sts, us, scs):
            st.run(u, T, sc)

    reset()
    batch()                                         # tunes the Jacobi plans and captures the graph
    separate()
    torch.cuda.synchronize()
    plans = [_plan_dict(st, u, T) for st, u in zip(sts, us)]
    sampler = ClockSampler(dev.index or 0).start()
    c0 = S.stencil_launch_count()
    ms_batch = _timed(batch, reset, reps, stream)
    launches = (S.stencil_launch_count() - c0) // reps
    ms_sep = _timed(separate, reset, reps, stream)
    for st in sts:
        st.set_plan(S.STENCIL_KERNEL_PLAIN)
    ms_plain = _timed(separate, reset, 1, stream)
    clocks = sampler.stop()
    for st in sts:
        if st.status() != 0:
            raise RuntimeError("batch512: device status")
        st.close()
    npts = 512 ** 3
    upd = 3 * npts * T
    ops = npts * T * sum(ks)
    sm = clocks.get("sm_mhz")
    s = ms_batch * 1e-3
    out = {"workload": "Jacobi 3D 7-point + Jacobi 3D 27-point + Gauss-Seidel 3D 7-point, 512^3 FP64 periodic, "
                       "T=100 each, one stencil_run_batch call (persistent launch, CUDA graph)",
           "plans_separate": dict(zip(names, plans)), "ms": round(ms_batch, 2),
           "launches_per_run": launches, "reps": reps,
           "gstencil_s": round(upd / s / 1e9, 3), "fp64_gops": round(ops / s / 1e9, 1),
           "fp64_frac": round(ops / s / 1e9 / roofs.fp64_peak(sm), 4),
           "hbm_algorithmic_bytes": 16 * upd, "hbm_gbs": round(16 * upd / s / 1e9, 1),
           "hbm_frac": round(16 * upd / s / 1e9 / roofs.hbm_gbs, 4),
           "separate_tuned": {"ms": round(ms_sep, 2), "gstencil_s": round(upd / ms_sep / 1e6, 3)},
           "plain": {"ms": round(ms_plain, 2), "gstencil_s": round(upd / ms_plain / 1e6, 3), "timed": "full T"},
           "speedup_vs_plain": round(ms_plain / ms_batch, 3), "speedup_vs_separate": round(ms_sep / ms_batch, 3),
           "traffic_per_launch": None, "clocks": clocks}
    del u0, us, scs, flush
    torch.cuda.empty_cache()
    return out


def _serving(args, dev):
    from paper_2010_04868_gb300 import serve
    sampler = ClockSampler(dev.index or 0).start()
    out = serve.bench_run(args.serve_requests, args.serve_rate, slots=args.serve_slots)
    out["clocks"] = sampler.stop()
    return out


def method_configs(args, roofs, dev):
    out = {"fp64_probe_lane_ops_per_sm_clk": roofs.ops_per_sm_clk, "hbm_peak_gbs": roofs.hbm_gbs,
           "hbm_peak_source": roofs.hbm_src,
           "l2": "a 512 MiB buffer is written between timed runs (outside the CUDA-event windows)"}
    out["heat1d"] = _single("heat1d", "Jacobi 1D 3-point heat (1/4, 1/2, 1/4), N=65536 FP64, zero halo, T=256",
                            roofs, dev, reps=20, plain_reps=20)
    out["gs2d"] = _single("gs2d5", "Gauss-Seidel 2D 5-point lexicographic, 4096^2 FP64, zero halo, T=200",
                          roofs, dev, reps=3, plain_reps=1)
    out["gs1d"] = _single("gs1d3", "Gauss-Seidel 1D 3-point lexicographic, N=2^24 FP64, zero halo, T=200",
                          roofs, dev, reps=2, plain_T=2, plain_reps=1)
    out["batch512"] = _batch512(roofs, dev, reps=2)
    out["serving"] = _serving(args, dev)
    return out


# ------------------------------------------------------------------ CPU baseline and reference arm

def cpu_baseline(budget_s=12.0):
    """The oracle as it stands, on the host cores, on a bounded sample of the workload."""
    import oracle
    u0 = initial_grid()
    cores = oracle.max_threads()
    # calibrate with one step of each stencil, then size the sample to the budget
    t0 = time.perf_counter()
    for name, shape, k in STENCILS:
        oracle.run(u0, 1, dim=2, shape=shape, r=1, weights=weights(k))
    per_step = time.perf_counter() - t0
    T = max(1, int(budget_s / max(per_step, 1e-6)))
    T = min(T, T_STEPS)
    t0 = time.perf_counter()
    for name, shape, k in STENCILS:
        oracle.run(u0, T, dim=2, shape=shape, r=1, weights=weights(k))
    dt = time.perf_counter() - t0
    updates = len(STENCILS) * N_SIDE * N_SIDE * T
    return {"value": round(updates / dt / 1e9, 4), "unit": "GStencil/s", "cores": cores, "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": "both stencils on the full 4096^2 grids for T=%d steps (of 1000), %.1f s" % (T, dt)}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    u0 = initial_grid()
    cores = oracle.max_threads()
    T = 2   # each step: a bounded sample of the workload (2 of the 1000 time steps of both stencils)
    for _ in range(args.warmup):
        for name, shape, k in STENCILS:
            oracle.run(u0, 1, dim=2, shape=shape, r=1, weights=weights(k))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for name, shape, k in STENCILS:
            oracle.run(u0, T, dim=2, shape=shape, r=1, weights=weights(k))
    dt = time.perf_counter() - t0
    updates = args.steps * len(STENCILS) * N_SIDE * N_SIDE * T
    value = updates / dt / 1e9
    sample = "both stencils on the full 4096^2 grids, %d of the 1000 time steps per step" % T
    line = {"impl": "reference", "metric": "FP64 GStencil/s", "value": round(value, 4), "unit": "GStencil/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(world),
            "cpu_baseline": {"value": round(value, 4), "unit": "GStencil/s", "cores": cores,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GStencil/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.source_hash:
        print(json.dumps({k: source_hash(v) for k, v in PLAN_SOURCES.items()}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
