"""Benchmark: FP64 stencil throughput on one GB300 (GStencil/s = point updates per second).

Workload (one "step"): the Jacobi 2D 5-point star and 9-point box stencils on
4096 x 4096 FP64 grids, seeded uniform [0, 1) inputs, seeded positive weights
normalised to sum 1, zero Dirichlet halo, T = 1000 time steps each, run
through the library's C ABI with its default (autotuned) kernel choice. The
paper's Table 1 lists Heat-2D and 2D9P on 8000^2 x 2000; this is the same
kind of workload at a size one step of which takes well under a second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line. --impl reference times the CPU oracle (the plain
definition in C, OpenMP over the host cores) on a bounded sample of the same
workload instead. Under torchrun (N > 1) every rank runs an independent
replica (the workload has no cross-grid exchange), timed between barriers;
rank 0 reports the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 4096
T_STEPS = 1000
STENCILS = (("2d5p", 0, 5), ("2d9p", 1, 9))   # name, shape id, K
# FP64 pipe throughput measured on this GPU with a DFMA/DADD/DMUL micro-benchmark
# (python -m paper_2010_04868_gb300.peak): 1.684 lane operations per SM clock for
# all three instructions, 152 SMs, i.e. 529.9 Gop/s at the 2070 MHz maximum clock.
FP64_OPS_PER_SM_CLK = 1.684
N_SM = 152
KERNEL_NAMES = {1: "plain", 2: "blocked", 3: "wavefront", 4: "diamond"}
# DRAM bytes (read + write) per launch on this workload, from ncu captures
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by stencil and plan
# (kernel, T_b, tile); a plan without a capture reports null. Plain: one step
# per launch, algorithmically 16 B per point update (268.4 MB per launch).
# Split (diamond) tiles: four launches (one per tile type) per band of T_b steps; the figure is the
# band's total over four, so it includes the per-level edge bands the tiles exchange through L2/HBM.
NCU_TRAFFIC = {("2d9p", "plain", 1, (0, 0, 0)): 134_256_128 + 94_363_392,
               ("2d9p", "diamond", 16, (0, 88, 88)): (464_250_112 + 175_210_752) // 4}


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


def algorithmic_bytes_per_launch(plan, launches):
    """16 B per point per pass over the grid (one read, one write): every step for the plain kernel,
    every T_b steps for the blocked and split-tiled kernels."""
    tb = max(1, plan["tb"]) if plan["kernel"] in ("blocked", "diamond") else 1
    passes = -(-T_STEPS // tb)
    return 16 * N_SIDE * N_SIDE * passes // max(1, launches)


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

    sampler = ClockSampler(local)
    sampler.start()
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
    launches_dom = max(1, nlaunch[dom])                      # kernel launches per run of the dominant stencil
    ops_per_launch = N_SIDE * N_SIDE * T_STEPS * k_dom / launches_dom   # FMA mode: K FP64 ops per update
    avg_launch_ms = times[dom] / args.steps / launches_dom
    achieved = ops_per_launch / (avg_launch_ms * 1e-3) / 1e9
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak = FP64_OPS_PER_SM_CLK * N_SM * sm_mhz * 1e6 / 1e9
    pd = plans[dom]
    traffic = NCU_TRAFFIC.get((dom, pd["kernel"], pd["tb"], tuple(pd["tile"])))
    roofline = {"bound": "alu",
                "kernel": "Jacobi 2D %dP %s (%d launches per run)" % (k_dom, pd["kernel"], launches_dom),
                "achieved": round(achieved, 2), "peak": round(peak, 2), "unit": "Gop/s (FP64 lane operations)",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": algorithmic_bytes_per_launch(pd, launches_dom)}

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

    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(work, u0_host, stream, S)

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
            "per_stencil_gstencil_s": per_stencil, "plain_kernel_gstencil_s": plain, "plans": plans,
            "roofline": roofline, "clocks": clocks, "gpu_launches": int(launches),
            "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    for name in work:
        work[name]["st"].close()
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
    return {"value": round(updates / dt / 1e9, 4), "unit": "GStencil/s", "cores": cores, "kind": "oracle",
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
            "cpu_baseline": {"value": round(value, 4), "unit": "GStencil/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GStencil/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
