"""Continuous-batching request loop for stencil solves.

A request is one stencil solve: (method, dim, shape, extents, T, seed). The
server keeps up to ``slots`` requests on the GPU at once, each on its own CUDA
stream so that their kernels overlap on the device. Arriving requests wait in
a FIFO queue and are admitted as soon as a slot is free and their device
memory (grid, plus scratch for Jacobi) fits under ``mem_cap`` bytes; their
grids stay resident on the device for the whole solve. Completions are found
by polling CUDA events, and each request's latency is its completion time
minus its arrival time. Every solve goes through the library's C ABI
(``stencil_run`` with the autotuned plan, or a fixed plan), so a request
gives the same result alone and in the mix.

The scheduling logic (:class:`Server`) is independent of the executor, so it
can be driven by a simulated executor on the CPU.

Workload recipe (seeded; see :func:`request_mix`): method Jacobi or
Gauss-Seidel, dimension 1/2/3 uniform, Jacobi shape star or box uniform,
Gauss-Seidel star, 1D N log-uniform in [2^12, 2^22], 2D side log-uniform in
[256, 4096], 3D side log-uniform in [64, 384], T uniform in [10, 500],
radius 1, zero Dirichlet halo, Poisson arrivals.
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import inputs


@dataclass
class Request:
    rid: int
    method: int          # 0 Jacobi, 1 Gauss-Seidel
    dim: int
    shape: int           # 0 star, 1 box
    ext: tuple
    T: int
    seed: int
    arrival: float = 0.0

    @property
    def points(self) -> int:
        return int(np.prod(self.ext))

    @property
    def nbytes(self) -> int:
        return self.points * 8 * (2 if self.method == 0 else 1)

    @property
    def updates(self) -> int:
        return self.points * self.T


def _log_uniform_int(u, lo, hi):
    return int(round(math.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))))


def request_mix(n: int, seed: int = inputs.SEED_BASE + 5) -> list:
    """n requests drawn from the serving recipe (deterministic in seed)."""
    u = inputs.uniform(seed, 5 * n).reshape(n, 5)
    reqs = []
    for i in range(n):
        method = 0 if u[i, 0] < 0.5 else 1
        dim = 1 + min(2, int(u[i, 1] * 3))
        shape = (0 if u[i, 2] < 0.5 else 1) if (method == 0 and dim > 1) else 0
        if dim == 1:
            ext = (_log_uniform_int(u[i, 3], 1 << 12, 1 << 22),)
        elif dim == 2:
            s = _log_uniform_int(u[i, 3], 256, 4096)
            ext = (s, s)
        else:
            s = _log_uniform_int(u[i, 3], 64, 384)
            ext = (s, s, s)
        T = 10 + min(490, int(u[i, 4] * 491))
        reqs.append(Request(i, method, dim, shape, ext, T, seed * 1000003 + i))
    return reqs


def poisson_arrivals(reqs, rate: float, seed: int = inputs.SEED_BASE + 6):
    """Set arrival times of reqs to a Poisson process of the given rate (requests/s)."""
    u = inputs.uniform(seed, len(reqs))
    t = 0.0
    for r, x in zip(reqs, u):
        t += -math.log(1.0 - x) / rate
        r.arrival = t
    return reqs


def weights_for(req: Request):
    k = 2 * req.dim + 1 if req.shape == 0 else 3 ** req.dim
    return inputs.normalized_weights(req.seed + 17, k)


class GpuExecutor:
    """Runs requests through the C ABI, one CUDA stream per slot."""

    def __init__(self, slots: int, plan=None, keep_results: bool = False, device: int = 0):
        import torch
        self.torch = torch
        from . import stencil as S
        self.S = S
        self.dev = torch.device("cuda", device)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.free_streams = list(range(slots))
        self.plan = plan
        self.keep = keep_results
        self.results = {}

    def input_grid(self, req: Request):
        g = self.torch.Generator(device=self.dev)
        g.manual_seed(req.seed)
        return self.torch.rand(req.ext, dtype=self.torch.float64, device=self.dev, generator=g)

    def start(self, req: Request):
        torch, S = self.torch, self.S
        sid = self.free_streams.pop()
        stream = self.streams[sid]
        with torch.cuda.stream(stream):
            u = self.input_grid(req)
            scratch = torch.empty_like(u) if req.method == 0 else None
            st = S.Stencil(req.dim, req.shape, 1, list(weights_for(req)), req.method)
            if self.plan is not None:
                st.set_plan(self.plan)
            st.run(u, req.T, scratch, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return dict(req=req, sid=sid, u=u, scratch=scratch, st=st, ev=ev)

    def done(self, job) -> bool:
        return job["ev"].query()

    def finish(self, job):
        rc = job["st"].status(stream=self.streams[job["sid"]])
        if rc != 0:
            raise RuntimeError("request %d: %s" % (job["req"].rid, self.S.strerror(rc)))
        job["st"].close()
        if self.keep:
            self.results[job["req"].rid] = job["u"]
        self.free_streams.append(job["sid"])
        job.clear()


class SimExecutor:
    """CPU stand-in: a request finishes after updates / rate seconds (for scheduler tests)."""

    def __init__(self, slots: int, rate_updates_per_s: float = 1e10):
        self.rate = rate_updates_per_s
        self.started = {}
        self.max_inflight = 0

    def start(self, req: Request):
        job = dict(req=req, t_end=time.perf_counter() + req.updates / self.rate)
        self.started[req.rid] = job
        self.max_inflight = max(self.max_inflight, sum(1 for j in self.started.values() if "t_end" in j))
        return job

    def done(self, job) -> bool:
        return time.perf_counter() >= job["t_end"]

    def finish(self, job):
        job.pop("t_end", None)


@dataclass
class ServeStats:
    completed: int = 0
    rejected: int = 0
    makespan_s: float = 0.0
    latencies_ms: list = field(default_factory=list)
    updates: int = 0
    max_queue: int = 0
    max_mem: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"completed": self.completed, "rejected": self.rejected, "makespan_s": round(self.makespan_s, 4),
                "req_per_s": round(self.completed / self.makespan_s, 3) if self.makespan_s > 0 else None,
                "gstencil_s": round(self.updates / self.makespan_s / 1e9, 3) if self.makespan_s > 0 else None,
                "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "max_queue": self.max_queue, "max_mem_gb": round(self.max_mem / 1e9, 3)}


class Server:
    """FIFO admission by free slot and device-memory budget; completions by polling."""

    def __init__(self, executor, slots: int = 8, mem_cap: int = 40 * 10 ** 9):
        self.ex = executor
        self.slots = slots
        self.mem_cap = mem_cap

    def serve(self, reqs) -> ServeStats:
        pending = collections.deque(sorted(reqs, key=lambda r: (r.arrival, r.rid)))
        queue = collections.deque()
        inflight = []
        mem = 0
        stats = ServeStats()
        t0 = time.perf_counter()
        while pending or queue or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                if r.nbytes > self.mem_cap:
                    stats.rejected += 1
                    continue
                queue.append(r)
            stats.max_queue = max(stats.max_queue, len(queue))
            progressed = False
            while queue and len(inflight) < self.slots and mem + queue[0].nbytes <= self.mem_cap:
                r = queue.popleft()
                mem += r.nbytes
                stats.max_mem = max(stats.max_mem, mem)
                inflight.append((r, self.ex.start(r)))
                progressed = True
            still = []
            for r, job in inflight:
                if self.ex.done(job):
                    t_done = time.perf_counter() - t0
                    self.ex.finish(job)
                    mem -= r.nbytes
                    stats.completed += 1
                    stats.updates += r.updates
                    stats.latencies_ms.append((t_done - r.arrival) * 1e3)
                    progressed = True
                else:
                    still.append((r, job))
            inflight = still
            if not progressed:
                if inflight:
                    time.sleep(20e-6)
                elif pending:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
        stats.makespan_s = time.perf_counter() - t0
        return stats


def fifo_one_at_a_time(arrivals, service_s):
    """Latencies (s) of a one-at-a-time FIFO server with the given service times."""
    t, lat = 0.0, []
    for a, s in zip(arrivals, service_s):
        t = max(t, a) + s
        lat.append(t - a)
    return lat


def bench_run(n_requests: int, rate: float, slots: int = 8, mem_cap: int = 40 * 10 ** 9) -> dict:
    """The first n_requests of the seeded mix at a fixed Poisson rate (requests/s): latency and throughput.

    One request of each (method, dim, shape) class is served first, outside the measurement, so that
    first launches and plan lookups are not counted. Plans come from the tuner's cache or its static
    defaults (no tuning while serving).
    """
    import os

    import torch
    os.environ["STENCIL_NO_TUNE"] = "1"
    reqs = request_mix(n_requests)
    ex = GpuExecutor(slots)
    seen = set()
    for r in reqs:
        key = (r.method, r.dim, r.shape)
        if key not in seen:
            seen.add(key)
            Server(ex, slots, mem_cap).serve([Request(-1, r.method, r.dim, r.shape, r.ext, r.T, r.seed)])
    torch.cuda.synchronize()
    poisson_arrivals(reqs, rate)
    st = Server(GpuExecutor(slots), slots, mem_cap).serve(reqs).summary()
    st.update({"workload": "first %d requests of the seeded serving mix (Jacobi/Gauss-Seidel 1D-3D, T 10..500), "
                           "Poisson arrivals at %.1f requests/s, %d slots, %.0f GB cap" % (n_requests, rate, slots,
                                                                                          mem_cap / 1e9),
               "rate_req_s": rate, "slots": slots})
    return st


def main():
    ap = argparse.ArgumentParser(description="serving benchmark (continuous batching vs plain one at a time)")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--rates", default="0.5,0.8,1.1", help="arrival rates as multiples of the measured capacity")
    ap.add_argument("--plain-sample", type=int, default=12,
                    help="requests of the mix whose plain one-at-a-time service time is measured")
    ap.add_argument("--plain-T", type=int, default=4,
                    help="steps the plain service time is measured over (plain time is linear in T)")
    ap.add_argument("--tune", action="store_true", help="let the autotuner time plans for unseen shapes")
    args = ap.parse_args()
    import os

    import torch
    if not args.tune:
        os.environ["STENCIL_NO_TUNE"] = "1"   # cached plans if any, else the static defaults

    from . import stencil as S
    reqs = request_mix(args.requests)
    # warm-up and tuning outside the measurement: one request of each class
    ex = GpuExecutor(args.slots)
    seen = set()
    for r in reqs:
        key = (r.method, r.dim, r.shape)
        if key not in seen:
            seen.add(key)
            Server(ex, args.slots).serve([Request(-1, r.method, r.dim, r.shape, r.ext, r.T, r.seed)])
    torch.cuda.synchronize()
    # capacity of this server: everything arrives at once
    for r in reqs:
        r.arrival = 0.0
    sat = Server(GpuExecutor(args.slots), args.slots).serve(reqs).summary()
    cap = sat["req_per_s"]
    # plain kernels, one request at a time, on a sample: service times
    sample = reqs[:args.plain_sample]
    plain_s = []
    exp = GpuExecutor(1, plan=S.STENCIL_KERNEL_PLAIN)
    for r in sample:
        tp = min(r.T, args.plain_T)
        t0 = time.perf_counter()
        Server(exp, 1).serve([Request(r.rid, r.method, r.dim, r.shape, r.ext, tp, r.seed)])
        plain_s.append((time.perf_counter() - t0) * r.T / tp)
    ours_one = []
    exo = GpuExecutor(1)
    for r in sample:
        t0 = time.perf_counter()
        Server(exo, 1).serve([Request(r.rid, r.method, r.dim, r.shape, r.ext, r.T, r.seed)])
        ours_one.append(time.perf_counter() - t0)
    plain_cap = len(sample) / sum(plain_s)
    out = {"requests": args.requests, "slots": args.slots, "saturated": sat,
           "plain_one_at_a_time": {"sample": len(sample), "measured_T": args.plain_T, "req_per_s": round(plain_cap, 4),
                                   "mean_service_s": round(float(np.mean(plain_s)), 4),
                                   "sample_speedup_vs_ours_one_at_a_time": round(sum(plain_s) / sum(ours_one), 2)},
           "rates": []}
    for m in [float(x) for x in args.rates.split(",")]:
        rate = m * cap
        poisson_arrivals(reqs, rate)
        st = Server(GpuExecutor(args.slots), args.slots).serve(reqs).summary()
        # the plain one-at-a-time server at the same arrival times, from its measured service times
        svc = [plain_s[i % len(plain_s)] for i in range(len(reqs))]
        lat = np.array(fifo_one_at_a_time([r.arrival for r in reqs], svc)) * 1e3
        out["rates"].append({"multiple_of_capacity": m, "rate_req_s": round(rate, 3), "ours": st,
                             "plain_one_at_a_time_model": {"p50_ms": round(float(np.percentile(lat, 50)), 1),
                                                           "p99_ms": round(float(np.percentile(lat, 99)), 1)}})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
