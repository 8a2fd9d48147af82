"""Continuous-batching request loop for stencil solves.

A request is one stencil solve: (method, dim, shape, extents, T, seed). It names
one of the server's stencil operators (a catalog of one seeded operator per
(method, dim, shape) class) and carries its input as a seed: its grid is the
seeded uniform [0, 1) grid of inputs.grid(seed, extents), generated on the
device when the request is admitted.

The server keeps up to ``slots`` requests on the GPU at once, each on its own
CUDA stream so that their kernels overlap on the device. Arriving requests wait
in a FIFO queue and are admitted as soon as a slot is free and their device
memory (grid, plus scratch for Jacobi) fits in the server's arena: one device
allocation of ``mem_cap`` bytes made at start-up and handed out in 256-byte
aligned first-fit blocks, so admission counts exactly the memory the requests
hold. Their grids stay resident in the arena for the whole solve. Every slot
owns one library handle per operator class, created at start-up, so nothing on
the request path allocates or frees device memory through CUDA (freeing
synchronizes the whole device, which would serialize the slots). Completions
are found by polling CUDA events, and each request's latency is its completion
time minus its arrival time. Every solve goes through the library's C ABI
(``stencil_run`` with the autotuned plan, or a fixed plan), so a request gives
the same result alone and in the mix.

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

ALIGN = 256


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
    def grid_bytes(self) -> int:
        return (self.points * 8 + ALIGN - 1) // ALIGN * ALIGN

    @property
    def nbytes(self) -> int:
        """Arena bytes: the grid, plus a scratch grid for Jacobi (each 256-byte aligned)."""
        return self.grid_bytes * (2 if self.method == 0 else 1)

    @property
    def updates(self) -> int:
        return self.points * self.T

    @property
    def cls(self) -> tuple:
        return (self.method, self.dim, self.shape)


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


CLASSES = [(m, d, s) for m in (0, 1) for d in (1, 2, 3) for s in (0, 1) if not (s == 1 and (m == 1 or d == 1))]


def class_weights(cls) -> np.ndarray:
    """The catalog operator of a (method, dim, shape) class: seeded positive weights normalised to 1."""
    method, dim, shape = cls
    k = 2 * dim + 1 if shape == 0 else 3 ** dim
    return inputs.normalized_weights(inputs.SEED_BASE + 900 + 10 * method + 3 * dim + shape, k)


def weights_for(req: Request) -> np.ndarray:
    return class_weights(req.cls)


class ArenaBlocks:
    """First-fit allocation of 256-byte aligned blocks inside [0, cap) (offsets only; no memory)."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.free = [(0, self.cap)]          # sorted, disjoint, coalesced (offset, length)
        self.used = 0

    def alloc(self, nbytes: int):
        size = (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= size:
                if ln == size:
                    del self.free[i]
                else:
                    self.free[i] = (off + size, ln - size)
                self.used += size
                return off
        return None

    def release(self, off: int, nbytes: int):
        size = (int(nbytes) + ALIGN - 1) // ALIGN * ALIGN
        self.used -= size
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, size))
        # coalesce with the neighbours
        if i + 1 < len(self.free) and self.free[i][0] + self.free[i][1] == self.free[i + 1][0]:
            self.free[i] = (self.free[i][0], self.free[i][1] + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]


class GpuExecutor:
    """Runs requests through the C ABI: one CUDA stream and one handle per operator class per slot,
    request memory in one device arena of mem_cap bytes."""

    def __init__(self, slots: int, mem_cap: int, plan=None, keep_results=None, device: int = 0):
        import torch
        self.torch = torch
        from . import stencil as S
        self.S = S
        self.dev = torch.device("cuda", device)
        self.arena = torch.empty(int(mem_cap), dtype=torch.uint8, device=self.dev)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(slots)]
        self.handles = [{c: S.Stencil(c[1], c[2], 1, list(class_weights(c)), c[0]) for c in CLASSES}
                        for _ in range(slots)]
        if plan is not None:
            for hs in self.handles:
                for st in hs.values():
                    st.set_plan(plan)
        self.keep = set(keep_results or ())       # request ids whose results are copied to the host
        self.results = {}

    def views(self, req: Request, off: int):
        u = self.arena[off:off + req.points * 8].view(self.torch.float64).view(req.ext)
        sc = None
        if req.method == 0:
            o2 = off + req.grid_bytes
            sc = self.arena[o2:o2 + req.points * 8].view(self.torch.float64).view(req.ext)
        return u, sc

    def start(self, req: Request, off: int, slot: int):
        torch = self.torch
        stream = self.streams[slot]
        st = self.handles[slot][req.cls]
        with torch.cuda.stream(stream):
            u, sc = self.views(req, off)
            inputs.grid_into(u, req.seed)
            st.run(u, req.T, sc, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        return dict(req=req, slot=slot, u=u, st=st, ev=ev)

    def done(self, job) -> bool:
        return job["ev"].query()

    def finish(self, job):
        rc = job["st"].status(stream=self.streams[job["slot"]])
        if rc != 0:
            raise RuntimeError("request %d: %s" % (job["req"].rid, self.S.strerror(rc)))
        if job["req"].rid in self.keep:
            self.results[job["req"].rid] = job["u"].cpu().numpy()
        job.clear()

    def close(self):
        for hs in self.handles:
            for st in hs.values():
                st.close()
        self.handles = []


class SimExecutor:
    """CPU stand-in: a request finishes after updates / rate seconds (for scheduler tests)."""

    def __init__(self, slots: int, rate_updates_per_s: float = 1e10):
        self.rate = rate_updates_per_s
        self.inflight = {}
        self.max_inflight = 0
        self.slots_seen = set()

    def start(self, req: Request, off: int, slot: int):
        assert slot not in {j["slot"] for j in self.inflight.values()}, "a slot runs one request at a time"
        job = dict(req=req, slot=slot, off=off, t_end=time.perf_counter() + req.updates / self.rate)
        self.inflight[req.rid] = job
        self.slots_seen.add(slot)
        self.max_inflight = max(self.max_inflight, len(self.inflight))
        return job

    def done(self, job) -> bool:
        return time.perf_counter() >= job["t_end"]

    def finish(self, job):
        self.inflight.pop(job["req"].rid, None)


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
    """FIFO admission by free slot and arena block; completions by polling."""

    def __init__(self, executor, slots: int = 8, mem_cap: int = 40 * 10 ** 9):
        self.ex = executor
        self.slots = slots
        self.mem_cap = mem_cap

    def serve(self, reqs) -> ServeStats:
        pending = collections.deque(sorted(reqs, key=lambda r: (r.arrival, r.rid)))
        queue = collections.deque()
        inflight = []
        arena = ArenaBlocks(self.mem_cap)
        free_slots = list(range(self.slots - 1, -1, -1))
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
            while queue and free_slots:
                off = arena.alloc(queue[0].nbytes)
                if off is None:
                    break                     # FIFO: the head waits for memory
                r = queue.popleft()
                stats.max_mem = max(stats.max_mem, arena.used)
                slot = free_slots.pop()
                inflight.append((r, off, slot, self.ex.start(r, off, slot)))
                progressed = True
            still = []
            for r, off, slot, job in inflight:
                if self.ex.done(job):
                    t_done = time.perf_counter() - t0
                    self.ex.finish(job)
                    arena.release(off, r.nbytes)
                    free_slots.append(slot)
                    stats.completed += 1
                    stats.updates += r.updates
                    stats.latencies_ms.append((t_done - r.arrival) * 1e3)
                    progressed = True
                else:
                    still.append((r, off, slot, job))
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


def tune_keys(reqs):
    """One representative request per plan-cache key the tuner would use (class, extent buckets, T class)."""
    def bucket(n):
        b = 0
        while (1 << b) < n:
            b += 1
        return b
    seen = {}
    for r in reqs:
        tcls = 0 if r.T < 8 else (1 if r.T < 64 else (2 if r.T < 512 else 3))
        key = (r.cls, tuple(bucket(e) for e in r.ext), tcls)
        if key not in seen or r.points > seen[key].points:
            seen[key] = r
    return list(seen.values())


def prepare(ex: GpuExecutor, reqs, grow: bool = True):
    """Outside any measurement: tune every plan the requests will use, and run one request of each
    class in every slot (first launches; with grow, workspaces grown to the class's largest
    request, else a small request of each class)."""
    torch = ex.torch
    for r in tune_keys(reqs):
        u, _ = ex.views(r, 0)
        ex.handles[0][r.cls].plan(u, r.T)
    if not grow:
        small = {}
        for r in reqs:
            if r.cls not in small or r.updates < small[r.cls].updates:
                small[r.cls] = r
        for slot in range(len(ex.streams)):
            for r in small.values():
                job = ex.start(Request(-1, r.method, r.dim, r.shape, r.ext, 2, r.seed), 0, slot)
                torch.cuda.synchronize()
                ex.finish(job)
        return
    largest = {}
    for r in reqs:
        if r.cls not in largest or r.points > largest[r.cls].points:
            largest[r.cls] = r
    for slot in range(len(ex.streams)):
        for r in largest.values():
            # the wavefront's workspace grows with T as well; Jacobi workspaces do not
            T = r.T if r.method == 1 else min(r.T, 40)
            job = ex.start(Request(-1, r.method, r.dim, r.shape, r.ext, T, r.seed), 0, slot)
            torch.cuda.synchronize()
            ex.finish(job)


def service_times(reqs, plan=None, mem_cap: int = 8 * 10 ** 9):
    """Seconds each request takes alone on a one-slot server (input generation and the full T solve)."""
    ex = GpuExecutor(1, mem_cap, plan=plan)
    prepare(ex, reqs, grow=False)
    out = []
    for r in reqs:
        t0 = time.perf_counter()
        Server(ex, 1, mem_cap).serve([Request(r.rid, r.method, r.dim, r.shape, r.ext, r.T, r.seed)])
        out.append(time.perf_counter() - t0)
    ex.close()
    return out


def fit_service_model(reqs, secs):
    """Per class, seconds = a + b * updates (least squares on the measured requests)."""
    model = {}
    for c in CLASSES:
        xs = [(r.updates, s) for r, s in zip(reqs, secs) if r.cls == c]
        if not xs:
            continue
        x = np.array([u for u, _ in xs], dtype=np.float64)
        y = np.array([s for _, s in xs], dtype=np.float64)
        if len(xs) >= 2 and np.ptp(x) > 0:
            b, a = np.polyfit(x, y, 1)
            a = max(a, 0.0)
        else:
            a, b = 0.0, float(y.mean() / x.mean())
        model[c] = (float(a), float(max(b, 0.0)))
    return model


def stratified_sample(reqs, per_class: int):
    """The first per_class requests of every class, spread over the size range (sorted by updates)."""
    out = []
    for c in CLASSES:
        rs = sorted([r for r in reqs if r.cls == c], key=lambda r: r.updates)
        if not rs:
            continue
        idx = np.unique(np.linspace(0, len(rs) - 1, min(per_class, len(rs))).round().astype(int))
        out += [rs[i] for i in idx]
    return out


def bench_run(n_requests: int, rate: float, slots: int = 8, mem_cap: int = 40 * 10 ** 9) -> dict:
    """The first n_requests of the seeded mix at a fixed Poisson rate (requests/s): latency and throughput.

    Tuning, first launches and workspace growth happen before the measurement (prepare)."""
    reqs = request_mix(n_requests)
    ex = GpuExecutor(slots, mem_cap)
    prepare(ex, reqs)
    ex.torch.cuda.synchronize()
    poisson_arrivals(reqs, rate)
    st = Server(ex, slots, mem_cap).serve(reqs).summary()
    ex.close()
    st.update({"workload": "first %d requests of the seeded serving mix (Jacobi/Gauss-Seidel 1D-3D, T 10..500), "
                           "Poisson arrivals at %.1f requests/s, %d slots, %.0f GB arena" % (n_requests, rate, slots,
                                                                                            mem_cap / 1e9),
               "rate_req_s": rate, "slots": slots})
    return st


def main():
    ap = argparse.ArgumentParser(description="serving benchmark (continuous batching vs plain one at a time)")
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--cap", type=float, default=40e9, help="device-memory arena in bytes")
    ap.add_argument("--rates", default="0.5,0.8,1.1", help="arrival rates as multiples of the measured capacity")
    ap.add_argument("--capacity-requests", type=int, default=2000,
                    help="requests of the mix (a prefix) served all at once to measure the capacity")
    ap.add_argument("--plain-per-class", type=int, default=6,
                    help="requests per operator class whose plain one-at-a-time service time is measured at full T "
                         "(0: not measured)")
    ap.add_argument("--capacity", type=float, default=0.0,
                    help="use this capacity (requests/s, from an earlier run) instead of measuring it")
    args = ap.parse_args()
    import torch

    from . import stencil as S
    cap = int(args.cap)
    reqs = request_mix(args.requests)
    ex = GpuExecutor(args.slots, cap)
    t0 = time.perf_counter()
    prepare(ex, reqs)
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    # capacity of this server: a prefix of the mix, everything arriving at once
    out = {"requests": args.requests, "slots": args.slots, "arena_gb": cap / 1e9, "prepare_s": round(prep_s, 1),
           "rates": []}
    if args.capacity > 0:
        capacity = args.capacity
        out["capacity_given_req_s"] = capacity
    else:
        head = [Request(r.rid, r.method, r.dim, r.shape, r.ext, r.T, r.seed) for r in reqs[:args.capacity_requests]]
        sat = Server(ex, args.slots, cap).serve(head).summary()
        capacity = sat["req_per_s"]
        out["saturated"] = dict(sat, requests=len(head))
    for m in [float(x) for x in args.rates.split(",")]:
        rate = m * capacity
        poisson_arrivals(reqs, rate)
        st = Server(ex, args.slots, cap).serve(reqs).summary()
        out["rates"].append({"multiple_of_capacity": m, "rate_req_s": round(rate, 3), "ours": st})
    ex.close()
    if args.plain_per_class <= 0:
        print(json.dumps(out))
        return
    # the plain kernels, one request at a time: service times measured at full T on a stratified sample,
    # a per-class linear model (seconds = a + b * updates) for the rest, FIFO at the same arrival times
    sample = stratified_sample(reqs, args.plain_per_class)
    secs = service_times(sample, plan=S.STENCIL_KERNEL_PLAIN)
    model = fit_service_model(sample, secs)
    measured = {r.rid: s for r, s in zip(sample, secs)}
    svc = [measured.get(r.rid, model[r.cls][0] + model[r.cls][1] * r.updates) for r in reqs]
    out["plain_one_at_a_time"] = {
        "sample": len(sample), "measured_full_T": True, "capacity_req_s": round(len(reqs) / sum(svc), 4),
        "model_s_per_update": {"%d/%d/%d" % c: v for c, v in model.items()},
        "sample_seconds_total": round(sum(secs), 2)}
    for entry in out["rates"]:
        poisson_arrivals(reqs, entry["rate_req_s"])
        lat = np.array(fifo_one_at_a_time([r.arrival for r in reqs], svc)) * 1e3
        entry["plain_one_at_a_time"] = {"p50_ms": round(float(np.percentile(lat, 50)), 1),
                                        "p99_ms": round(float(np.percentile(lat, 99)), 1)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
