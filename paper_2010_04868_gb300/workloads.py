"""The benchmark workloads, runnable one at a time with a chosen kernel family.

    python -m paper_2010_04868_gb300.workloads --config NAME [--kernel auto|plain|blocked|wavefront|diamond|stream]
                                               [--T STEPS] [--reps N] [--tb TB] [--tile A,B,C]
                                               [--ext E0,E1,...]

Prints one JSON line per configuration: GStencil/s (point updates per second),
the FP64-operation rate against the FP64 pipe's measured peak, and the
algorithmic HBM bandwidth of one-pass-per-step execution. Inputs are the
seeded synthetic grids of the recipes below (uniform [0, 1) values, seeded
positive weights normalised to sum 1); they stand in for the synthetic
benchmarks of the paper's Table 1.

Configurations (name: stencil, grid, T, boundary):
  heat1d      Jacobi 1D 3-point, weights (1/4, 1/2, 1/4), N = 65536, T = 256, zero halo
  jacobi2d5   Jacobi 2D 5-point star, 4096^2, T = 1000, zero halo
  jacobi2d9   Jacobi 2D 9-point box, 4096^2, T = 1000, zero halo
  gs2d5       Gauss-Seidel 2D 5-point, 4096^2, T = 200, zero halo
  gs1d3       Gauss-Seidel 1D 3-point, N = 2^24, T = 200, zero halo
  jacobi3d7   Jacobi 3D 7-point star, 512^3, T = 100, periodic
  jacobi3d27  Jacobi 3D 27-point box, 512^3, T = 100, periodic
  gs3d7       Gauss-Seidel 3D 7-point, 512^3, T = 100, periodic
  jacobi1d5   Jacobi 1D 5-point (radius 2), N = 2^24, T = 100, zero halo
  jacobi2d9s  Jacobi 2D 9-point star (radius 2), 4096^2, T = 200, zero halo
  jacobi3d13  Jacobi 3D 13-point star (radius 2), 256^3, T = 100, zero halo
  gs2d9s      Gauss-Seidel 2D 9-point star (radius 2), 4096^2, T = 100, zero halo
  jacobi2d5v  Jacobi 2D 5-point, per-point weights (a coefficient field), 4096^2, T = 200, zero halo
  gs2d5v      Gauss-Seidel 2D 5-point, per-point weights, 4096^2, T = 200, zero halo
  gs1d3v      Gauss-Seidel 1D 3-point, per-point weights, N = 2^24, T = 200, zero halo
  jacobi3d7v  Jacobi 3D 7-point, per-point weights, 256^3, T = 100, periodic
              (fields: inputs.normalized_field, positive and summing to about 1 at each point)
  batch3d     jacobi3d7 + jacobi3d27 + gs3d7 in one stencil_run_batch call (one persistent launch
              replayed from a CUDA graph), against the same three run one after another
  life        Game of Life B2S23 (Section 3.4), 8000^2 cells, T = 2000 (the paper's Table 1 size),
              dead boundary, seeded cells of density 1/2; --tb sets the steps per launch
  lcs         LCS (Section 3.4) of two seeded sequences of 200000 symbols over 4 letters (the paper's
              Table 1 size); --kernel dp or bits (default: both)
"""
from __future__ import annotations

import argparse
import json

from . import inputs

_PIPE = {}


def pipe_peak_gops(sm_mhz):
    """FP64 lane operations per second (in G) of this GPU at sm_mhz: the SM count read from the
    device times the lane operations per SM clock that the FP64 pipe micro-benchmark
    (peak/fp64_peak, built by build.build_probe) measures on it."""
    if "ops" not in _PIPE:
        import subprocess

        import torch

        from . import build as _b
        out = subprocess.run([_b.build_probe()], capture_output=True, text=True, timeout=120).stdout
        rows = [json.loads(ln) for ln in out.splitlines() if ln.startswith("{") and "fp64_lane_ops_per_sm_clk" in ln]
        if not rows:
            raise RuntimeError("FP64 probe printed no result: %s" % out[-300:])
        _PIPE["ops"] = float(rows[-1]["fp64_lane_ops_per_sm_clk"])
        _PIPE["nsm"] = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return _PIPE["ops"] * _PIPE["nsm"] * sm_mhz / 1e3

CONFIGS = {
    # name: (dim, shape, method, ext, T, bc, weights seed offset or explicit weights)
    "heat1d": (1, 0, 0, (65536,), 256, 0, [0.25, 0.5, 0.25]),
    "jacobi2d5": (2, 0, 0, (4096, 4096), 1000, 0, 105),
    "jacobi2d9": (2, 1, 0, (4096, 4096), 1000, 0, 109),
    "gs2d5": (2, 0, 1, (4096, 4096), 200, 0, 105),
    "gs1d3": (1, 0, 1, (1 << 24,), 200, 0, 103),
    "jacobi3d7": (3, 0, 0, (512, 512, 512), 100, 1, 207),
    "jacobi3d27": (3, 1, 0, (512, 512, 512), 100, 1, 227),
    "gs3d7": (3, 0, 1, (512, 512, 512), 100, 1, 208),
    # higher order (radius 2)
    "jacobi1d5": (1, 0, 0, (1 << 24,), 100, 0, 305),
    "jacobi2d9s": (2, 0, 0, (4096, 4096), 200, 0, 309),
    "jacobi3d13": (3, 0, 0, (256, 256, 256), 100, 0, 313),
    "gs2d9s": (2, 0, 1, (4096, 4096), 100, 0, 319),
    # variable coefficients (the weights come from a per-point field; the seed offset seeds the field)
    "jacobi2d5v": (2, 0, 0, (4096, 4096), 200, 0, 405),
    "gs2d5v": (2, 0, 1, (4096, 4096), 200, 0, 415),
    "gs1d3v": (1, 0, 1, (1 << 24,), 200, 0, 403),
    "jacobi3d7v": (3, 0, 0, (256, 256, 256), 100, 1, 407),
}

FIELD = {"jacobi2d5v", "gs2d5v", "gs1d3v", "jacobi3d7v"}

RADIUS = {"jacobi1d5": 2, "jacobi2d9s": 2, "jacobi3d13": 2, "gs2d9s": 2}

KERNELS = {"auto": 0, "plain": 1, "blocked": 2, "wavefront": 3, "diamond": 4, "stream": 5}


def k_points(dim, shape, r=1):
    return 2 * dim * r + 1 if (shape == 0 or dim == 1) else (2 * r + 1) ** dim


def config_weights(name):
    dim, shape, _, _, _, _, w = CONFIGS[name]
    if isinstance(w, list):
        return list(w)
    return list(inputs.normalized_weights(inputs.SEED_BASE + w, k_points(dim, shape, RADIUS.get(name, 1))))


def config_field(name, ext=None):
    """The configuration's weight field, on its own extents or on ext (a smaller case)."""
    dim, shape, _, ext0, _, _, seed = CONFIGS[name]
    return inputs.normalized_field(inputs.SEED_BASE + seed, k_points(dim, shape, RADIUS.get(name, 1)),
                                   ext0 if ext is None else ext)


def config_grid(name):
    ext = CONFIGS[name][3]
    return inputs.grid(inputs.SEED_BASE + 10 + list(CONFIGS).index(name), ext)


def run(name, kernel="auto", T=None, reps=2, tb=0, tile=(0, 0, 0), sm_mhz=2070.0, ext=None):
    import torch

    from . import stencil as S
    dim, shape, method, ext0, T0, bc, _ = CONFIGS[name]
    ext = tuple(ext) if ext else ext0
    r = RADIUS.get(name, 1)
    T = T0 if T is None else T
    u0 = torch.from_numpy(config_grid(name) if ext == ext0 else inputs.grid(inputs.SEED_BASE + 10, ext)).cuda()
    st = S.Stencil(dim, shape, r, config_weights(name), method, bc)
    if name in FIELD:
        st.set_field(torch.from_numpy(config_field(name, ext)).cuda())
    if kernel != "auto":
        st.set_plan(KERNELS[kernel], tb, tile)
    u = u0.clone()
    scratch = torch.empty_like(u) if method == 0 else None
    st.run(u, T, scratch)                       # warm-up (and tuning for the automatic plan)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        u.copy_(u0)
        n0 = S.stencil_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        st.run(u, T, scratch)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, S.stencil_launch_count() - n0)
    rc = st.status()
    st.close()
    if rc != 0:
        raise RuntimeError("%s: %s" % (name, S.strerror(rc)))
    npts = 1
    for e in ext:
        npts *= e
    ms, launches = best
    gst = npts * T / ms / 1e6
    k = k_points(dim, shape, r)
    peak = pipe_peak_gops(sm_mhz)
    # one pass per step moves the grid in and out, plus the K field planes with per-point weights
    bytes_pt = 16 + (8 * k if name in FIELD else 0)
    return {"config": name, "kernel": kernel, "r": r, "T": T, "ms": round(ms, 3), "gstencil_s": round(gst, 3),
            "launches": launches, "fp64_gops": round(gst * k, 1), "fp64_frac_of_peak": round(gst * k / peak, 4),
            "hbm_gbs_one_pass_per_step": round(gst * bytes_pt, 1)}


# Integer operations per 32-cell word and step of the bit-sliced Life update, the unit of its ALU
# roofline: 4 full adders (2 three-input logic ops each) + 3 half adders (2 each) + the B2S23 rule (2)
# = 16 logic ops, plus the west and east alignment of the new row (one funnel shift each).
LIFE_OPS_PER_WORD = 18


def run_life(T=2000, tb=0, reps=2, ext=(8000, 8000)):
    import torch

    from . import life
    c0 = torch.from_numpy(inputs.cells(inputs.SEED_BASE + 500, ext, 0.5)).cuda()
    c = c0.clone()
    ws = torch.empty(life.life_workspace_bytes(ext), dtype=torch.uint8, device="cuda")
    life.run(c, T, tb=tb, workspace=ws)
    torch.cuda.synchronize()
    best = None
    from . import stencil as S
    for _ in range(reps):
        c.copy_(c0)
        n0 = S.stencil_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        life.run(c, T, tb=tb, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, S.stencil_launch_count() - n0)
    ms, launches = best
    cells = ext[0] * ext[1]
    words = ext[0] * ((ext[1] + 31) // 32)
    return {"config": "life", "tb": tb, "T": T, "ms": round(ms, 3), "gcell_updates_s": round(cells * T / ms / 1e6, 1),
            "launches": launches, "int_gops": round(words * T * LIFE_OPS_PER_WORD / ms / 1e6, 1),
            "live_fraction_after": round(float(c.float().mean()), 4)}


def run_lcs(kernel="bits", n=200000, sigma=4, reps=2):
    import torch

    from . import lcs
    from . import stencil as S
    kid = {"dp": lcs.LCS_KERNEL_DP, "bits": lcs.LCS_KERNEL_BITS}[kernel]
    A = torch.from_numpy(inputs.sequence(inputs.SEED_BASE + 700, n, sigma)).cuda()
    B = torch.from_numpy(inputs.sequence(inputs.SEED_BASE + 701, n, sigma)).cuda()
    ws = torch.empty(lcs.lcs_workspace_bytes(n, n, kid), dtype=torch.uint8, device="cuda")
    row = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    lcs.run(A, B, kid, row=row, workspace=ws)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        n0 = S.stencil_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        lcs.run(A, B, kid, row=row, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, S.stencil_launch_count() - n0)
    if lcs.lcs_status(ws.data_ptr()) != 0:
        raise RuntimeError("lcs: a bounded wait timed out")
    ms, launches = best
    return {"config": "lcs", "kernel": kernel, "n": n, "sigma": sigma, "ms": round(ms, 3),
            "gcell_updates_s": round(n * n / ms / 1e6, 1), "launches": launches, "lcs_length": int(row[-1])}


def run_batch3d(reps=2, ext=None, T=None):
    """The three 512^3 periodic problems batched, and the same three run separately (ext and T
    override the extents and the steps per problem: a smaller case of the same batch)."""
    import ctypes

    import torch

    from . import stencil as S
    names = ["jacobi3d7", "jacobi3d27", "gs3d7"]
    sts, us, scs, u0s = [], [], [], []
    for n in names:
        dim, shape, method, ext0, _, bc, _ = CONFIGS[n]
        e = tuple(ext) if ext else ext0
        u0 = torch.from_numpy(config_grid(n) if e == ext0 else inputs.grid(inputs.SEED_BASE + 10, e)).cuda()
        st = S.Stencil(dim, shape, 1, config_weights(n), method, bc)
        sts.append(st)
        u0s.append(u0)
        us.append(u0.clone())
        scs.append(torch.empty_like(u0) if method == 0 else None)
    Ts = [CONFIGS[n][4] if T is None else T for n in names]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    grids = [st.grid(u, sc) for st, u, sc in zip(sts, us, scs)]

    def timed(fn):
        best = None
        for _ in range(reps + 1):          # the first call prepares (tunes, captures the graph)
            for u, u0 in zip(us, u0s):
                u.copy_(u0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None or ms < best else best
        return best

    ms_batch = timed(lambda: S.stencil_run_batch([s.handle for s in sts], grids, Ts, stream))
    ms_solo = timed(lambda: [st.run(u, T, sc) for st, u, sc, T in zip(sts, us, scs, Ts)])
    for st in sts:
        if st.status() != 0:
            raise RuntimeError("batch3d: device status")
        st.close()
    npts = 1
    for e in us[0].shape:
        npts *= e
    upd = sum(npts * t for t in Ts)
    return {"config": "batch3d", "ext": list(us[0].shape), "T": Ts, "ms_batch": round(ms_batch, 2), "ms_separate": round(ms_solo, 2),
            "gstencil_s_batch": round(upd / ms_batch / 1e6, 3), "gstencil_s_separate": round(upd / ms_solo / 1e6, 3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="all")
    ap.add_argument("--kernel", default="auto", choices=list(KERNELS) + ["dp", "bits"])
    ap.add_argument("--T", type=int, default=None)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tb", type=int, default=0)
    ap.add_argument("--tile", default="0,0,0")
    ap.add_argument("--ext", default="", help="override the grid extents, e.g. 1048576 or 512,512 (small cases)")
    a = ap.parse_args()
    names = list(CONFIGS) + ["batch3d", "life", "lcs"] if a.config == "all" else a.config.split(",")
    tile = tuple(int(x) for x in a.tile.split(","))
    for n in names:
        if n == "batch3d":
            ext = tuple(int(x) for x in a.ext.split(",")) if a.ext else None
            print(json.dumps(run_batch3d(a.reps, ext=ext, T=a.T)), flush=True)
        elif n == "life":
            print(json.dumps(run_life(a.T or 2000, a.tb, a.reps)), flush=True)
        elif n == "lcs":
            for k in (("dp", "bits") if a.kernel == "auto" else (a.kernel,)):
                print(json.dumps(run_lcs(k, reps=a.reps)), flush=True)
        else:
            ext = tuple(int(x) for x in a.ext.split(",")) if a.ext else None
            print(json.dumps(run(n, a.kernel, a.T, a.reps, a.tb, tile, ext=ext)), flush=True)


if __name__ == "__main__":
    main()
