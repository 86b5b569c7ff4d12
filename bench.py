"""Benchmark of the cutting voxel projector on the 512^3 x 496-view cone-beam workload.

One step = forward projection b = A x and backprojection x' = A^T y of both variants
(near-exact and relaxed), i.e. every row of the hot path: per-view geometry is set up
once at plan creation, then voxel footprints, column cuts, exact and relaxed row cuts,
accumulation, pixel factors and the gather adjoint run inside each step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl kct|reference]

Prints one JSON line (rank 0). `value` is whole-job voxel-views per second of P + BP:
each step processes 2 * (512^3 * 496) voxel-view units (one P+BP per variant); N ranks
run N independent replicas (the path needs no exchange between GPUs).
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cvp512"
METRIC = "CVP project+backproject Gvoxel·views/s at 512³×496 views; CGLS time-to-1e-3 residual"
UNIT = "Gvoxel·views/s"

# Per-kernel counts from one ncu capture of each projector kernel on the benchmark geometry
# restricted to 8 of its views (python bench.py --profile-case cvp512 --views 8 ...):
#   flop_per_vv  FP32 operations (thread-level FADD + FMUL + 2 FFMA, the paired FADD2 / FMUL2 /
#                FFMA2 counted as 2 / 2 / 4) per voxel-view,
#   warp_per_vv  warp instructions issued per voxel-view, simt: active lanes per instruction / 32,
#   dram_8       DRAM bytes read + written by that 8-view launch.
# A full 496-view launch processes 62x the voxel-views; the forward kernel re-reads the
# volume once per chunk of views (the capture's 8 views are one chunk) and adds one projection
# per view, the adjoint reads one projection tile per view and writes the volume once, so
# traffic is scaled as below.
NCU = {
    "exact project": {"flop_per_vv": 732.6, "warp_per_vv": 79.6, "simt": 0.78,
                      "dram_read_8": 5.75e8, "dram_write_8": 3.01e7},
    "exact backproject": {"flop_per_vv": 818.2, "warp_per_vv": 84.6, "simt": 0.80,
                          "dram_read_8": 5.23e7, "dram_write_8": 4.89e8},
    "relaxed project": {"flop_per_vv": 186.1, "warp_per_vv": 23.6, "simt": 0.77,
                        "dram_read_8": 5.71e8, "dram_write_8": 2.93e7},
    "relaxed backproject": {"flop_per_vv": 233.9, "warp_per_vv": 30.3, "simt": 0.77,
                            "dram_read_8": 4.55e7, "dram_write_8": 4.89e8},
}


def full_launch_traffic(name: str, nviews: int, chunk: int = 16) -> float:
    c = NCU[name]
    if name.endswith("backproject"):      # per-view tile reads scale, the volume write does not
        return c["dram_read_8"] * nviews / 8 + c["dram_write_8"]
    chunks = (nviews + chunk - 1) // chunk  # volume re-read per chunk of views, writes per view
    return c["dram_read_8"] * chunks + c["dram_write_8"] * nviews / 8


def default_args():
    """The arguments of a run without command-line options."""
    return parse([])


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kct", choices=["kct", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--scaling", default="cos", choices=["cos", "exact"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cgls", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default forward view chunk (16)")
    ap.add_argument("--accuracy", action="store_true",
                    help="compare both variants and scalings with supersampled ray integration (K = 32, 64) and exit")
    ap.add_argument("--convs", action="store_true",
                    help="time the warm-start U-Net's tensor-core convolutions at 128^3 and exit")
    ap.add_argument("--paper-geometries", action="store_true",
                    help="time P and BP at the geometries of the paper's Tables I and II and exit")
    ap.add_argument("--throughput", default=None, metavar="WORKLOAD",
                    help="time P and BP of both variants at one workload (with nonzero pairs per second) and exit")
    ap.add_argument("--batch", action="store_true",
                    help="batched operator: 8 perfusion frames of 256^3 through 248 views, P + BP captured in a "
                         "CUDA graph and replayed, and exit")
    ap.add_argument("--cgls-max-iter", type=int, default=200)
    ap.add_argument("--profile-case", default=None, metavar="WORKLOAD",
                    help="run one projector call on a sub-sampled workload (for ncu captures) and exit")
    ap.add_argument("--variant", default="exact", choices=["exact", "relaxed"])
    ap.add_argument("--direction", default="fwd", choices=["fwd", "bwd"])
    ap.add_argument("--views", type=int, default=32)
    return ap.parse_args(argv)


def run_profile_case(args):
    """Two untimed calls and one timed call of one direction of one variant on the first
    `--views` evenly spaced views of a workload: a small, self-contained case to capture
    with ncu (`-s 2 -c 1` skips the untimed launches of the captured kernel)."""
    import torch

    from paper_2110_09841_b300 import inputs
    from paper_2110_09841_b300.kct import Projector

    g = inputs.workload_geometry(args.profile_case)
    step = max(1, g.nviews // args.views)
    g = g.subset_views(list(range(0, g.nviews, step))[:args.views])
    x = inputs.workload_phantom(args.profile_case, device="cuda")
    y = inputs.uniform_projections(g.proj_shape, 3, device="cuda")
    A = Projector(g, args.variant, args.scaling)
    call = (lambda: A.project(x)) if args.direction == "fwd" else (lambda: A.backproject(y))
    call()
    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    call()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print(json.dumps({"case": args.profile_case, "views": g.nviews, "variant": args.variant,
                      "direction": args.direction, "ms": ms, "gvv_s": g.voxel_views / (ms / 1e3) / 1e9}))


E2E_STEPS = 1      # steps of the end-to-end measurement (after one untimed end-to-end step)


def max_over_ranks(ms: float, device) -> float:
    """The slowest rank's time: every rank returns the maximum over the process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gvv_s(units_per_step: float, steps: int, ms: float, world: int) -> float:
    """Whole-job throughput: every replica processes units_per_step voxel-views per step."""
    return world * units_per_step * steps / (ms / 1e3) / 1e9


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clock and throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [[p.strip() for p in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = max((num(r[2]) for r in rows if num(r[2]) is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in rows for q in range(4) if r[5 + q].lower() == "active"})
        load = [v for v in sm if mx and v > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


def probe_fp32_tflops():
    """FP32 FMA throughput measured on this GPU by the probe kernel (2 FLOP per FMA)."""
    import ctypes

    from paper_2110_09841_b300 import build

    lib = ctypes.CDLL(build.PROBE_LIB)
    lib.kct_probe_fp32.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_float)]
    lib.kct_probe_fp32.restype = ctypes.c_int
    flops, ms = ctypes.c_double(0.0), ctypes.c_float(0.0)
    rc = lib.kct_probe_fp32(8, 20000, ctypes.byref(flops), ctypes.byref(ms))
    return flops.value / 1e12 if rc == 0 else None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(geom, seconds: float, seed: int = 5):
    """The FP64 oracle's adjoint on randomly drawn voxels (all views), time-bounded.
    Returns (voxel-views per second for P+BP, sample description, threads). The forward
    projection clips the same voxel-pixel pairs, so one P+BP costs twice the adjoint."""
    import numpy as np

    import oracle
    from paper_2110_09841_b300 import inputs

    threads = oracle.num_threads()
    y = inputs.uniform_projections(geom.proj_shape, seed).numpy()
    rng = np.random.default_rng(seed)
    done = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        vox = np.stack([rng.integers(0, geom.nz, threads), rng.integers(0, geom.ny, threads),
                        rng.integers(0, geom.nx, threads)], axis=1)
        oracle.backproject_voxels(geom, y, vox)
        done += threads
    dt = time.perf_counter() - t0
    return (done * geom.nviews / dt / 2.0,
            f"FP64 adjoint of {done} random voxels x {geom.nviews} views in {dt:.1f} s; P+BP = 2 x adjoint cost",
            threads)


WORKLOAD_DESC = ("cvp512: 512^3 voxels @ 0.25 mm, 496 views / 360 deg, SID 400 / SDD 600 mm, "
                 "1232x960 detector @ 0.154 mm, seeded 40-ellipsoid phantom")


CGLS_DESC = ("cgls128: 128^3 voxels @ 0.5 mm, 180 views / 360 deg, SID 750 / SDD 1200 mm, 256x192 detector "
             "@ 0.8 mm, seeded 20-ellipsoid phantom, Poisson noise at 1e5 photons per pixel, CGLS from 0")


def run_cgls(dev, scaling: str, max_iter: int, tol: float = 1e-3):
    """Time to the normal-equation residual |A^T(b - A x)| / |A^T b| <= tol with kct_cgls, for
    both variants, on noisy projections of a seeded phantom made with the same variant.
    The timed region is the whole kct_cgls call (start, steps, per-step residual reads); for the
    relaxed variant also from the learned warm start (run_warm_start)."""
    import torch

    from paper_2110_09841_b300 import inputs
    from paper_2110_09841_b300.kct import Projector

    g = inputs.workload_geometry("cgls128")
    truth = inputs.workload_phantom("cgls128", device=dev)
    out = {"workload": CGLS_DESC, "tol": tol, "max_iter": max_iter}
    for v in ("exact", "relaxed"):
        A = Projector(g, v, scaling)
        b = inputs.poisson_log_data(A.project(truth), 1e5, 77)
        ws = A.cgls_workspace()
        x = torch.empty(g.vol_shape, dtype=torch.float32, device=dev)
        A.cgls(b, max_iter=2, tol=0.0, out=x, workspace=ws)          # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x, info = A.cgls(b, max_iter=max_iter, tol=tol, out=x, workspace=ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        k = info["iterations"]
        out[v] = {"iterations": k, "converged": info["converged"], "time_s": ms / 1e3,
                  "ms_per_iteration": ms / max(k, 1), "normal_residual": float(info["normal"][-1]),
                  "data_residual": float(info["data"][-1]),
                  "rel_error_vs_phantom": float((x - truth).norm() / truth.norm())}
        if v == "relaxed":
            out["relaxed_warm_start"] = run_warm_start(A, b, truth, ws, max_iter, tol)
    return out


def run_warm_start(A, b, truth, ws, max_iter: int, tol: float):
    """CGLS from the learned warm start (the stored U-Net, trained for this geometry with the
    relaxed operator): the timed region is the backprojection of b (the network input, reused by
    CGLS as A^T b), the network's inference and CGLS from its output to the same residual."""
    import torch

    from paper_2110_09841_b300 import warmstart
    from paper_2110_09841_b300.unet import UNet3D

    path = os.path.join(ROOT, "paper_2110_09841_b300", "weights", "unet_cgls128.pt")
    if not os.path.exists(path):
        return None
    model = warmstart.load_model(UNet3D().cuda(), path)
    ones = torch.ones(A.geom.vol_shape, device="cuda")
    norm = A.backproject(A.project(ones))
    norm.clamp_(min=1e-6 * float(norm.max()))
    x = torch.empty(A.geom.vol_shape, dtype=torch.float32, device="cuda")

    def solve():
        atb = A.backproject(b)
        with torch.no_grad():
            x0 = model((atb / norm)[None])[0].contiguous()
        return A.cgls(b, x0=x0, max_iter=max_iter, tol=tol, out=x, workspace=ws, atb=atb)

    solve()                                                      # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    x, info = solve()
    e1.record()
    torch.cuda.synchronize()
    k = info["iterations"]
    return {"iterations": k, "converged": info["converged"], "time_s": e0.elapsed_time(e1) / 1e3,
            "start_normal_residual": float(info["normal"][0]), "normal_residual": float(info["normal"][-1]),
            "rel_error_vs_phantom": float((x - truth).norm() / truth.norm()),
            "network": "3D U-Net 16/32/64/128, BF16 tcgen05 convolutions, weights/unet_cgls128.pt"}


def bench_config(args, world: int) -> dict:
    """The workload description both arms report."""
    return {"workload": WORKLOAD_DESC, "step": "project + backproject, near-exact and relaxed variants",
            "scaling": args.scaling, "parallelism": f"replicas x{world}",
            "l2": "inputs (0.54 GB volume, 2.35 GB projections) larger than L2; no flush"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2110_09841_b300 import inputs

    geom = inputs.workload_geometry(args.workload)
    for _ in range(args.warmup):
        cpu_baseline(geom, 1.0)
    vals, desc, threads = [], "", 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, desc, threads = cpu_baseline(geom, 5.0)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": bench_config(args, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_kct(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2110_09841_b300 import build, inputs
    from paper_2110_09841_b300.kct import Projector

    build.build()
    geom = inputs.workload_geometry(args.workload)
    x = inputs.workload_phantom(args.workload, device=dev)
    y = inputs.uniform_projections(geom.proj_shape, 2024, device=dev)
    variants = ("exact", "relaxed")
    ops = {v: Projector(geom, v, args.scaling) for v in variants}
    # the forward view chunk picked by the plan's own autotuner (kct_plan_autotune), before any
    # timing; the chunks are reported in the JSON line
    tuned = {}
    if not args.no_autotune:
        scratch = torch.empty(geom.proj_shape, dtype=torch.float32, device=dev)
        for v in variants:
            tuned[v] = ops[v].autotune(x, scratch)[0]
        del scratch
    b = {v: torch.empty(geom.proj_shape, dtype=torch.float32, device=dev) for v in variants}
    xb = {v: torch.empty(geom.vol_shape, dtype=torch.float32, device=dev) for v in variants}
    stream = torch.cuda.current_stream()

    def step(ev=None):
        for v in variants:
            if ev is not None:
                ev[v][0].record(stream)
            ops[v].project(x, out=b[v])
            if ev is not None:
                ev[v][1].record(stream)
            ops[v].backproject(y, out=xb[v])
            if ev is not None:
                ev[v][2].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
            torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    for v in variants:
        assert ops[v].device_error() == 0, "device-side footprint check failed"
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    events = [{v: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for v in variants}
              for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    t_start.record(stream)
    for s in range(args.steps):
        step(events[s])
    t_end.record(stream)
    barrier()
    clocks = sampler.stop()
    total_ms = t_start.elapsed_time(t_end)
    per = {v: {"project_ms": statistics.median(e[v][0].elapsed_time(e[v][1]) for e in events),
               "backproject_ms": statistics.median(e[v][1].elapsed_time(e[v][2]) for e in events)}
           for v in variants}
    total_ms = max_over_ranks(total_ms, dev)
    units_per_step = 2 * geom.voxel_views          # one P+BP per variant
    value = aggregate_gvv_s(units_per_step, args.steps, total_ms, world)
    for v in variants:
        p = per[v]
        p["view_chunk"] = ops[v].view_chunk
        p["p_bp_gvv_s"] = geom.voxel_views / ((p["project_ms"] + p["backproject_ms"]) / 1e3) / 1e9
        p["nnz_pairs"] = ops[v].count_pairs()
        p["nnz_pairs_per_s_p_bp"] = 2 * p["nnz_pairs"] / ((p["project_ms"] + p["backproject_ms"]) / 1e3)

    # end to end through the public API from pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        xh = x.cpu().pin_memory()
        yh = y.cpu().pin_memory()
        bh = {v: torch.empty(geom.proj_shape, dtype=torch.float32).pin_memory() for v in variants}
        xbh = {v: torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory() for v in variants}
        xd = torch.empty_like(x)
        yd = torch.empty_like(y)

        def e2e_step():
            xd.copy_(xh, non_blocking=True)
            yd.copy_(yh, non_blocking=True)
            for v in variants:
                ops[v].project(xd, out=b[v])
                ops[v].backproject(yd, out=xb[v])
                bh[v].copy_(b[v], non_blocking=True)
                xbh[v].copy_(xb[v], non_blocking=True)

        e2e_step()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(E2E_STEPS):
            e2e_step()
        e1.record(stream)
        barrier()
        ems = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": aggregate_gvv_s(units_per_step, E2E_STEPS, ems, world), "unit": UNIT, "steps": E2E_STEPS,
               "h2d_bytes_per_step": (x.numel() + y.numel()) * 4,
               "d2h_bytes_per_step": len(variants) * (x.numel() + y.numel()) * 4}

    cgls = None if args.no_cgls else run_cgls(dev, args.scaling, args.cgls_max_iter)

    if rank != 0:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()
        return

    # roofline of the dominant kernel; the projector kernels are bound by FP32 ALU work
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz", 2032.0)
    peak_tflops = sms * 128 * 2 * max_mhz * 1e6 / 1e12
    dom_v, dom_k = max(((v, k) for v in variants for k in ("project_ms", "backproject_ms")),
                       key=lambda q: per[q[0]][q[1]])
    dom_ms = per[dom_v][dom_k]
    name = f"{dom_v} {dom_k[:-3]}"
    flop_vv = NCU[name]["flop_per_vv"] if args.workload == WORKLOAD else None
    achieved = (flop_vv * geom.voxel_views / (dom_ms / 1e3) / 1e12) if flop_vv else None
    traffic = full_launch_traffic(name, geom.nviews, ops[dom_v].view_chunk) if args.workload == WORKLOAD else None
    fp32_probe = probe_fp32_tflops()
    # the same kernel against the instruction-issue limit (4 warp instructions per SM and cycle)
    wpv = NCU[name]["warp_per_vv"] if args.workload == WORKLOAD else None
    clk = (clocks.get("sm_mhz") or max_mhz) * 1e6
    issue = ({"warp_inst_per_voxel_view": wpv, "achieved_per_s": wpv * geom.voxel_views / (dom_ms / 1e3),
              "peak_per_s": sms * 4 * clk, "frac": wpv * geom.voxel_views / (dom_ms / 1e3) / (sms * 4 * clk),
              "simt_efficiency": NCU[name]["simt"], "basis": "ncu warp instruction count x event-timed launch"}
             if wpv else None)
    # the peak is the FP32 FMA rate measured on this GPU by the probe kernel (at the running clock);
    # the derived SMs x 128 lanes x 2 FLOP x max clock figure is kept beside it
    peak = fp32_probe if fp32_probe else peak_tflops
    roofline = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "peak_derived_tflops": peak_tflops, "issue": issue,
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu, 8-view capture scaled to the full launch)",
                "launch_ms": dom_ms, "flop_per_voxel_view": flop_vv,
                "peak_basis": ("measured: FP32 FMA probe kernel on this GPU" if fp32_probe else
                               f"derived (probe unavailable): {sms} SMs x 128 lanes x 2 FLOP x {max_mhz:.0f} MHz")}

    cb_val, cb_desc, cb_threads = cpu_baseline(geom, 10.0)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32",
           "data": "synthetic (seeded ellipsoid phantom; U[0,1) projections for the adjoint)",
           "config": bench_config(args, world),
           "variants": per, "roofline": roofline,
           "cpu_baseline": {"value": cb_val / 1e9, "unit": UNIT, "cores": cb_threads, "kind": "oracle",
                            "sample": cb_desc},
           "e2e": e2e, "gpu_launches": 4 * args.steps, "clocks": clocks, "cgls": cgls}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


# The paper's own projector timings at its Table I / II geometries (Gvoxel-views/s from its
# per-call seconds; Radeon VII, FP64 near-exact with elevation correction, FP32 relaxed).
PAPER_GVV_S = {
    "long2010": {"exact": {"project": 0.615, "backproject": 1.226}, "relaxed": {"project": 1.964, "backproject": 4.646},
                 "source": "Sec. IV-A Table I, AMD Radeon VII"},
    "pfeiffer2021": {"exact": {"project": 0.0746, "backproject": 0.1190},
                     "relaxed": {"project": 0.224, "backproject": 0.409},
                     "source": "Sec. IV-A Table II, AMD Radeon VII"},
}


def time_calls(call, reps: int = 3) -> float:
    """ms per call: one warm-up call, then reps calls between CUDA events on the current stream."""
    import torch

    call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_throughput(args):
    """P and BP of both variants at one workload (seeded phantom, U[0,1) projections; one
    warm-up and three timed calls each, CUDA events), with the number of nonzero voxel-pixel
    pairs counted on the device and the pairs per second it implies."""
    import torch

    from paper_2110_09841_b300 import build, inputs
    from paper_2110_09841_b300.kct import Projector

    build.build()
    name = args.throughput
    g = inputs.workload_geometry(name)
    x = inputs.workload_phantom(name, device="cuda")
    y = inputs.uniform_projections(g.proj_shape, 2024, device="cuda")
    out = {"mode": "throughput", "workload": name, "voxel_views": g.voxel_views, "scaling": args.scaling,
           "unit": UNIT, "results": {}}
    for v in ("exact", "relaxed"):
        A = Projector(g, v, args.scaling)
        b = torch.empty(g.proj_shape, device="cuda")
        xb = torch.empty(g.vol_shape, device="cuda")
        nnz = A.count_pairs()
        r = {"nnz_pairs": nnz, "pairs_per_voxel_view": nnz / g.voxel_views}
        for d, call in (("project", lambda: A.project(x, out=b)), ("backproject", lambda: A.backproject(y, out=xb))):
            ms = time_calls(call)
            r[d] = {"ms": ms, "gvv_s": g.voxel_views / (ms / 1e3) / 1e9, "gpairs_s": nnz / (ms / 1e3) / 1e9}
        assert A.device_error() == 0
        out["results"][v] = r
    print(json.dumps(out), flush=True)


def run_batch(args):
    """The batched operator: 8 perfusion-like frames of 256^3 (one seeded phantom plus five
    vessel ellipsoids with Gaussian bolus curves) through 248 shared views over 200 deg onto a
    616x480 detector. The forward view chunk is autotuned on one frame; then one batched
    projection and one batched backprojection of its result (one launch each) are captured in
    a CUDA graph, which is replayed: time per replay from CUDA events around 5 replays after a
    warm-up replay. Throughput counts 8 frames x 256^3 voxels x 248 views per direction."""
    import torch

    from paper_2110_09841_b300 import build, inputs
    from paper_2110_09841_b300.kct import Projector

    build.build()
    g = inputs.workload_geometry("cvp256")
    nb = 8
    frames = inputs.perfusion_frames(g, 4004, frames=nb, device="cuda")
    proj = torch.empty((nb,) + g.proj_shape, device="cuda")
    back = torch.empty((nb,) + g.vol_shape, device="cuda")
    units = nb * g.voxel_views
    out = {"mode": "batch", "workload": "8 perfusion frames of 256^3 @ 0.5 mm, 248 views / 200 deg, SID 750 / "
           "SDD 1200 mm, 616x480 detector @ 0.616 mm", "scaling": args.scaling, "unit": UNIT, "results": {}}
    for v in ("exact", "relaxed"):
        A = Projector(g, v, args.scaling)
        chunk, tune_ms = A.autotune(frames[0].contiguous())
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            A.project_batch(frames, out=proj)
            A.backproject_batch(proj, out=back)
        torch.cuda.current_stream().wait_stream(s)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            A.project_batch(frames, out=proj)
            A.backproject_batch(proj, out=back)
        ms = time_calls(graph.replay, reps=5)
        # eager timing of each direction, and the replay checked against eager calls
        ms_p = time_calls(lambda: A.project_batch(frames, out=proj))
        ms_b = time_calls(lambda: A.backproject_batch(proj, out=back))
        graph.replay()
        torch.cuda.synchronize()
        ref = A.backproject_batch(A.project_batch(frames))
        agree = float((back - ref).abs().max() / ref.abs().max())
        assert A.device_error() == 0
        out["results"][v] = {"view_chunk": chunk, "graph_replay_ms": ms, "gvv_s_p_plus_bp": 2 * units / (ms / 1e3) / 1e9,
                             "project_ms": ms_p, "project_gvv_s": units / (ms_p / 1e3) / 1e9,
                             "backproject_ms": ms_b, "backproject_gvv_s": units / (ms_b / 1e3) / 1e9,
                             "replay_vs_eager_max_rel": agree}
    print(json.dumps(out), flush=True)


def run_paper_geometries(args):
    """P and BP of both variants at the paper's Table I and II geometries (one warm-up and
    one timed call each, CUDA events), next to the paper's published throughput."""
    import torch

    from paper_2110_09841_b300 import build, inputs
    from paper_2110_09841_b300.kct import Projector

    build.build()
    out = {"mode": "paper geometries", "unit": UNIT, "scaling": args.scaling, "results": {}}
    for name in ("long2010", "pfeiffer2021"):
        g = inputs.workload_geometry(name)
        x = inputs.workload_phantom(name, device="cuda")
        y = inputs.uniform_projections(g.proj_shape, 2024, device="cuda")
        res = {"voxel_views": g.voxel_views, "paper": PAPER_GVV_S[name]}
        for v in ("exact", "relaxed"):
            A = Projector(g, v, args.scaling)
            b = torch.empty(g.proj_shape, device="cuda")
            xb = torch.empty(g.vol_shape, device="cuda")
            r = {}
            for d, call in (("project", lambda: A.project(x, out=b)), ("backproject", lambda: A.backproject(y, out=xb))):
                call()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                call()
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                r[d] = {"ms": ms, "gvv_s": g.voxel_views / (ms / 1e3) / 1e9,
                        "x_paper": g.voxel_views / (ms / 1e3) / 1e9 / PAPER_GVV_S[name][v][d]}
            r["nnz_pairs"] = A.count_pairs()
            res[v] = r
        out["results"][name] = res
    print(json.dumps(out), flush=True)


def run_convs(args):
    """Forward, input-gradient and weight-gradient convolutions of every layer shape of the
    warm-start U-Net at 128^3 (CUDA events, 2 warm-up and 5 timed calls each), as TFLOP/s
    against the measured BF16 dense peak."""
    import torch

    from paper_2110_09841_b300 import build, conv

    build.build()
    peak = measured_peaks().get("bf16_tflops") or 1800.0
    shapes = [  # (spatial edge, cin, cout) of the U-Net's convolutions (input padded to 16 channels)
        (128, 16, 16), (128, 32, 16), (64, 16, 32), (64, 32, 32), (64, 64, 32), (32, 32, 64), (32, 64, 64),
        (32, 128, 64), (16, 64, 128), (16, 128, 128)]
    rows = []
    g = torch.Generator(device="cuda").manual_seed(0)
    for (e, ci, co) in shapes:
        x = torch.randn((1, e, e, e, ci), device="cuda", generator=g).to(torch.bfloat16)
        w = (0.1 * torch.randn((co, 27, ci), device="cuda", generator=g)).to(torch.bfloat16)
        gy = torch.randn((1, e, e, e, co), device="cuda", generator=g).to(torch.bfloat16)
        flop = 2.0 * e ** 3 * 27 * ci * co
        r = {"edge": e, "cin": ci, "cout": co, "gflop": flop / 1e9}
        for name, call in (("fwd", lambda: conv.conv3d_fwd(x, w)), ("dgrad", lambda: conv.conv3d_dgrad(gy, w)),
                           ("wgrad", lambda: conv.conv3d_wgrad(x, gy))):
            for _ in range(2):
                call()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                call()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            r[name] = {"ms": ms, "tflops": flop / (ms / 1e3) / 1e12, "frac_of_bf16_peak": flop / (ms / 1e3) / 1e12 / peak}
        rows.append(r)
    assert int(conv.err_word("cuda").item()) == 0
    print(json.dumps({"mode": "convs", "bf16_peak_tflops": peak, "peak_basis": "MEASURED_PEAKS.json bf16_tflops (burst)",
                      "note": "wgrad times include the channels-first copies of its operands", "layers": rows}),
          flush=True)


def run_accuracy(args):
    """Accuracy of the CVP variants against supersampled ray integration (K x K rays per pixel,
    exact path lengths; equal weights for the cos scaling, solid-angle weights for the exact
    scaling) on 8 evenly spaced views of the 512^3 workloads (7 deg and 20 deg half cone
    angle), with references at K = 32 and K = 64: the difference between the two references
    bounds what the comparison resolves. Errors: |b - ref|_2 / |ref|_2 and max |b - ref| /
    max |ref| over the pixels of the 8 views."""
    import torch

    from paper_2110_09841_b300 import build, inputs
    from paper_2110_09841_b300.kct import Projector

    build.build()
    ks = (32, 64)
    out = {"mode": "accuracy", "reference": "K x K rays per pixel, exact path lengths, K = 32 and 64", "results": {}}
    for name in ("cvp512", "cvp512wide"):
        g = inputs.workload_geometry(name)
        g = g.subset_views(list(range(0, g.nviews, g.nviews // 8))[:8])
        x = inputs.workload_phantom(name, device="cuda")
        R = Projector(g, "exact", "cos")
        ref = {(K, w): R.siddon(x, K=K, weighted=w) for K in ks for w in (False, True)}
        one = R.siddon(x, K=1)

        def err(b, r):
            return {"rel_l2": float((b - r).norm() / r.norm()), "rel_max": float((b - r).abs().max() / r.abs().max())}

        res = {"single_ray_vs_K64": err(one, ref[(64, False)]),
               "K32_vs_K64_equal_weights": err(ref[(32, False)], ref[(64, False)]),
               "K32_vs_K64_solid_angle": err(ref[(32, True)], ref[(64, True)])}
        for v in ("exact", "relaxed"):
            for sc in ("cos", "exact"):
                b = Projector(g, v, sc).project(x)
                for K in ks:
                    res[f"{v}/{sc}_vs_K{K}"] = err(b, ref[(K, sc == "exact")])
        torch.cuda.synchronize()
        out["results"][name] = res
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.profile_case:
        run_profile_case(args)
    elif args.accuracy:
        run_accuracy(args)
    elif args.convs:
        run_convs(args)
    elif args.paper_geometries:
        run_paper_geometries(args)
    elif args.throughput:
        run_throughput(args)
    elif args.batch:
        run_batch(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_kct(args)


if __name__ == "__main__":
    main()
