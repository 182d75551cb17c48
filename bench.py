#!/usr/bin/env python
"""Benchmark: FDK back-projection throughput (GUPS) on GB300.

One step = one FDK pass of the paper-scale workload (1248x960 detector, 496
views over 360 deg, 512^3 volume at 0.25 mm, 50-ellipsoid phantom): the
cosine-weighted Ram-Lak filter of every projection, then the back-projection
of all views into the volume. GUPS = nx*ny*nz*np / t / 1e9 (the paper's
metric). Inputs are generated on the device before timing and are larger
than L2 (2.38 GB of projections), so no L2 flush is needed between steps.

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU
oracle on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UPD_PER_CLK_SM = 8        # smem-bound FP32 bilinear: 4 x 4-byte taps per update at 128 B/clk/SM


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="c3_paper")
    ap.add_argument("--tk", type=int, default=0, help="voxels per thread along z (32/64; 0 = plan)")
    ap.add_argument("--ctas", type=int, default=2, help="CTAs per SM the TK=32 back-projector targets")
    ap.add_argument("--views", type=int, default=0, help="override the number of views (profiling runs)")
    ap.add_argument("--subsets", type=int, default=0, help="view subsets of --op mlem / sart (0 = 1 / 10)")
    ap.add_argument("--op", choices=["fdk", "fp", "ls", "mlem", "sart", "unet"], default="fdk",
                    help="fdk: filter + back-projection (the benchmark); fp: matched forward projection "
                         "of the workload's volume(s); ls: least-squares iterations (differentiable workload)")
    ap.add_argument("--grid", nargs="*", default=None,
                    help="time back-projection alone on the paper's problems P1..P10 (all when empty); "
                         "one JSON line per problem")
    ap.add_argument("--depth-sweep", nargs="*", type=int, default=None,
                    help="time the back-projection of the workload at these pipeline depths "
                         "(views in flight, default 1 2 3 4 6 8); one JSON line per depth")
    ap.add_argument("--no-sym", action="store_true",
                    help="FP32 back-projection without the mid-plane symmetry (Section 3.1.2)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the forward projector / least-squares / MLEM / SART timings of the default line")
    ap.add_argument("--oracle-table", action="store_true",
                    help="time the FP64 oracle on c1 and c2 in full and on the c3 slab, one thread and all "
                         "threads (one JSON line per case; no GPU)")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the few-view workload (train the network, held-out RMSE, wall time vs full view)")
    return ap.parse_args(argv)


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The slowest rank's time: an all-reduce (MAX) of one number, the only
    collective of the replicas layout (each rank reconstructs its own data)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Whole-job throughput (GUPS) of world independent replicas: all ranks'
    updates over the slowest rank's time."""
    return world * units_per_rank / (slowest_ms * 1e-3) / 1e9


def backprojector_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_2104_13248_gb300/csrc/k_backproject.cu", "paper_2104_13248_gb300/csrc/geom_dev.cuh"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200", "-f", self.path]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(", ") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[2]))
                mx.append(float(r[3]))
                for n, v in zip(names, r[6:10]):
                    if v.strip() == "Active":
                        reasons.add(n)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def _oracle_slab_rate(oracle, P, q, g, k0, max_slices, chunk, budget_s):
    """Back-project chunks of slices from k0 until max_slices or budget_s;
    returns (GUPS, slices done, seconds, slab)."""
    import numpy as np
    done, t, parts = 0, 0.0, []
    while done < max_slices and t < budget_s:
        n = min(chunk, max_slices - done)
        t0 = time.perf_counter()
        parts.append(oracle.backproject_slab(P, q, g["nx"], g["ny"], k0 + done, n, math.pi / g["np"]))
        t += time.perf_counter() - t0
        done += n
    upd = float(g["nx"]) * g["ny"] * done * g["np"]
    return upd / t / 1e9, done, t, np.concatenate(parts, axis=0)


def cpu_baseline(g, budget_s=12.0, max_slices=64, budget_1t_s=6.0):
    """The FP64 oracle back-projecting a central z-slab of the workload on the
    host cores (bounded in time), on all threads and on one. The slab is
    split over (slice, row) pairs, so every thread works even on a thin slab.
    Data: seeded uniform projections, FP32 values (the oracle's cost does not
    depend on them). Returns the timing record and (k0, slices, projections,
    oracle slab) for the parity check of the GPU volume."""
    import numpy as np

    import oracle
    from paper_2104_13248_gb300 import inputs
    P = oracle.matrices(g)
    q32 = inputs.uniform_array(99, (g["np"], g["nv"], g["nu"]), -1.0, 1.0).astype(np.float32)
    q = q32.astype(np.float64)
    k0 = g["nz"] // 2 - max_slices // 2
    threads = oracle.num_threads()
    rate, done, t, slab = _oracle_slab_rate(oracle, P, q, g, k0, max_slices, 2, budget_s)
    oracle.set_threads(1)
    try:
        rate1, done1, t1, _ = _oracle_slab_rate(oracle, P, q, g, k0, max_slices, 1, budget_1t_s)
    finally:
        oracle.set_threads(threads)
    upd = float(g["nx"]) * g["ny"] * done * g["np"]
    rec = {"value": rate, "unit": "GUPS", "cores": threads, "kind": "oracle",
           "single_thread": {"value": rate1, "unit": "GUPS", "cores": 1,
                             "sample": f"slices {k0}..{k0 + done1 - 1}, {t1:.1f} s"},
           "nproc": os.cpu_count(), "cpu_model": cpu_model(),
           "sample": f"FP64 oracle back-projection of slices {k0}..{k0 + done - 1} "
                     f"({g['nx']}x{g['ny']}x{done} voxels x {g['np']} views, {upd:.3g} updates, {t:.1f} s) "
                     f"on {threads} OpenMP threads over (slice, row) pairs"}
    return rec, (k0, done, q32, slab)


def slab_parity(ctx, g, sample) -> dict:
    """Max error of the GPU volume against the oracle's slab (relative to the
    slab's largest value): the FP32 path the step times, and FP16-stored
    projections (whose oracle input is the unquantised FP32 values)."""
    import numpy as np
    import torch

    from paper_2104_13248_gb300 import api
    k0, n, q32, ref = sample
    scale = math.pi / g["np"]
    out = {"slices": f"{k0}..{k0 + n - 1}", "metric": "max|gpu - oracle| / max|oracle|",
           "tolerance_f32": 1e-5, "tolerance_f16": 2e-3}
    dq = torch.from_numpy(q32).cuda()
    for key, qd in (("f32", dq), ("f16", dq.half())):
        vol = api.bp_backproject(ctx, qd, scale=scale)
        got = vol[k0:k0 + n].double().cpu().numpy()
        out["max_rel_err_" + key] = float(np.abs(got - ref).max() / np.abs(ref).max())
        del vol
    api.bp_device_status(ctx)
    return out


def bench_config(g, workload: str, world: int) -> dict:
    """The line's config: the workload with its sizes (both arms print the same)."""
    proj_gb = 4.0 * g["np"] * g["nv"] * g["nu"] / 1e9
    return {"workload": f"{workload}: {g['nu']}x{g['nv']}x{g['np']} -> "
                        f"{g['nx']}x{g['ny']}x{g['nz']}, FP32 projections, filter + back-projection",
            "l2": "inputs larger than L2 (projections %.2f GB), no flush" % proj_gb,
            "parallelism": "replicas" if world > 1 else "single-gpu"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle timed on a bounded sample (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2104_13248_gb300 import inputs
    oracle.build()
    g = inputs.preset(args.workload)["geom"]
    P = oracle.matrices(g)
    q = inputs.uniform_array(99, (g["np"], g["nv"], g["nu"]), -1.0, 1.0)
    nks = 2
    k0 = g["nz"] // 2 - 1
    scale = math.pi / g["np"]
    for _ in range(max(1, args.warmup)):
        oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, scale)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, scale)
        times.append(time.perf_counter() - t0)
    upd = float(g["nx"]) * g["ny"] * nks * g["np"]
    t = statistics.mean(times)
    val = upd / t / 1e9
    sample = (f"each step: FP64 oracle back-projection of a {g['nx']}x{g['ny']}x{nks} slab "
              f"({g['np']} views, {upd:.3g} updates) of the {args.workload} workload, "
              f"{oracle.num_threads()} OpenMP threads over (slice, row) pairs")
    line = {"impl": "reference", "metric": "fdk_backprojection_gups", "value": val, "unit": "GUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": bench_config(g, args.workload, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": val, "unit": "GUPS", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample, "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": val, "unit": "GUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_unet(args):
    """Inference of the few-view network on one volume (random weights; the
    cost does not depend on them): --views sets the edge length (default 256)."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2104_13248_gb300.unet import UNet, conv_flops

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.views or 256
    net = UNet(seed=0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((n, n, n), device="cuda", generator=gen)
    for _ in range(args.warmup):
        net.forward(x)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        net.forward(x)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / args.steps
    flops = conv_flops((1, n, n, n))
    print(json.dumps({"metric": "unet_inference_tflops", "value": flops / (ms * 1e-3) / 1e12, "unit": "TFLOP/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "config": {"workload": f"few-view U-Net inference, {n}^3 volume",
                                 "flop_per_step": flops}}), flush=True)


def measure_op(op, workload, steps, warmup, views=0, subsets=0) -> dict:
    """One secondary operator on a workload (forward projection, a least-squares
    iteration, an MLEM or SART pass), timed with CUDA events; the record of the
    JSON line of ``--op`` and of the main line's ``variants``."""
    import torch

    from paper_2104_13248_gb300 import api, autograd, inputs

    p = inputs.preset(workload)
    g = p["geom"]
    if views:
        g = inputs.scaled_geom(g, np=views)
    batch = p.get("batch", 1)
    ctx = api.bp_create(g)
    U = float(g["nx"]) * g["ny"] * g["nz"] * g["np"] * batch
    raws = torch.stack([api.bp_phantom_project(ctx, inputs.random_ellipsoids(p["seed"] + b, p["n_ell"], p["axes"], g))
                        for b in range(batch)])
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((batch,) + ctx.vol_shape(), device="cuda", generator=gen)
    proj = torch.empty_like(raws)
    sub = None
    if op == "fp":
        def step():
            api.fp_project(ctx, x, proj=proj)
        upd, unit_desc = U, "forward-projection"
    elif op in ("mlem", "sart"):
        from paper_2104_13248_gb300 import iterative
        nsub = subsets or (1 if op == "mlem" else 10)
        sub = iterative.Subsets(ctx, nsub, need_rays=op == "sart")
        state = {"x": x[0].clone()}

        def step():
            if op == "mlem":
                state["x"] = iterative.mlem(ctx, raws[0], iters=1, x0=state["x"], sub=sub)
            else:
                state["x"] = iterative.sart(ctx, raws[0], iters=1, x0=state["x"], sub=sub, nonneg=True)
        U = U / batch
        upd = 2 * U
        unit_desc = (f"one {op.upper()} pass over {nsub} view subset(s): a forward and a back-projection "
                     f"of every view plus the element-wise steps (batch 1)")
    else:
        L = autograd.lipschitz(ctx, iters=5)

        def step():
            autograd.least_squares(ctx, raws, iters=1, x0=x, L=L)
        upd, unit_desc = 2 * U, "least-squares iteration (one forward + one back-projection)"
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        step()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    api.bp_device_status(ctx)
    if sub is not None:
        sub.close()
    ctx.close()
    del raws, x, proj
    torch.cuda.empty_cache()
    return {"value": upd / (ms * 1e-3) / 1e9, "unit": "GUPS", "ms_per_step": ms, "steps": steps,
            "workload": workload, "batch": 1 if sub else batch, "step": unit_desc}


def run_op(args):
    """Secondary measurements (forward projector, least squares, MLEM, SART) in the same JSON form."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    if args.op == "unet":
        return run_unet(args)
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = measure_op(args.op, args.workload, args.steps, args.warmup, views=args.views, subsets=args.subsets)
    print(json.dumps({"metric": f"{args.op}_gups", "value": r["value"], "unit": "GUPS",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": args.workload, "batch": r["batch"], "step": r["step"]}}),
          flush=True)


def secondary_variants(steps=5, warmup=3) -> dict:
    """The other operators of the path, timed in the default run: the matched
    forward projector on c2 (360 views, 256^3), one batched least-squares
    iteration on c4 (4 x 256^3, 180 views), and one MLEM and one 10-subset
    SART pass on c4 (one volume)."""
    out = {}
    for key, op, wl in (("fp", "fp", "c2_fdk256"), ("ls_iter", "ls", "c4_diff"),
                        ("mlem_pass", "mlem", "c4_diff"), ("sart_pass", "sart", "c4_diff")):
        try:
            out[key] = measure_op(op, wl, steps, warmup)
        except Exception as e:   # the line keeps the back-projection numbers either way
            out[key] = {"error": f"{type(e).__name__}: {e}"}
    return out


def run_grid(args):
    """The paper's problem grid: back-projection alone (no filter), per problem
    the device-resident time and the time including the host-to-device copy of
    the projections from pinned memory (the volume stays on the device), the
    two ways the paper reports its CPU and GPU results."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2104_13248_gb300 import api, inputs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    labels = args.grid or list(inputs.PROBLEMS)
    stream = torch.cuda.current_stream()
    for label in labels:
        g = inputs.paper_problem(label, views=args.views or 512)
        ctx = api.bp_create(g)
        if args.no_sym:
            api.bp_set_symmetry(ctx, False)
        gen = torch.Generator(device="cuda").manual_seed(5)
        q = torch.rand(ctx.proj_shape(), device="cuda", generator=gen)
        vol = torch.empty(ctx.vol_shape(), device="cuda")
        host = torch.empty(q.shape, dtype=torch.float32, pin_memory=True)
        host.copy_(q)
        scale = math.pi / g["np"]
        U = float(g["nx"]) * g["ny"] * g["nz"] * g["np"]

        def timed(fn):
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            return statistics.median(ms)

        ms_dev = timed(lambda: api.bp_backproject(ctx, q, vol=vol, scale=scale))

        def with_h2d():
            q.copy_(host, non_blocking=True)
            api.bp_backproject(ctx, q, vol=vol, scale=scale)

        ms_h2d = timed(with_h2d)
        api.bp_device_status(ctx)
        print(json.dumps({
            "metric": "bp_gups", "problem": label, "value": U / (ms_dev * 1e-3) / 1e9, "unit": "GUPS",
            "ms": ms_dev, "with_h2d": {"value": U / (ms_h2d * 1e-3) / 1e9, "ms": ms_h2d,
                                       "h2d_bytes": host.numel() * 4},
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic (uniform)",
            "config": {"detector": f"{g['nu']}x{g['nv']}", "views": g["np"],
                       "volume": f"{g['nx']}^3", "volume_gb": U / g["np"] * 4 / 1e9,
                       "plan": api.bp_get_plan(ctx)}}), flush=True)
        del q, vol, host
        ctx.close()
        torch.cuda.empty_cache()


def run_depth_sweep(args):
    """Back-projection alone at several staging depths (views in flight), FP32
    and FP16 storage: the GPU analogue of the paper's view-batch experiment
    (Section 4.3), where the batch is the number of views prefetched ahead of
    the voxel updates."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2104_13248_gb300 import _lib, api, inputs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    g = inputs.preset(args.workload)["geom"]
    if args.views:
        g = inputs.scaled_geom(g, np=args.views)
    ctx = api.bp_create(g)
    gen = torch.Generator(device="cuda").manual_seed(5)
    q32 = torch.rand(ctx.proj_shape(), device="cuda", generator=gen)
    q16 = q32.half()
    vol = torch.empty(ctx.vol_shape(), device="cuda")
    scale = math.pi / g["np"]
    U = float(g["nx"]) * g["ny"] * g["nz"] * g["np"]
    stream = torch.cuda.current_stream()

    def timed(q):
        for _ in range(args.warmup):
            api.bp_backproject(ctx, q, vol=vol, scale=scale)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            api.bp_backproject(ctx, q, vol=vol, scale=scale)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    for depth in (args.depth_sweep or [1, 2, 3, 4, 6, 8]):
        try:
            api.bp_set_pipeline_depth(ctx, depth)
        except _lib.BPError as e:
            print(json.dumps({"metric": "bp_gups", "workload": args.workload, "stages": depth,
                              "skipped": str(e)}), flush=True)
            continue
        ms32, ms16 = timed(q32), timed(q16)
        api.bp_device_status(ctx)
        print(json.dumps({"metric": "bp_gups", "workload": args.workload, "stages": depth,
                          "value": U / (ms32 * 1e-3) / 1e9, "unit": "GUPS", "ms": ms32,
                          "fp16_storage": {"value": U / (ms16 * 1e-3) / 1e9, "ms": ms16},
                          "steps": args.steps, "warmup": args.warmup, "plan": api.bp_get_plan(ctx)}),
              flush=True)
    ctx.close()


def learned_block() -> dict:
    """The few-view workload (60 of 360 views -> 256^3): train the U-Net on
    crops of generated pairs, held-out RMSE against the full-view FDK, and the
    wall time of few-view FDK + network against full-view FDK on this GPU."""
    from paper_2104_13248_gb300 import learned
    t0 = time.perf_counter()
    try:
        r = learned.run(steps=16000, lr=5e-4, log_every=0)
    except Exception as e:   # the line keeps the back-projection numbers either way
        return {"error": f"{type(e).__name__}: {e}"}
    keys = ("rmse_few_view", "rmse_few_view_plus_net", "rmse_ratio", "ms_full_view_fdk", "ms_few_view_fdk",
            "ms_net", "speedup_vs_full_view", "net_tflops", "steps", "train_s", "heldout")
    out = {k: r[k] for k in keys}
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    out["net_frac_of_bf16_peak"] = r["net_tflops"] / peak
    out["bf16_peak_tflops"] = f"{peak:.1f} ({src}, burst)"
    out["workload"] = "c5: 60 of 360 views, 512x512 detector -> 256^3; 3-level residual U-Net, BF16 tensor cores"
    out["wall_s"] = time.perf_counter() - t0
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2104_13248_gb300 import api, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    def slowest(x: float) -> float:
        return max_over_ranks(x, world, dev)

    p = inputs.preset(args.workload)
    g = p["geom"]
    if args.views:
        g = inputs.scaled_geom(g, np=args.views)
    ctx = api.bp_create(g)
    if args.tk or args.ctas != 2:
        api.bp_set_tuning(ctx, args.tk or 32, args.ctas)
    if args.no_sym:
        api.bp_set_symmetry(ctx, False)
    plan = api.bp_get_plan(ctx)
    E = inputs.random_ellipsoids(p["seed"] + 7919 * rank, p["n_ell"], p["axes"], g)
    raw = api.bp_phantom_project(ctx, E)
    q32 = torch.empty_like(raw)
    q16 = torch.empty(raw.shape, dtype=torch.float16, device=dev)
    vol = torch.empty(ctx.vol_shape(), dtype=torch.float32, device=dev)
    scale = math.pi / g["np"]
    U = float(g["nx"]) * g["ny"] * g["nz"] * g["np"]
    stream = torch.cuda.current_stream()

    def time_steps(q, n_steps, bp_events):
        for _ in range(args.warmup):
            api.bp_filter(ctx, raw, out=q)
            api.bp_backproject(ctx, q, vol=vol, scale=scale)
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(n_steps):
            api.bp_filter(ctx, raw, out=q)
            bp_events[i][0].record(stream)
            api.bp_backproject(ctx, q, vol=vol, scale=scale)
            bp_events[i][1].record(stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        step_ms = ev0.elapsed_time(ev1) / n_steps
        bp_ms = statistics.mean(a.elapsed_time(b) for a, b in bp_events[:n_steps])
        return step_ms, bp_ms

    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    with ClockSampler(uuid) as clk:
        step_ms, bp_ms = time_steps(q32, K, evs)
    clocks = clk.summary()
    api.bp_device_status(ctx)
    step_ms_max = slowest(step_ms)
    bp_ms_max = slowest(bp_ms)
    step16_ms, bp16_ms = time_steps(q16, K, evs)
    api.bp_device_status(ctx)
    step16_ms = slowest(step16_ms)
    bp16_ms = slowest(bp16_ms)

    peaks, peak_src = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_gups = n_sm * UPD_PER_CLK_SM * sm_mhz * 1e6 / 1e9
    achieved = U / (bp_ms_max * 1e-3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "bp_c3_traffic.json")
    if os.path.exists(tp) and args.workload == "c3_paper" and not args.views:
        try:
            rec = json.load(open(tp))
            # counters only count while the kernel source is the one they were taken on
            if rec.get("source_sha256_16") == backprojector_source_hash():
                traffic = rec.get("dram_bytes_per_launch")
        except Exception:
            traffic = None

    # end to end through the public API: pinned host projections in, volume out
    e2e = None
    if not args.no_e2e:
        host_proj = torch.empty(raw.shape, dtype=torch.float32, pin_memory=True)
        host_proj.copy_(raw)
        host_vol = torch.empty(ctx.vol_shape(), dtype=torch.float32, pin_memory=True)
        pipe = api.HostPipeline(ctx)
        for _ in range(args.warmup):
            pipe.run(host_proj, host_vol)
        torch.cuda.synchronize()
        barrier()
        n_e2e = max(5, min(K, 20))
        ts = []
        for _ in range(n_e2e):
            t0 = time.perf_counter()
            pipe.run(host_proj, host_vol)
            torch.cuda.current_stream().synchronize()
            float(host_vol[g["nz"] // 2, g["ny"] // 2, g["nx"] // 2])   # read the result
            ts.append(time.perf_counter() - t0)
        # the median step: single steps on a shared host occasionally stall for milliseconds
        t_e2e = statistics.median(ts)
        barrier()
        t_e2e = slowest(t_e2e)
        api.bp_device_status(ctx)
        e2e = {"value": world * U / t_e2e / 1e9, "unit": "GUPS",
               "h2d_bytes_per_step": host_proj.numel() * 4, "d2h_bytes_per_step": host_vol.numel() * 4,
               "ms_per_step": t_e2e * 1e3, "ms_per_step_mean": 1e3 * sum(ts) / len(ts), "steps": n_e2e,
               "pipeline": f"{len(pipe.blocks)} view blocks, {len(pipe.parts)} slab parts with mirrors"}

    others = None
    if rank == 0 and not args.no_variants and args.workload == "c3_paper" and not args.views:
        others = secondary_variants()

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, sample = cpu_baseline(g)
        parity = slab_parity(ctx, g, sample)

    # the metric's second half: the learned few-view path against the plain full-view FDK
    learned_res = None
    if rank == 0 and not args.no_learned and args.workload == "c3_paper" and not args.views:
        learned_res = learned_block()

    # the launches inside the timed region: filter + back-projection per step
    line = {
        "metric": "fdk_backprojection_gups",
        "value": replica_value(U, world, step_ms_max),
        "unit": "GUPS",
        "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": step_ms_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(g, args.workload, world),
        "plan": plan,
        "gpu_launches": 2 * K,
        "roofline": {"bound": "alu", "resource": "shared-memory taps (4 x 4 B per update at 128 B/clk/SM)",
                     "achieved": achieved, "peak": peak_gups, "unit": "GUPS",
                     "frac": achieved / peak_gups, "traffic": traffic,
                     "peak_basis": f"{n_sm} SMs x {UPD_PER_CLK_SM} updates/clk x {sm_mhz:.0f} MHz "
                                   f"(sm_max_mhz, {peak_src})",
                     "kernel_ms": bp_ms_max},
        "clocks": clocks,
        "variants": {"fp16_storage": {"value": world * U / (step16_ms * 1e-3) / 1e9, "unit": "GUPS",
                                      "ms_per_step": step16_ms, "bp_kernel_ms": bp16_ms,
                                      "bp_kernel_gups": U / (bp16_ms * 1e-3) / 1e9}},
    }
    if others:
        line["variants"].update(others)
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    if parity:
        line["parity"] = parity
    if learned_res:
        line["learned"] = learned_res
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_oracle_table(args):
    """The FP64 oracle's own throughput on the host: c1 and c2 in full and the
    central 64-slice slab of c3, on one thread and on all threads (the arm of
    the CPU baseline table). No GPU is used."""
    import numpy as np

    import oracle
    from paper_2104_13248_gb300 import inputs
    oracle.build()
    threads = oracle.num_threads()
    model = cpu_model()
    for name, k0, nks in (("c1_small", None, None), ("c2_fdk256", None, None), ("c3_paper", 224, 64)):
        g = inputs.preset(name)["geom"]
        P = oracle.matrices(g)
        q = inputs.uniform_array(99, (g["np"], g["nv"], g["nu"]), -1.0, 1.0).astype(np.float32).astype(np.float64)
        if k0 is None:
            k0, nks = 0, g["nz"]
        upd = float(g["nx"]) * g["ny"] * nks * g["np"]
        for n in (threads, 1):
            oracle.set_threads(n)
            t0 = time.perf_counter()
            oracle.backproject_slab(P, q, g["nx"], g["ny"], k0, nks, math.pi / g["np"])
            t = time.perf_counter() - t0
            print(json.dumps({"metric": "oracle_backprojection_gups", "workload": name,
                              "slices": f"{k0}..{k0 + nks - 1}", "updates": upd, "threads": n,
                              "value": upd / t / 1e9, "unit": "GUPS", "seconds": t, "nproc": os.cpu_count(),
                              "cpu_model": model}), flush=True)
        oracle.set_threads(threads)


def main(argv=None):
    args = parse_args(argv)
    if args.oracle_table:
        run_oracle_table(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.grid is not None:
        run_grid(args)
    elif args.depth_sweep is not None:
        run_depth_sweep(args)
    elif args.op != "fdk":
        run_op(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
