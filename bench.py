#!/usr/bin/env python
"""Benchmark of the Krylov CBCT hot path on GB300.

Workload (the 256^3 medical configuration): 256^3 x 1 mm volume, 512 x 512
detector of 0.8 mm pixels, 360 angles over 360 deg, DSO 1000 / DSD 1536 mm,
random-ellipsoid phantom x 0.02 mm^-1, Poisson noise with I0 = 1e5.  One step
= LSQR 30 iterations + LSMR 30 iterations on that b (both through the C ABI,
FP32 vectors, FP64 scalars).

Printed JSON line (rank 0):
  value      ray-voxel Gupdates/s of the whole step (nnz(A) x projector
             launches / step time), inputs resident in HBM, on the solvers'
             default path (one CUDA graph per iteration, replayed);
  e2e        the same metric with b read from pinned host memory and x
             written back to the host inside the timed region;
  roofline   the dominant projector kernel (per-launch CUDA-event times from
             one extra profiled step): nnz x 4 B gathered per launch / its
             launch time against the measured HBM copy peak, and the bound
             t_bound = max(compulsory HBM bytes / HBM peak, gather bytes /
             L2 peak, warp instructions / issue peak) term by term;
  serving    the serving stream (64 requests of 128^3..384^3 scans, Poisson
             arrivals at 0.8 of the one-at-a-time throughput, from measured
             service times) through the
             continuous-batching server and through the one-request-at-a-time
             solver, both fed in real time: recon/s, p50 / p99 / mean latency
             and the largest relative difference between their results (at
             N = 1 only);
  cpu_baseline  the FP64 oracle on the host cores, on a 24-angle sample.
`--impl reference` times that oracle alone (the CPU reference arm).
Multi-GPU (torchrun): independent replicas, one per rank, weak scaling.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ray-voxel Gupdates/s and LSQR iters/s at 256^3; serving recon/s, p50/p99 latency"
UNIT = "Gupdates/s"
ITERS = 30
I0 = 1e5
BYTES_PER_UPDATE = 4          # one FP32 voxel (forward) or projection (backward) value per ray-voxel update
CPU_SAMPLE_ANGLES = 24          # about 20 s of FP64 oracle work on 16 host cores
REF_STEP_ANGLES = 8             # --impl reference: about 7 s per step, so K steps stay within minutes

# Counters of one launch of each solver projector kernel at 256^3 / 512^2 /
# 360 from ncu (dram__bytes_read.sum + dram__bytes_write.sum, and
# smsp__inst_executed.sum = warp instructions), keyed by the code of the
# projector sources they were measured on (projector_hash(), comments
# ignored) and the launch shape (rays per lane, transpose configuration);
# the bench reports null once either differs.
NCU_COUNTERS = {
    "forward": {"hash": "bf0c463e413182ae", "shape": [4, 3], "kernel": "forward_kernel<float, 0, 4, 1>",
                "dram_bytes": 3018182400, "warp_inst": 19929252800},
    "backward": {"hash": "bf0c463e413182ae", "shape": [4, 3], "kernel": "backward_kernel<float, 1, 2, 2, 1, 0>",
                 "dram_bytes": 2791051008, "warp_inst": 31975031028},
}

# Instruction issue: one warp instruction per cycle per SM sub-partition.
SMS, SUBPARTITIONS = 152, 4


def workload_config():
    import synth
    g = synth.config("c2")
    return g, {
        "workload": "256^3 medical CBCT: LSQR 30 + LSMR 30 iterations per step",
        "volume": [g.nx, g.ny, g.nz], "voxel_mm": g.dx,
        "detector": [g.nu, g.nv], "pixel_mm": g.du, "angles": g.nangles,
        "dso_mm": g.dso, "dsd_mm": g.dsd, "phantom": "10 random ellipsoids (seed 1) x 0.02 mm^-1",
        "noise": "Poisson I0=1e5, log-transformed",
        "l2": "inputs larger than L2 (projection stack 360 MiB, Krylov vectors 64-360 MiB each)",
    }


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def code_only(text):
    """C/C++ source without its comments, whitespace runs collapsed to one
    space (string and character literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def projector_hash(sources=None):
    """sha256 over the code of the projector kernel sources (projector.cu,
    projector_device.cuh, transpose.cuh; comments and whitespace dropped), first 16 hex
    digits: the ncu counters stay attached to the kernels while only their
    comments change."""
    h = hashlib.sha256()
    for name in ("projector.cu", "projector_device.cuh", "transpose.cuh"):
        if sources is not None:
            text = sources[name]
        else:
            with open(os.path.join(ROOT, "paper_2211_14212_gb300", "csrc", name)) as f:
                text = f.read()
        h.update(code_only(text).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None:
            return None
        self.out.flush()
        rows = []
        with open(self.out.name) as f:
            for line in f:
                p = [c.strip() for c in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.out.name)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(v, world, device):
    """Largest value of `v` over the ranks of the default process group (the
    job's time is its slowest replica's)."""
    if world == 1:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, elapsed_s):
    """Replicas: every rank processes the same number of units (weak scaling);
    the job rate is all ranks' units over the slowest rank's time."""
    return world * units_per_rank / elapsed_s


def oracle_sample_rate(g, nangles=CPU_SAMPLE_ANGLES, gpu_nnz=None):
    """FP64 oracle A x and A^T y on `nangles` angles of the workload; Gupdates/s."""
    import numpy as np
    import oracle
    import synth
    sub = g.angle_subset(nangles)
    x = synth.ellipsoid_phantom(g, 10, seed=1, scale=0.02).astype(np.float64)
    y = synth.random_projections(sub, 3)
    nnz = gpu_nnz(sub) if gpu_nnz else oracle.nnz(sub)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.project(sub, x, cores)
    oracle.backproject(sub, y, cores)
    dt = time.perf_counter() - t0
    return 2 * nnz / dt / 1e9, cores, dt, nnz


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    g, config = workload_config()
    for _ in range(args.warmup):
        oracle_sample_rate(g, 2)
    vals, times = [], []
    cores = nnz = None
    for _ in range(args.steps):
        v, cores, dt, nnz = oracle_sample_rate(g, REF_STEP_ANGLES)
        vals.append(v)
        times.append(dt)
    value = sum(2 * nnz for _ in times) / sum(times) / 1e9
    sample = "FP64 oracle A x + A^T y on %d of %d angles (%d updates each)" % (REF_STEP_ANGLES, g.nangles, nnz)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def roofline_block(g, nnz, fwd_ms, bwd_ms, clocks, shape=None):
    """Roofline of the dominant projector kernel.  `achieved` is the gather-
    equivalent bandwidth (nnz x 4 B per launch / launch time) against the
    measured HBM copy peak, the scope table's projector target.  The kernels
    are bound by instruction issue, so `t_bound` lists the three floors of
    max(compulsory HBM bytes / HBM peak, gather bytes / L2 peak, warp
    instructions / issue peak): no L2 peak is measured on this machine (null),
    and the warp-instruction count comes from ncu (NCU_COUNTERS, null once the
    kernel source changed or when the run's launch shape `shape` = (rays per
    lane, transpose configuration) is not the one the counters were taken
    on)."""
    dominant = "forward" if fwd_ms >= bwd_ms else "backward"
    avg_ms = fwd_ms if dominant == "forward" else bwd_ms
    peak, peak_kind = measured_peak()
    achieved = nnz * BYTES_PER_UPDATE / (avg_ms * 1e-3) / 1e9
    c = NCU_COUNTERS.get(dominant)
    fresh = c is not None and c.get("hash") == projector_hash() and \
        (shape is None or tuple(c.get("shape", ())) == tuple(shape))
    warp_inst = c["warp_inst"] if fresh else None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    issue_peak = SMS * SUBPARTITIONS * mhz * 1e6            # warp instructions per second
    compulsory = (g.num_voxels + g.num_rays) * 4             # one read of the input, one write of the output
    hbm_ms = compulsory / (peak * 1e9) * 1e3
    issue_ms = warp_inst / issue_peak * 1e3 if warp_inst else None
    terms = {"hbm": hbm_ms, "l2": None, "issue": issue_ms}
    known = {k: v for k, v in terms.items() if v is not None}
    return {"bound": "issue", "kernel": dominant, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / peak, "traffic": c["dram_bytes"] if fresh else None,
            "avg_launch_ms": avg_ms, "forward_ms_per_launch": fwd_ms, "backward_ms_per_launch": bwd_ms,
            "t_bound": {"hbm_ms": hbm_ms, "l2_ms": None, "issue_ms": issue_ms,
                        "binding": max(known, key=known.get) if known else None,
                        "notes": "hbm: (M + N) x 4 B compulsory bytes; l2: no L2 peak measured; issue: "
                                 "ncu warp instructions of one launch / (152 SMs x 4 issue slots x SM clock)"},
            "issue_util": issue_ms / avg_ms if issue_ms else None}


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct

    g, config = workload_config()
    dev = torch.device("cuda", local)
    geom = cbct.Geometry(g)
    tune = cbct.autotune(geom, max_angles=32)
    x_true = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=1, scale=0.02)).to(dev)
    b_clean = cbct.project(geom, x_true).cpu().numpy()
    b_host = torch.from_numpy(synth.poisson_log_noise(b_clean, I0, seed=2 + rank)).pin_memory()
    b = b_host.to(dev)
    del b_clean
    nnz = cbct.count_nnz(geom)
    s = torch.cuda.Stream(device=dev)
    x1 = torch.empty(geom.vol_shape, device=dev)
    x2 = torch.empty(geom.vol_shape, device=dev)

    def step(bb, xa, xb, profile):
        r1 = cbct.lsqr(geom, bb, ITERS, x=xa, stream=s, profile=profile)[1]
        t_lsqr = time.perf_counter()
        r2 = cbct.lsmr(geom, bb, ITERS, x=xb, stream=s, profile=profile)[1]
        return r1, r2, t_lsqr

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            step(b, x1, x2, False)
    barrier()

    # ---- timed region: inputs resident in HBM, the solvers' default (graph-replayed) path
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and all(p.strip().isdigit() for p in vis.split(",")):
        gpu_index = int(vis.split(",")[local])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    products = launches = 0
    lsqr_s = 0.0
    with ClockSampler(gpu_index) as clk:
        with torch.cuda.stream(s):
            torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed launches
            ev0.record(s)
            for _ in range(args.steps):
                t0 = time.perf_counter()
                r1, r2, t1 = step(b, x1, x2, False)
                lsqr_s += t1 - t0          # the solver synchronises its stream before returning
                for r in (r1, r2):
                    products += r.forward_launches + r.backward_launches
                    launches += r.kernel_launches
            ev1.record(s)
            torch.cuda.nvtx.range_pop()
        barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    clocks = clk.summary()
    value = whole_job_rate(nnz * products, world, elapsed_ms * 1e-3) / 1e9
    lsqr_ips = ITERS * args.steps / lsqr_s

    # ---- one profiled step (plain launches, CUDA events around every projector launch)
    fwd_ms = bwd_ms = 0.0
    fwd_n = bwd_n = 0
    with torch.cuda.stream(s):
        for r in step(b, x1, x2, True)[:2]:
            fwd_ms += r.forward_ms
            bwd_ms += r.backward_ms
            fwd_n += r.forward_launches
            bwd_n += r.backward_launches
    barrier()

    # ---- end to end: b from pinned host memory, x back to host, inside the timed region
    xh1 = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
    xh2 = torch.empty(geom.vol_shape, dtype=torch.float32).pin_memory()
    bh = b_host.numpy()
    barrier()
    t0 = time.perf_counter()
    e2e_products = 0
    with torch.cuda.stream(s):
        for _ in range(args.steps):
            r1, r2, _ = step(bh, xh1.numpy(), xh2.numpy(), False)
            e2e_products += r1.forward_launches + r1.backward_launches + r2.forward_launches + r2.backward_launches
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e_value = whole_job_rate(nnz * e2e_products, world, e2e_s) / 1e9
    del x1, x2, b

    serving = None
    # the serving stream runs on one GPU for about ten minutes: at N = 1 only,
    # so that a multi-GPU run does not hold the other GPUs idle meanwhile
    if not args.no_serving and world == 1:
        serving = serving_compare(cbct, torch, dev, args.requests, args.serving_scale,
                                  args.serving_slots, args.serving_budget_gb, args.serving_schedule)

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    cpu = None
    if not args.no_cpu_baseline:
        def gpu_nnz(sub):
            return cbct.count_nnz(cbct.Geometry(sub))
        v, cores, dt, snnz = oracle_sample_rate(g, CPU_SAMPLE_ANGLES, gpu_nnz)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "FP64 oracle A x + A^T y on %d of %d angles (%d updates each, %.1f s)"
                         % (CPU_SAMPLE_ANGLES, g.nangles, snnz, dt)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "lsqr_iters_per_s": lsqr_ips,
        "nnz": nnz,
        "roofline": roofline_block(g, nnz, fwd_ms / max(fwd_n, 1), bwd_ms / max(bwd_n, 1), clocks,
                                   (tune["fwd_rows"], tune["bwd_config"])),
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * geom.num_rays,
                "d2h_bytes_per_step": 2 * 4 * geom.num_voxels},
        "gpu_launches": launches,
        "clocks": clocks,
        "launch_shapes": {"fwd_rows": tune["fwd_rows"], "bwd_brick": tune["bwd_shape"]},
        "serving": serving if world == 1 else {"measured": "at N = 1 only (one GPU, about ten minutes)"},
    }
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_projectors(args):
    """Standalone forward / backward projector launches on the workload (per-kernel timing)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    g, config = workload_config()
    dev = torch.device("cuda", 0)
    geom = cbct.Geometry(g)
    tune = cbct.autotune(geom, max_angles=32)
    x = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=1, scale=0.02)).to(dev)
    y = torch.empty(geom.proj_shape, device=dev)
    xb = torch.empty(geom.vol_shape, device=dev)
    nnz = cbct.count_nnz(geom)
    s = torch.cuda.current_stream()
    for _ in range(args.warmup):
        cbct.project(geom, x, out=y)
        cbct.backproject(geom, y, out=xb)
    torch.cuda.synchronize()
    times = {"forward": [], "backward": [], "voxel_driven_backward": []}
    for _ in range(args.steps):
        for name, fn in (("forward", lambda: cbct.project(geom, x, out=y)),
                         ("backward", lambda: cbct.backproject(geom, y, out=xb)),
                         ("voxel_driven_backward", lambda: cbct.backproject_voxel_driven(geom, y, out=xb))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            times[name].append(e0.elapsed_time(e1))
    out = {"mode": "projectors", "config": config, "nnz": nnz, "autotune": tune}
    for name, t in times.items():
        ms = statistics.median(t)
        out[name] = {"ms": ms, "gupdates_per_s": nnz / (ms * 1e-3) / 1e9,
                     "gather_gbs": nnz * BYTES_PER_UPDATE / (ms * 1e-3) / 1e9}
    print(json.dumps(out), flush=True)
    return 0


PRECISION_REF = os.path.join(ROOT, "tests", "golden", "precision_reference.json")


def run_precision(args):
    """Storage-precision study (Krylov vectors, basis, volumes and projections
    stored in FP32, FP16 or BF16; FP32 ray sums, Kahan-compensated for the
    16-bit formats; FP64 Krylov scalars), errors against the FP64 oracle's
    stored values (tests/golden/precision_reference.json):
      * 512^3 scan (768 x 512 detector, 720 angles): A x and A^T y at sampled
        rays / voxels; hybrid LSQR 50 (GCV) on noisy data, time per iteration
        and the distance of each result from the FP32 one and from the phantom;
      * 64^3 scan: LSQR, LSMR and hybrid LSQR after 20 iterations against the
        FP64 iterates at sampled voxels;
      * basis memory: hybrid LSQR with 70 iterations on a 1024^3 volume keeps
        70 basis volumes, more than the device holds in FP32, run in FP16."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    with open(PRECISION_REF) as f:
        ref = json.load(f)
    dev = torch.device("cuda", 0)
    dts = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}

    def rel(a, b):
        a = np.asarray(a, np.float64)
        b = np.asarray(b, np.float64)
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    # ---- 512^3: projectors against FP64, hybrid LSQR 50 per storage
    g = synth.config("c3")
    geom = cbct.Geometry(g)
    tune = cbct.autotune(geom, max_angles=32)
    nnz = cbct.count_nnz(geom)
    c3 = ref["c3"]
    rays = torch.from_numpy(np.asarray(c3["rays"])).to(dev)
    vox = torch.from_numpy(np.asarray(c3["voxels"])).to(dev)
    x32 = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=c3["phantom_seed"], scale=0.02)).to(dev)
    y32 = torch.from_numpy(synth.random_projections(g, c3["y_seed"]).astype(np.float32)).to(dev)
    proj = {}
    for st, dt in dts.items():
        x, y = x32.to(dt), y32.to(dt)
        ax = cbct.project(geom, x)
        aty = cbct.backproject(geom, y)
        torch.cuda.synchronize()
        times = []
        for fn in (lambda: cbct.project(geom, x, out=ax), lambda: cbct.backproject(geom, y, out=aty)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        proj[st] = {"forward_rel_err_vs_fp64": rel(ax.view(-1)[rays].double().cpu(), c3["project_rays"]),
                    "backward_rel_err_vs_fp64": rel(aty.view(-1)[vox].double().cpu(), c3["backproject_voxels"]),
                    "forward_ms": times[0], "backward_ms": times[1]}
        del x, y, ax, aty
    del y32
    b = cbct.project(geom, x32).cpu().numpy()
    b = torch.from_numpy(synth.poisson_log_noise(b, 1e5, seed=25).astype(np.float32)).to(dev)
    iters = 50
    hyb, xref = {}, None
    xt = x32.double()
    for st in dts:
        cbct.hybrid_lsqr(geom, b, 2, storage=st)                   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rep = cbct.hybrid_lsqr(geom, b, iters, storage=st)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xd = x.double()
        if xref is None:
            xref = xd.clone()
        hyb[st] = {"s_per_solve": dt, "ms_per_iter": 1000 * dt / iters, "gupdates_per_s": 2 * nnz * iters / dt / 1e9,
                   "rel_diff_vs_f32": float((xd - xref).norm() / xref.norm()),
                   "rel_err_vs_phantom": float((xd - xt).norm() / xt.norm()),
                   "lambda_last": float(rep.lam[-1])}
        del x, xd
    del xref, xt, x32, b, geom

    # ---- 64^3: solvers against the FP64 iterates
    md = ref["medium"]
    gm = synth.Geometry(64, 64, 64, 4.0, 4.0, 4.0, 128, 128, 3.2, 3.2, 1000.0, 1536.0, synth.circular_angles(90))
    geom = cbct.Geometry(gm)
    bm = torch.from_numpy(synth.random_projections(gm, md["b_seed"]).astype(np.float32)).to(dev)
    mvox = torch.from_numpy(np.asarray(md["voxels"])).to(dev)
    solv = {}
    for st in dts:
        solv[st] = {}
        for method in ("lsqr", "lsmr", "hybrid_lsqr"):
            x, _ = getattr(cbct, method)(geom, bm, md["iters"], storage=st)
            solv[st][method] = rel(x.view(-1)[mvox].double().cpu(), md[method]["sampled"])
    del geom, bm

    # ---- basis memory: 1024^3 volume, hybrid LSQR 70 iterations in FP16
    gb = synth.Geometry(1024, 1024, 1024, 0.25, 0.25, 0.25, 512, 512, 1.0, 1.0, 1000.0, 1536.0,
                        synth.circular_angles(180))
    free, total = torch.cuda.mem_get_info(dev)
    k = 70
    need = {st: (k + 4) * gb.num_voxels * (4 if st == "f32" else 2) + 3 * gb.num_rays * 4 for st in ("f32", "f16")}
    geom = cbct.Geometry(gb)
    bb = torch.from_numpy(synth.random_projections(gb, 76).astype(np.float32)).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, rep = cbct.hybrid_lsqr(geom, bb, k, storage="f16")
    torch.cuda.synchronize()
    basis = {"volume": [1024, 1024, 1024], "detector": [512, 512], "angles": 180, "iters": k,
             "device_total_bytes": total, "approx_bytes_needed": need,
             "f32_fits": need["f32"] <= total, "f16_fits": need["f16"] <= total,
             "f16_iters_done": rep.iters_done, "f16_s": time.perf_counter() - t0,
             "f16_finite": bool(torch.isfinite(x).all())}
    del x, bb, geom
    print(json.dumps({"mode": "precision",
                      "config": {"workload": "512^3 CBCT precision study: projectors and hybrid LSQR 50 (GCV)",
                                 "volume": [g.nx, g.ny, g.nz], "voxel_mm": g.dx, "detector": [g.nu, g.nv],
                                 "pixel_mm": g.du, "angles": g.nangles, "dso_mm": g.dso, "dsd_mm": g.dsd,
                                 "noise": "Poisson I0=1e5"},
                      "nnz": nnz, "launch_shapes": {"fwd_rows": tune["fwd_rows"], "bwd": tune["bwd_shape"]},
                      "projectors_vs_fp64": proj, "hybrid_lsqr_50": hyb,
                      "solvers_64cube_k20_rel_err_vs_fp64": solv, "basis_memory": basis}), flush=True)
    return 0


def run_microct(args):
    """The micro-CT scan: 1024^3 x 0.1 mm volume (ellipsoids and a sample-holder
    cylinder, x 0.02 mm^-1), 1536^2 x 0.6 mm detector, 1600 angles, DSO 200 /
    DSD 1200 mm (magnification 6), Poisson noise with I0 = 2e5; LSMR 50
    iterations with Tikhonov damping lambda = 1e-2 ||b|| (Sec. 2.2, Eq. 7).
    One solve, CUDA events around every projector launch: s per solve,
    Gupdates/s of the solve and the per-launch projector roofline."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    g = synth.config("c5")
    dev = torch.device("cuda", 0)
    geom = cbct.Geometry(g)
    tune = cbct.autotune(geom, max_angles=32)
    x_true = torch.from_numpy(synth.ellipsoid_phantom(g, 4, seed=4, scale=0.02, cylinder=True)).to(dev)
    b = cbct.project(geom, x_true)
    del x_true
    gen = torch.Generator(device=dev).manual_seed(41)
    for chunk in b.view(-1).split(1 << 28):             # photon noise in place, in chunks
        counts = torch.poisson(2e5 * torch.exp(-chunk), generator=gen)
        chunk.copy_(-torch.log(torch.clamp(counts, min=1.0) / 2e5))
        del counts
    nnz = cbct.count_nnz(geom)
    bnorm = float(torch.linalg.vector_norm(b.double()))
    lam = 1e-2 * bnorm
    iters = 50
    torch.cuda.synchronize()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        x, rep = cbct.lsmr(geom, b, iters, lam=lam, profile=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    clocks = clk.summary()
    products = rep.forward_launches + rep.backward_launches
    fwd = rep.forward_ms / max(rep.forward_launches, 1)
    bwd = rep.backward_ms / max(rep.backward_launches, 1)
    rl = roofline_block(g, nnz, fwd, bwd, clocks, (tune["fwd_rows"], tune["bwd_config"]))
    rl["traffic"] = None
    rl["t_bound"]["issue_ms"] = None
    rl["issue_util"] = None
    out = {"mode": "microct",
           "config": {"workload": "1024^3 micro-CT: LSMR 50 iterations, damping 1e-2 ||b||",
                      "volume": [g.nx, g.ny, g.nz], "voxel_mm": g.dx, "detector": [g.nu, g.nv],
                      "pixel_mm": g.du, "angles": g.nangles, "dso_mm": g.dso, "dsd_mm": g.dsd,
                      "phantom": "4 random ellipsoids + cylinder (seed 4) x 0.02 mm^-1", "noise": "Poisson I0=2e5"},
           "nnz": nnz, "iters_done": rep.iters_done, "lambda": lam, "s_per_solve": dt,
           "gupdates_per_s": nnz * products / dt / 1e9, "projector_launches": products,
           "resid_last": float(rep.resid[-1]), "normal_resid_last": float(rep.normal_resid[-1]),
           "roofline": rl, "clocks": clocks, "launch_shapes": {"fwd_rows": tune["fwd_rows"],
                                                               "bwd_brick": tune["bwd_shape"]}}
    print(json.dumps(out), flush=True)
    return 0


def run_profile_solve(args):
    """A target for ncu: the 256^3 scan with the benchmark's launch shapes
    (by default 4 rays per lane, 2 x 4 columns x 64 transpose tile; the
    autotuner's choice at this size) and one LSQR solve
    of 2 iterations on a random b, plain launches.  Its first forward_kernel
    and backward_kernel launches are the instantiations the benchmark's
    solvers run (v-fastest projections with the weighted copy, z-fastest
    volume)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    g, _ = workload_config()
    geom = cbct.Geometry(g)
    cbct.set_launch(geom, args.fwd_rows, args.bwd_config)
    b = torch.from_numpy(synth.random_projections(g, 5).astype(np.float32)).cuda()
    x, rep = cbct.lsqr(geom, b, 2, use_graph=False)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "profile-solve", "iters_done": rep.iters_done,
                      "launch": [args.fwd_rows, args.bwd_config], "projector_hash": projector_hash()}))
    return 0


def serving_requests(count, scale, seed=3):
    """The serving stream: volumes in {128, 192, 256, 384}^3 over a 256 mm field
    of view, square detectors of 256..768 pixels (409.6 mm wide), 90..720 angles
    over 360 deg or a 200 deg short scan, LSQR or LSMR with 20..40 iterations,
    photon noise I0 = 5e4.  `scale` shrinks volumes and detectors (quick runs)."""
    import numpy as np
    import synth
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice([128, 192, 256, 384]))
        nu = int(rng.integers(256, 769))
        nangles = int(rng.integers(90, 721))
        short = bool(rng.integers(0, 2))
        n_s = max(16, int(round(n * scale / 8)) * 8)
        nu_s = max(32, int(round(nu * scale)))
        g = synth.serving_request_geometry(n_s, nu_s, nangles, short)
        reqs.append({"geom": g, "solver": ["lsqr", "lsmr"][int(rng.integers(0, 2))],
                     "iters": int(rng.integers(20, 41)), "seed": 1000 + i,
                     "desc": [n_s, nu_s, nangles, "200deg" if short else "360deg"]})
    return reqs


def serving_inputs(cbct, torch, dev, reqs, i0=5e4):
    """Measured projections of every request (input generation, untimed): the
    GPU forward projection of its phantom with photon noise at I0 = 5e4; and
    nnz(A) of its scan (the work model that sets the arrival rate)."""
    import numpy as np
    import synth
    gen = torch.Generator(device=dev)
    for r in reqs:
        g = r["geom"]
        geom = cbct.Geometry(g)
        x = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=r["seed"], scale=0.02)).to(dev)
        b = cbct.project(geom, x)
        gen.manual_seed(r["seed"])
        counts = torch.poisson(i0 * torch.exp(-b), generator=gen)
        r["b"] = np.ascontiguousarray((-torch.log(torch.clamp(counts, min=1.0) / i0)).float().cpu().numpy().ravel())
        r["nnz"] = cbct.count_nnz(geom)
        del x, b, counts, geom
    torch.cuda.synchronize(dev)


def plain_arm(cbct, reqs, arrivals):
    """One request at a time, in arrival order, fed in real time: request i
    starts when it has arrived and request i - 1 is done; its latency runs
    from its arrival to the end of its solve (scan set-up, b from host memory,
    the solve, x back to host memory, all through the C ABI)."""
    import numpy as np
    lat, xs = [], []
    t0 = time.perf_counter()
    for a, r in zip(arrivals, reqs):
        wait = a - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        geom = cbct.Geometry(r["geom"])
        x, rep = getattr(cbct, r["solver"])(geom, r["b"], r["iters"])
        geom.close()
        lat.append(time.perf_counter() - t0 - a)
        xs.append(x)
    span = time.perf_counter() - t0
    return np.array(lat), xs, span


def server_arm(cbct, reqs, arrivals, slots, budget_gb, schedule, x_ref=None):
    """The continuous-batching server fed in real time (a feeder thread submits
    request i at its arrival time); latency = finish - submit by the server's
    clock.  With `x_ref`, the largest relative difference of the results from
    those."""
    import threading

    import numpy as np
    srv = cbct.Server(int(budget_gb * (1 << 30)), max_slots=slots, use_graph=True, schedule=schedule)
    ids = [None] * len(reqs)
    t0 = time.perf_counter()

    def feeder():
        for i, (a, r) in enumerate(zip(arrivals, reqs)):
            wait = a - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids[i] = srv.submit(r["geom"], r["b"], r["solver"], r["iters"])

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    lat, diff = [], 0.0
    first, last = None, None
    for i in range(len(reqs)):
        res = srv.wait(ids[i])
        lat.append(res.finish_s - res.submit_s)
        first = res.submit_s if first is None else min(first, res.submit_s)
        last = res.finish_s if last is None else max(last, res.finish_s)
        if x_ref is not None:
            ref = x_ref[i].ravel().astype(np.float64)
            diff = max(diff, float(np.linalg.norm(res.x.ravel() - ref) / max(np.linalg.norm(ref), 1e-300)))
    stats = srv.stats()
    srv.close()
    return np.array(lat), last - first, diff, stats


def latency_summary(lat, span, count):
    import numpy as np
    return {"recon_per_s": count / span, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "max_s": float(lat.max())}


def calibrate_service(cbct, reqs, picks=4):
    """One-at-a-time service time model of the stream, measured: the requests
    at `picks` quantiles of nnz(A) are solved (through the same path as the
    plain arm) at 3 and 6 iterations; the difference gives the time of one
    iteration per nnz (updates/s) and the rest a fixed cost per request per
    (rays + voxels) (scan set-up, b in, x out).  Returns the predicted service
    time of every request and the fitted figures."""
    import numpy as np
    order = np.argsort([r["nnz"] for r in reqs])
    idx = sorted({int(order[int(round(q * (len(order) - 1)))]) for q in np.linspace(0.0, 1.0, picks)})
    rates, fixed = [], []
    for i in idx:
        r = reqs[i]
        t = {}
        for k in (3, 6):
            t0 = time.perf_counter()
            geom = cbct.Geometry(r["geom"])
            getattr(cbct, r["solver"])(geom, r["b"], k)
            geom.close()
            t[k] = time.perf_counter() - t0
        per_iter = max((t[6] - t[3]) / 3.0, 1e-6)
        data = r["geom"].num_rays + r["geom"].num_voxels
        rates.append(2.0 * r["nnz"] / per_iter)
        fixed.append(max(t[3] - 3.0 * per_iter, 0.0) / data)
    rate, fix = float(np.median(rates)), float(np.median(fixed))
    svc = np.array([2.0 * r["nnz"] * r["iters"] / rate + fix * (r["geom"].num_rays + r["geom"].num_voxels)
                    for r in reqs])
    return svc, {"updates_per_s": rate, "fixed_s_per_element": fix, "calibration_requests": idx}


def serving_compare(cbct, torch, dev, count, scale, slots, budget_gb, schedule, load=0.8):
    """The serving stream through the one-request-at-a-time solver and through
    the server, both fed in real time with the same Poisson arrivals.  The
    arrival rate is `load` x the one-at-a-time throughput predicted by the
    measured service model (calibrate_service)."""
    import numpy as np
    reqs = serving_requests(count, scale)
    serving_inputs(cbct, torch, dev, reqs)
    for r in reqs[:2]:                                  # warm-up of both paths (untimed)
        geom = cbct.Geometry(r["geom"])
        getattr(cbct, r["solver"])(geom, r["b"], 2)
        geom.close()
    server_arm(cbct, reqs[:2], [0.0, 0.0], slots, budget_gb, schedule)
    svc, model = calibrate_service(cbct, reqs)
    est_total_s = float(svc.sum())
    rate = load * len(reqs) / est_total_s
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    arrivals -= arrivals[0]
    lat_p, xs, span_p = plain_arm(cbct, reqs, arrivals)
    lat_s, span_s, diff, stats = server_arm(cbct, reqs, arrivals, slots, budget_gb, schedule, xs)
    return {"workload": "%d requests: %d^3..%d^3 volumes, %d..%d px square detectors, %d..%d angles, "
                        "LSQR/LSMR %d..%d iterations, I0 = 5e4" % (
                            len(reqs), min(r["geom"].nx for r in reqs), max(r["geom"].nx for r in reqs),
                            min(r["geom"].nu for r in reqs), max(r["geom"].nu for r in reqs),
                            min(r["geom"].nangles for r in reqs), max(r["geom"].nangles for r in reqs),
                            min(r["iters"] for r in reqs), max(r["iters"] for r in reqs)),
            "scale": scale, "offered_load": load, "arrival_rate_per_s": rate,
            "predicted_one_at_a_time_s": est_total_s, "service_model": model,
            "plain": latency_summary(lat_p, span_p, len(reqs)),
            "server": dict(latency_summary(lat_s, span_s, len(reqs)), schedule=schedule, max_slots=slots,
                           budget_gb=budget_gb, steps=stats["steps"], graph_replays=stats["graph_replays"]),
            "max_rel_diff_server_vs_plain": diff}


def run_serving(args):
    """The serving stream alone: one-at-a-time vs the server under each
    schedule (exploration; the default run reports the default schedule)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2211_14212_gb300 import cbct
    dev = torch.device("cuda", 0)
    out = {"mode": "serving"}
    for sched in args.serving_schedule.split(","):
        out[sched] = serving_compare(cbct, torch, dev, args.requests, args.serving_scale,
                                     args.serving_slots, args.serving_budget_gb, sched)
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["solve", "projectors", "serving", "precision", "microct", "profile-solve"],
                    default="solve",
                    help="solve: the benchmark step (default); projectors: standalone A / A^T timing; "
                         "serving: continuous-batching server vs one request at a time; "
                         "precision: FP32 / FP16 / BF16 storage study at 512^3")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--serving-scale", type=float, default=1.0)
    ap.add_argument("--serving-slots", type=int, default=16)
    ap.add_argument("--serving-budget-gb", type=float, default=96.0)
    ap.add_argument("--serving-schedule", default="fifo",
                    help="server schedule (fifo, srpt, ratio, share; --mode serving takes a comma list)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving stream in the default run")
    ap.add_argument("--fwd-rows", type=int, default=4, help="--mode profile-solve: forward rays per lane")
    ap.add_argument("--bwd-config", type=int, default=3, help="--mode profile-solve: transpose tile")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.mode == "projectors":
        sys.exit(run_projectors(args))
    if args.mode == "serving":
        sys.exit(run_serving(args))
    if args.mode == "precision":
        sys.exit(run_precision(args))
    if args.mode == "microct":
        sys.exit(run_microct(args))
    if args.mode == "profile-solve":
        sys.exit(run_profile_solve(args))
    sys.exit(run_reference(args) if args.impl == "reference" else run_ours(args))


if __name__ == "__main__":
    main()
