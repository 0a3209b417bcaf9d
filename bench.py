#!/usr/bin/env python
"""Benchmark of the Krylov CBCT hot path on GB300.

Workload (the 256^3 medical configuration): 256^3 x 1 mm volume, 512 x 512
detector of 0.8 mm pixels, 360 angles over 360 deg, DSO 1000 / DSD 1536 mm,
random-ellipsoid phantom x 0.02 mm^-1, Poisson noise with I0 = 1e5.  One step
= LSQR 30 iterations + LSMR 30 iterations on that b (both through the C ABI,
FP32 vectors, FP64 scalars).

Printed JSON line (rank 0):
  value      ray-voxel Gupdates/s of the whole step (nnz(A) x projector
             launches / step time), inputs resident in HBM;
  e2e        the same metric with b read from pinned host memory and x
             written back to the host inside the timed region;
  roofline   the dominant projector kernel: nnz x 4 B gathered per launch /
             its CUDA-event launch time, against the measured HBM copy peak;
  cpu_baseline  the FP64 oracle on the host cores, on an 8-angle sample.
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

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by the code of the projector sources it was measured on
# (projector_hash(), comments ignored); the bench reports null once that code
# changed.
NCU_TRAFFIC = {
    # one launch of the 2x4x128 transpose tile at 256^3 / 512^2 / 360 (ncu --set full,
    # the cbct_backproject launch of the projectors mode; the solver's launch of the
    # same tile differs only in the output layout): 11.800 GB read + 0.122 GB written
    "backward": (11921397568, "5075f4334a6e209e"),
}


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
    """sha256 over the code of the projector kernel sources (projector.cu +
    projector_device.cuh, comments and whitespace dropped), first 16 hex
    digits: the ncu counters stay attached to the kernels while only their
    comments change."""
    h = hashlib.sha256()
    for name in ("projector.cu", "projector_device.cuh"):
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

    # ---- timed region: inputs resident in HBM
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and all(p.strip().isdigit() for p in vis.split(",")):
        gpu_index = int(vis.split(",")[local])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    products = launches = 0
    fwd_ms = bwd_ms = 0.0
    fwd_n = bwd_n = 0
    lsqr_s = 0.0
    with ClockSampler(gpu_index) as clk:
        with torch.cuda.stream(s):
            torch.cuda.nvtx.range_push("timed")        # lets a profiler select the timed launches
            ev0.record(s)
            for _ in range(args.steps):
                t0 = time.perf_counter()
                r1, r2, t1 = step(b, x1, x2, True)
                lsqr_s += t1 - t0          # the solver synchronises its stream before returning
                for r in (r1, r2):
                    products += r.forward_launches + r.backward_launches
                    launches += r.kernel_launches
                    fwd_ms += r.forward_ms
                    bwd_ms += r.backward_ms
                    fwd_n += r.forward_launches
                    bwd_n += r.backward_launches
            ev1.record(s)
            torch.cuda.nvtx.range_pop()
        barrier()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    clocks = clk.summary()
    value = whole_job_rate(nnz * products, world, elapsed_ms * 1e-3) / 1e9
    lsqr_ips = ITERS * args.steps / lsqr_s

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

    if rank != 0:
        return 0
    dominant = "forward" if fwd_ms >= bwd_ms else "backward"
    avg_ms = fwd_ms / max(fwd_n, 1) if dominant == "forward" else bwd_ms / max(bwd_n, 1)
    peak, peak_kind = measured_peak()
    achieved = nnz * BYTES_PER_UPDATE / (avg_ms * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get(dominant)
    traffic = tr[0] if tr and tr[1] == projector_hash() else None
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
        "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "avg_launch_ms": avg_ms,
                     "forward_ms_per_launch": fwd_ms / max(fwd_n, 1),
                     "backward_ms_per_launch": bwd_ms / max(bwd_n, 1)},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * 4 * geom.num_rays,
                "d2h_bytes_per_step": 2 * 4 * geom.num_voxels},
        "gpu_launches": launches,
        "clocks": clocks,
        "launch_shapes": {"fwd_rows": tune["fwd_rows"], "bwd_brick": tune["bwd_shape"]},
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


def run_precision(args):
    """Storage-precision study on the 512^3 scan (768 x 512 detector, 720 angles,
    noisy): hybrid LSQR 50 iterations with GCV, Krylov vectors and basis stored
    in FP32, FP16 or BF16 (FP32 ray sums, FP64 scalars); time per iteration,
    throughput, and the difference of each result from the FP32 one."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    g = synth.config("c3")
    dev = torch.device("cuda", 0)
    geom = cbct.Geometry(g)
    tune = cbct.autotune(geom, max_angles=32)
    x_true = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=2, scale=0.02)).to(dev)
    b = cbct.project(geom, x_true).cpu().numpy()
    b = torch.from_numpy(synth.poisson_log_noise(b, 1e5, seed=25).astype(np.float32)).to(dev)
    nnz = cbct.count_nnz(geom)
    iters = 50
    out = {"mode": "precision", "config": {"workload": "512^3 CBCT precision study: hybrid LSQR 50 (GCV)",
                                           "volume": [g.nx, g.ny, g.nz], "voxel_mm": g.dx,
                                           "detector": [g.nu, g.nv], "pixel_mm": g.du, "angles": g.nangles,
                                           "dso_mm": g.dso, "dsd_mm": g.dsd, "noise": "Poisson I0=1e5"},
           "nnz": nnz, "launch_shapes": {"fwd_rows": tune["fwd_rows"], "bwd": tune["bwd_shape"]}, "storage": {}}
    ref = None
    xt = x_true.double()
    for storage in ("f32", "f16", "bf16"):
        cbct.hybrid_lsqr(geom, b, 2, storage=storage)                    # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, rep = cbct.hybrid_lsqr(geom, b, iters, storage=storage)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        xd = x.double()
        if ref is None:
            ref = xd.clone()
        out["storage"][storage] = {
            "s_per_solve": dt, "ms_per_iter": 1000 * dt / iters,
            "gupdates_per_s": 2 * nnz * iters / dt / 1e9,
            "rel_diff_vs_f32": float((xd - ref).norm() / ref.norm()),
            "rel_err_vs_phantom": float((xd - xt).norm() / xt.norm()),
            "lambda_last": float(rep.lam[-1]), "resid_last": float(rep.resid[-1])}
        del x, xd
    print(json.dumps(out), flush=True)
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


def run_serving(args):
    """Continuous-batching server vs the one-request-at-a-time solver on the
    serving stream (Poisson arrivals at 0.8 of the one-at-a-time throughput)."""
    import threading

    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import synth
    from paper_2211_14212_gb300 import cbct
    dev = torch.device("cuda", 0)
    reqs = serving_requests(args.requests, args.serving_scale)
    gen = torch.Generator(device=dev)
    # measured projections: GPU forward projection + Poisson photon noise (input generation)
    for r in reqs:
        g = r["geom"]
        geom = cbct.Geometry(g)
        x = torch.from_numpy(synth.ellipsoid_phantom(g, 10, seed=r["seed"], scale=0.02)).to(dev)
        b = cbct.project(geom, x)
        gen.manual_seed(r["seed"])
        counts = torch.poisson(5e4 * torch.exp(-b), generator=gen)
        r["b"] = (-torch.log(torch.clamp(counts, min=1.0) / 5e4)).float().cpu().numpy().ravel()
        del x, b, counts, geom
    torch.cuda.synchronize()
    # one request at a time (plain solver, host b and x: end to end)
    service, keep = [], {}
    for i, r in enumerate(reqs[:2]):                      # warm-up
        getattr(cbct, r["solver"])(cbct.Geometry(r["geom"]), r["b"], 2)
    for i, r in enumerate(reqs):
        t0 = time.perf_counter()
        geom = cbct.Geometry(r["geom"])
        x, _ = getattr(cbct, r["solver"])(geom, r["b"], r["iters"])
        service.append(time.perf_counter() - t0)
        if i < 8:
            keep[i] = x
        del geom
    total = sum(service)
    rate = 0.8 * len(reqs) / total
    rng = np.random.default_rng(4)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    arrivals -= arrivals[0]
    finish, t = [], 0.0
    for a, sv in zip(arrivals, service):
        t = max(t, a) + sv
        finish.append(t)
    lat_plain = np.array(finish) - arrivals
    plain = {"recon_per_s": len(reqs) / (finish[-1] - arrivals[0]), "p50_s": float(np.percentile(lat_plain, 50)),
             "p99_s": float(np.percentile(lat_plain, 99)), "mean_service_s": total / len(reqs)}
    # the server, fed in real time, under each schedule
    def serve(schedule):
        srv = cbct.Server(int(args.serving_budget_gb * (1 << 30)), max_slots=args.serving_slots, use_graph=True,
                          schedule=schedule)
        ids = [None] * len(reqs)
        t_start = time.perf_counter()

        def feeder():
            for i, (a, r) in enumerate(zip(arrivals, reqs)):
                dt = a - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
                ids[i] = srv.submit(r["geom"], r["b"], r["solver"], r["iters"])

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        results = [srv.wait(i) for i in ids]
        stats = srv.stats()
        srv.close()
        lat = np.array([r.finish_s - r.submit_s for r in results])
        first = min(r.submit_s for r in results)
        last = max(r.finish_s for r in results)
        diffs = [float(np.linalg.norm(results[i].x - keep[i]) / np.linalg.norm(keep[i])) for i in keep]
        return {"recon_per_s": len(reqs) / (last - first), "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()), "steps": stats["steps"],
                "graph_replays": stats["graph_replays"], "max_slots": args.serving_slots,
                "budget_gb": args.serving_budget_gb,
                "max_rel_diff_vs_plain": max(diffs) if diffs else None}

    plain["mean_s"] = float(lat_plain.mean())
    out = {"mode": "serving", "requests": len(reqs), "offered_load": 0.8, "arrival_rate_per_s": rate,
           "scale": args.serving_scale, "unit": "recon/s",
           "plain_one_at_a_time": plain,
           "server_srpt": serve("srpt"),
           "server_ratio": serve("ratio"),
           "server_share": serve("share"),
           "request_mix": [r["desc"] + [r["solver"], r["iters"]] for r in reqs]}
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["solve", "projectors", "serving", "precision"], default="solve",
                    help="solve: the benchmark step (default); projectors: standalone A / A^T timing; "
                         "serving: continuous-batching server vs one request at a time; "
                         "precision: FP32 / FP16 / BF16 storage study at 512^3")
    ap.add_argument("--requests", type=int, default=64)
    ap.add_argument("--serving-scale", type=float, default=1.0)
    ap.add_argument("--serving-slots", type=int, default=16)
    ap.add_argument("--serving-budget-gb", type=float, default=96.0)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.mode == "projectors":
        sys.exit(run_projectors(args))
    if args.mode == "serving":
        sys.exit(run_serving(args))
    if args.mode == "precision":
        sys.exit(run_precision(args))
    sys.exit(run_reference(args) if args.impl == "reference" else run_ours(args))


if __name__ == "__main__":
    main()
