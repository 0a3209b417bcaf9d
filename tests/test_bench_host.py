"""Host-side parts of bench.py on the CPU: the oracle's CPU-baseline sample and
the reference arm's JSON line (the FP64 oracle timed on the host cores), on a
tiny workload in place of the 256^3 one; the clock-record summary; and the
source hash that keys the stored ncu counters."""
import json
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import synth  # noqa: E402


@pytest.fixture
def tiny_workload(monkeypatch):
    g = synth.config("small")
    monkeypatch.setattr(bench, "workload_config", lambda: (g, {"workload": "small test scan"}))
    monkeypatch.setattr(bench, "REF_STEP_ANGLES", 4)
    for var in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(var, raising=False)
    return g


def test_cpu_baseline_sample_counts_the_sampled_updates(tiny_workload):
    g = tiny_workload
    rate, cores, dt, nnz = bench.oracle_sample_rate(g, 4)
    sub = g.angle_subset(4)
    assert sub.nangles == 4
    assert nnz == oracle.nnz(sub)
    assert cores >= 1 and dt > 0
    assert rate == pytest.approx(2 * nnz / dt / 1e9)


def test_reference_arm_prints_one_complete_line(tiny_workload, capsys):
    args = SimpleNamespace(gpus=1, steps=2, warmup=3)
    assert bench.run_reference(args) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["config"] == {"workload": "small test scan"}
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and "4 of" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only(tiny_workload, monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.run_reference(SimpleNamespace(gpus=2, steps=1, warmup=3)) == 0
    assert capsys.readouterr().out.strip() == ""


def test_clock_record_summary(tmp_path):
    """Median SM clock, the largest max clock and the throttle reasons seen
    active while the timed region ran, from nvidia-smi's CSV rows."""
    rows = [
        "0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1201.7, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(0)
    s.proc = object()                      # stands for the sampling process
    s.out = open(path, "a")
    try:
        summary = s.summary()
    finally:
        s.out.close()
    assert summary == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not path.exists()               # the temporary record is removed


def test_clock_record_absent_without_sampler():
    assert bench.ClockSampler(0).summary() is None


def test_projector_hash_ignores_comments_only():
    """The ncu counters stay attached to the kernels while only comments or
    whitespace change, and detach when the code changes."""
    base = {"projector.cu": 'int f(int a) { return a + 1; } // one\n/* two */ const char *s = "//x /*y*/";\n',
            "projector_device.cuh": "#pragma once\nint g();\n", "transpose.cuh": "int h();\n"}
    h = bench.projector_hash(base)
    recommented = {"projector.cu": '/* header */\nint f(int a)\n{\n    return a + 1;  // changed note\n}\n'
                                   'const char *s = "//x /*y*/";\n',
                   "projector_device.cuh": "#pragma once   // guard\nint g();\n",
                   "transpose.cuh": "int h();  /* tiles */\n"}
    assert bench.projector_hash(recommented) == h
    changed = dict(base, **{"projector.cu": base["projector.cu"].replace("a + 1", "a + 2")})
    assert bench.projector_hash(changed) != h
    in_string = dict(base, **{"projector.cu": base["projector.cu"].replace('"//x /*y*/"', '"//x /*z*/"')})
    assert bench.projector_hash(in_string) != h
    assert bench.projector_hash(dict(base, **{"transpose.cuh": "int h2();\n"})) != h
    assert bench.code_only('a /* b */ c // d\n  e') == "a c e"



def test_roofline_counters_follow_code_and_launch_shape(monkeypatch):
    """ncu counters enter the roofline line only for the kernel code and the
    launch shape they were taken on; otherwise traffic and the issue floor
    are null."""
    import synth
    g = synth.config("c2")
    h = bench.projector_hash()
    monkeypatch.setattr(bench, "NCU_COUNTERS", {
        "backward": {"hash": h, "shape": [4, 3], "dram_bytes": 3.0e9, "warp_inst": 3.75e10}})
    rl = bench.roofline_block(g, 2.8e10, 24.0, 38.0, {"sm_mhz": 2070.0}, (4, 3))
    assert rl["kernel"] == "backward" and rl["bound"] == "issue"
    assert rl["traffic"] == 3.0e9
    assert abs(rl["t_bound"]["issue_ms"] - 3.75e10 / (152 * 4 * 2070e6) * 1e3) < 1e-9
    assert abs(rl["frac"] - 2.8e10 * 4 / 38e-3 / 1e9 / rl["peak"]) < 1e-12
    other = bench.roofline_block(g, 2.8e10, 24.0, 38.0, {"sm_mhz": 2070.0}, (4, 1))
    assert other["traffic"] is None and other["t_bound"]["issue_ms"] is None
    monkeypatch.setattr(bench, "NCU_COUNTERS", {
        "backward": {"hash": "0" * 16, "shape": [4, 3], "dram_bytes": 3.0e9, "warp_inst": 3.75e10}})
    stale = bench.roofline_block(g, 2.8e10, 24.0, 38.0, {"sm_mhz": 2070.0}, (4, 3))
    assert stale["traffic"] is None and stale["issue_util"] is None


def test_calibrate_service_recovers_rate_and_fixed_cost(monkeypatch):
    """calibrate_service fits the one-at-a-time service time as
    fixed x (rays + voxels) + iters x 2 nnz / rate: on a fake library whose
    solves advance a fake clock by exactly that, the fit returns both
    constants and the predicted service of every request."""
    import types

    import numpy as np

    import synth
    rate, fixed = 1.0e9, 6.0e-10          # per-iteration times well above the fit's 1 us floor
    clock = [0.0]
    monkeypatch.setattr(bench.time, "perf_counter", lambda: clock[0])

    class Geometry:
        def __init__(self, g):
            self.g = g

        def close(self):
            pass

    def solve(geom, b, iters):
        r = by_id[id(geom.g)]
        clock[0] += fixed * (r["geom"].num_rays + r["geom"].num_voxels) + iters * 2.0 * r["nnz"] / rate
        return None, None

    fake = types.SimpleNamespace(Geometry=Geometry, lsqr=solve, lsmr=solve)
    reqs = []
    for i, n in enumerate((16, 24, 32, 40, 48)):
        g = synth.Geometry(n, n, n, 1.0, 1.0, 1.0, 2 * n, n, 1.0, 1.0, 400.0, 640.0, synth.circular_angles(10 + i))
        reqs.append({"geom": g, "solver": ["lsqr", "lsmr"][i % 2], "iters": 20 + i, "b": None,
                     "nnz": g.num_rays * n})
    by_id = {id(r["geom"]): r for r in reqs}
    svc, model = bench.calibrate_service(fake, reqs)
    assert abs(model["updates_per_s"] / rate - 1) < 1e-9
    assert abs(model["fixed_s_per_element"] / fixed - 1) < 1e-9
    want = [fixed * (r["geom"].num_rays + r["geom"].num_voxels) + r["iters"] * 2.0 * r["nnz"] / rate for r in reqs]
    assert np.allclose(svc, want, rtol=1e-9)
    assert model["calibration_requests"] == [0, 1, 3, 4]
