"""Host-side logic of bench.py (no GPU): roofline bookkeeping, the capture
record's source check, and the reference arm's JSON line (the oracle timed on
the host on a bounded sample)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_roofline_is_algorithmic_bytes_over_launch_time():
    # 7 launches, 0.2625 ms in total, 13 B per point of a 2048^2 grid per launch
    nbytes = 7 * 13 * 2048 * 2048
    r = bench.kernel_roofline(2, 7, 0.2625, nbytes, 6776.6, "measured", 152, 2070.0)
    assert r["avg_launch_us"] == pytest.approx(37.5)
    # the unfused steps' 33 B per point (two sweeps of 3 words, prolongation +
    # correction 2.25 words); the fused kernel's compulsory 13 B beside it
    assert r["achieved"] == pytest.approx(33 * 2048 * 2048 / 37.5e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6776.6)
    assert r["compulsory"]["achieved"] == pytest.approx(13 * 2048 * 2048 / 37.5e-6 / 1e9)
    outer = bench.kernel_roofline(3, 4, 0.12, 4 * 20 * 2048 * 2048, 6776.6, "measured")
    assert outer["achieved"] == pytest.approx(20 * 2048 * 2048 / 30e-6 / 1e9) and "compulsory" not in outer
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    cap = bench.read_capture(2)
    if cap is not None:  # the committed capture matches this source
        assert r["traffic"] == cap["dram_bytes_per_launch"]
        wf = cap["smem_wavefronts_per_launch"]
        assert r["smem"]["frac"] == pytest.approx(wf / 37.5e-6 / (152 * 2070e6))
    coarse = bench.kernel_roofline(5, 7, 0.56, 7 * 36e6, 6776.6, "measured")
    assert coarse["bound"] == "launch/latency" and coarse["frac"] is None
    assert bench.kernel_roofline(1, 0, 0.0, 0.0, 6776.6, "measured") is None


def test_capture_record_is_ignored_for_another_source(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 40)
    assert bench.read_capture(1) is None
    r = bench.kernel_roofline(1, 7, 0.17, 7 * 47e6, 6776.6, "measured", 152, 2070.0)
    assert r["traffic"] is None and "smem" not in r


def test_capture_record_matches_the_committed_kernels():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    for kind in ("1", "2", "3", "6"):
        assert d[kind]["source_sha1"] == bench.kernel_source_sha(), f"kind {kind}: recapture or refresh"
        assert os.path.exists(os.path.join(ROOT, d[kind]["profile"]))


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    line = json.loads(lines[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "solves/s"
    assert line["higher_is_better"] is True and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]


def test_profile_commands_name_committed_entry_points():
    """Every ncu summary under profiles/ gives its command; the commands run
    committed entry points with options those entry points accept, and every
    command line has --clock-control none on its ncu invocation."""
    import glob
    import re
    ops = set(re.findall(r'"(\w+)"', open(os.path.join(ROOT, "profile_ops.py")).read()
                         .split('choices=[', 1)[1].split(']', 1)[0]))
    bench_flags = set(re.findall(r'add_argument\("(--[\w-]+)"', open(os.path.join(ROOT, "bench.py")).read()))
    md = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert md
    for path in md:
        text = open(path).read()
        cmd = text.split("Command", 1)[1].split("\n\n", 2)[1]  # the indented block after the heading line
        cmd = cmd.replace("\\\n", " ")
        assert "ncu " in cmd and "--clock-control none" in cmd, path
        for op in re.findall(r"profile_ops(?:\.py)? --op (\w+)", cmd):
            assert op in ops, (path, op)
        if "bench.py" in cmd:
            for flag in re.findall(r"(--[\w-]+)", cmd.split("bench.py", 1)[1]):
                if flag.startswith(("--metrics", "--clock-control", "--csv", "--log-file", "--set")):
                    continue
                assert flag in bench_flags, (path, flag)


def test_all_cores_cpu_figure_runs_one_solve_per_process():
    import numpy
    bench.np = numpy  # bench.main() binds it; the legs use the module global
    r = bench.cpu_all_cores()
    assert r.get("error") is None, r
    assert r["cores"] >= 1 and r["value"] > 0 and r["kind"] == "oracle"
