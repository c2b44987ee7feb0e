"""Host-side logic of bench.py (no GPU): the reference arm's JSON line, the
rank guard of that arm, and the lookup of DRAM traffic records from the ncu
summaries under profiles/ with its source-hash guard."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                          cwd=ROOT, env=e, timeout=600)


def test_reference_arm_prints_one_json_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"], env={"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == "", (r.stdout, r.stderr)


RECORDS = [("cpl_state_apply_kernel<0,false>", "slab_128x128x8_q2p1"),
           ("state_apply_kernel<float,false>", "slab_64x64x4_q3q1"),
           ("state_apply_kernel<float,false>", "slab_64x64x4_q4p3"),
           ("state_apply_kernel<float,false>", "forest_64x64x4_q3p2")]


def _record(kernel, workload):
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        for line in open(os.path.join(ROOT, "profiles", name)):
            if line.startswith("traffic-record:"):
                rec = json.loads(line.split(":", 1)[1])
                if rec["kernel"] == kernel and rec["workload"] == workload:
                    return rec, name
    return None, None


@pytest.mark.parametrize("kernel,workload", RECORDS)
def test_traffic_records_follow_the_kernel_sources(kernel, workload, monkeypatch):
    rec, name = _record(kernel, workload)
    assert rec is not None, (kernel, workload)
    got, src = bench.captured_traffic(kernel, workload)
    if rec["source_sha"] == bench.kernel_source_sha():
        assert got == rec["dram_bytes_per_launch"] and src == f"profiles/{name}"
    else:
        assert got is None and "changed" in src
    # any change of the kernel sources makes the record stale
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    got, src = bench.captured_traffic(kernel, workload)
    assert got is None and "changed" in src


def test_traffic_lookup_without_a_capture():
    got, src = bench.captured_traffic("cpl_state_apply_kernel<0,false>", "no_such_workload")
    assert got is None and src == "no capture of this kernel and workload"
