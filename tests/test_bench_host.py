"""bench.py's host-side parts on CPU: the reference arm (the CPU oracle timed
on a bounded sample, one JSON line) and the parsing of the committed ncu
summaries it reads for the traffic and issue figures."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_line():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "cell-updates/s" and d["steps"] == 1 and d["warmup"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "bifluid_two_vortices_512x1024x128"


def test_reference_arm_other_ranks_stay_silent():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "0", env={"RANK": "1"})
    assert r.returncode == 0 and not r.stdout.strip()


@pytest.mark.parametrize("tag", ["stage_fp32", "stage_fp64"])
def test_committed_profiles_parse(tag):
    """Each stage-kernel summary carries the figures bench.py reads (whether
    its source hash is current is bench.py's own check at run time)."""
    import glob
    paths = glob.glob(os.path.join(ROOT, "profiles", f"{tag}__*.txt"))
    assert paths
    for path in paths:
        vals = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.split("#")[0].strip()
        assert float(vals["cells"]) > 0 and float(vals["dram_bytes_per_launch"]) > 0
        assert float(vals["warp_instructions_per_cell"]) > 0
        assert len(vals["source_hash"]) == 16


def test_cpu_baseline_uses_every_process():
    """The CPU baseline runs one oracle process per core it is given and
    reports the job's throughput over the common wall-clock span."""
    sys.path.insert(0, ROOT)
    import bench
    import synthetic as syn
    d = bench.cpu_baseline(syn.THROUGHPUT, steps=1, shape=(8, 12, 8), procs=2)
    assert d["cores"] == 2 and d["kind"] == "oracle" and d["value"] > 0
    assert d["value"] > d["per_process_value"]  # two processes at once beat one
