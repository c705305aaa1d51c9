"""Host-side checks of bench.py (no GPU): the reference arm's JSON line and
the reading of the committed ncu summary that feeds roofline.traffic."""
import json
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--cpu-sample", "5000"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "sorted strings/s" and line["unit"] == "strings/s"
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 0
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "url-16m" and line["config"]["n"] == 5000
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == bench.host_cores() and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0 and e2e["value"] == line["value"]


def test_scatter_traffic_is_read_only_for_the_captured_source(monkeypatch):
    tb = bench.ncu_traffic("k_scatter", "url-16m")
    # the committed summary names the kernel source it was captured on
    with open(os.path.join(ROOT, "profiles", "k_scatter_url-16m.txt")) as f:
        text = f.read()
    captured = text.split("source_sha256_16:")[1].split()[0]
    if captured == bench.kernel_source_sha():
        assert tb is not None and 30.0 < tb < 1000.0
    else:
        assert tb is None
    # any other source: no traffic figure
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("k_scatter", "url-16m") is None
    assert bench.ncu_traffic("k_scatter", "no-such-workload") is None


def _free_port():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(script_args, nproc=2):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(nproc),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), *script_args]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    return subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, timeout=600, env=env)


def test_times_reduce_to_the_slowest_rank_over_gloo():
    r = _torchrun([os.path.join(ROOT, "tests", "dist_reduce_helper.py")])
    assert r.returncode == 0, r.stderr[-2000:]
    got = sorted(re.findall(r"rank (\d+) max ([0-9.]+)", r.stdout))
    assert got == [("0", "2.0"), ("1", "2.0")]


def test_reference_arm_under_two_ranks_prints_one_line():
    r = _torchrun([os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0",
                   "--cpu-sample", "3000"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["impl"] == "reference"
