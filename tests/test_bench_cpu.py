"""The benchmark's output contract, checked on the CPU through its reference arm
(the float64 oracle timed on the host cores): one JSON line with the metric, value,
unit, CPU-baseline and end-to-end objects, printed by rank 0 only when several
ranks are launched."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--workload", "cov2d", "--size", "1024", "--steps", "1", "--warmup", "1"]


def _json_lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["impl"] == "reference"
    assert line["unit"] == "s" and line["higher_is_better"] is False
    assert line["value"] > 0 and line["ms_per_step"] == line["value"] * 1e3
    assert line["steps"] == 1 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert "cov2d N=1024" in line["config"]["workload"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == "s"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_two_ranks_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2", *ARGS]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1, r.stdout
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def test_reference_arm_on_a_lattice_family_rounds_the_size():
    """A 3D lattice family with a size that is not a cube: the run uses the largest
    cube below it (17^3 = 4913) and says so."""
    args = ["--impl", "reference", "--workload", "helmholtz3d", "--size", "5000", "--steps", "1", "--warmup", "1"]
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = _json_lines(r.stdout)[-1]
    assert "helmholtz3d N=4913" in line["config"]["workload"] and "N=4913" in line["cpu_baseline"]["sample"]
