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


def test_uneven_batch_sub_batches_fit_the_budget():
    """The sub-batch split of the uneven batch (host logic): the default batch fits one
    GPU in one piece, the full-size batch splits into pieces within the budget."""
    import argparse
    import bench
    from h2gen import uneven_sizes
    base = dict(nsys=64, nmin=2048, mem_per_point_kb=240.0, mem_budget_gb=245.0)
    sizes, bins = bench._subbatches(argparse.Namespace(nmax=16384, **base), 0, 1)
    assert len(bins) == 1 and sorted(bins[0]) == list(range(64))
    sizes, bins = bench._subbatches(argparse.Namespace(nmax=131072, **base), 0, 1)
    assert sizes == uneven_sizes(64, 2048, 131072)
    assert len(bins) >= 2 and sorted(i for b in bins for i in b) == list(range(64))
    assert all(sum(sizes[i] for i in b) * 240e3 <= 245e9 for b in bins)
    # two ranks: each rank's share is split on its own
    _, b0 = bench._subbatches(argparse.Namespace(nmax=131072, **base), 0, 2)
    _, b1 = bench._subbatches(argparse.Namespace(nmax=131072, **base), 1, 2)
    assert sorted(i for b in b0 + b1 for i in b) == list(range(64))
