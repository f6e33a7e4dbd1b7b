"""The N>1 path on CPU: bench.py's replica plumbing over world_size-2 gloo
(barrier, max and sum over ranks), and the reference arm launched the way
the benchmark driver launches it (torch.distributed.run, 2 ranks): rank 0
alone prints one JSON line, every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SNIPPET = r"""
import os, sys
sys.path.insert(0, os.environ["LK_ROOT"])
from bench import Dist
d = Dist()
d.barrier()
assert d.world == 2
assert d.max(float(d.rank)) == 1.0
assert d.sum(1.0) == 2.0
assert d.max(10.0 - d.rank) == 10.0
d.barrier()
print("rank", d.rank, "ok")
"""


def test_dist_gloo_two_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), LK_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", SNIPPET], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate(timeout=180)[0] for p in procs]
    for r, (p, o) in enumerate(zip(procs, outs)):
        assert p.returncode == 0, o
        assert f"rank {r} ok" in o


def test_reference_arm_under_torchrun(oracle_lib):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["higher_is_better"] is False
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_submitter_cores_are_disjoint_per_rank(monkeypatch):
    """Each local rank pins its four submitting threads to its own cores, and
    leaves them unpinned when those cores are not in the process's set."""
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setattr(os, "sched_getaffinity", lambda pid: set(range(16)))
    assert [bench.submitter_cpus(r) for r in range(4)] == [2, 6, 10, -1]
    monkeypatch.setattr(os, "sched_getaffinity", lambda pid: {0, 1, 2, 3})
    assert bench.submitter_cpus(0) == -1


def test_percentiles_are_nearest_rank():
    """The bench's percentiles take the nearest rank over all samples: the
    ceil(q n)-th smallest value, never an interpolation."""
    sys.path.insert(0, ROOT)
    import bench

    v = list(range(100, 0, -1))                 # 1..100, unsorted
    assert bench.pct(v, 0.50) == 50 and bench.pct(v, 0.99) == 99 and bench.pct(v, 1.0) == 100
    assert bench.pct([3.0], 0.999) == 3.0 and bench.pct([], 0.5) is None
    assert bench.pct([1, 2, 3, 4, 5, 6, 7, 8, 9, 1000], 0.99) == 1000   # ceil(9.9) = 10th
    s = bench.lat_summary([5.0, 1.0, 3.0])
    assert (s["p50"], s["max"], s["count"]) == (3.0, 5.0, 3)
