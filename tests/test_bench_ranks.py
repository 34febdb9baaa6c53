"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank runs its own
replica, so the only cross-rank operations are the barrier and the max over ranks of the
timed interval; rank 0 alone prints.  The reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, ws, local = bench.dist_setup()
    assert (r, ws, local) == (rank, world, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(ws)
    m = bench.max_over_ranks(10.0 + rank, ws)
    q.put((rank, m))
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 11.0), (1, 11.0)]


def test_reference_arm_runs_on_rank0_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.workload_name(2048, "fp32", 0.0) == "kh_jet_2048x2048_dns_fp32"
    assert bench.workload_name(256, "fp32", 2.0) == "kh_jet_256x256_les_delta2_fp32"


def test_reference_arm_line_on_rank0():
    """Rank 0 of the reference arm times the oracle and prints one JSON line with the contract's
    keys; its e2e and cpu_baseline are the line's own value."""
    import json
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--n", "64"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_traffic_key_ignores_comments_and_whitespace():
    """The measured DRAM traffic is keyed by a hash of the kernel source that comment and
    whitespace edits do not change, while any code edit does."""
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int a) {\n  return a + 1;  // one\n}\n/* block */\n"
    same = "int f(int a){return a+1;}\n// another comment\n/* a\n longer block */"
    other = "int f(int a) { return a + 2; }"
    assert bench.source_hash(code) == bench.source_hash(same)
    assert bench.source_hash(code) != bench.source_hash(other)
    assert len(bench.kernel_hash()) == 16


def test_timed_windows_cover_five_repeats_and_one_second():
    """The K-step interval is timed at least 5 times and for at least one second in all,
    whatever K is (a 20-step run of a 0.14 ms step needs hundreds of windows)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.windows_needed(0.14, 20) == int(np.ceil(1.0 / (0.14e-3 * 20)))
    assert bench.windows_needed(0.14, 20) * 20 * 0.14e-3 >= 1.0
    assert bench.windows_needed(1.8, 20000) == 5       # long windows: the five repeats decide
    assert bench.windows_needed(0.0, 20) >= 5           # a zero estimate does not divide by zero
