"""The multi-GPU form is replicas (one subject per rank, no collective on the data
path): the whole-job figure is all ranks' units over the slowest rank's time. Checked
with world_size-2 gloo process groups on the CPU, and the torchrun launch of the
reference arm (rank 0 alone prints its line, the other rank exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    r, lr, w = bench.dist_env()
    ms = [1200.0, 1500.0][rank]  # the second replica is the slower one
    m = bench.max_over_ranks(ms, w, "cpu")
    units = 50.544e9
    val = bench.replica_throughput(units, 5, m, w)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, lr, w, m, val))


def test_max_over_ranks_and_whole_job_throughput_gloo():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, lr, ws, m, val) in enumerate(res):
        assert (rank, lr, ws) == (r, r, 2)
        assert m == 1500.0
        assert val == pytest.approx(2 * 50.544e9 * 5 / 1.5 / 1e9)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.replica_throughput(1e9, 2, 1000.0, 1) == pytest.approx(2.0)


def test_torchrun_reference_arm_two_ranks(tmp_path):
    env = dict(os.environ, MUSTER_PHANTOM_CACHE=str(tmp_path), OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
           "--workload", "c1", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1  # rank 0 alone
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
