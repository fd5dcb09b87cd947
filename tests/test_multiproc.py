"""Multi-process paths on the CPU (gloo, world size 2).

The solver shards only as independent replicas (no data-path collective):
each rank advances its own instance and the benchmark reports the units all
ranks processed over the slowest rank's time.  These tests cover that host
logic -- the max-over-ranks reduction, the aggregation, and the torchrun
launch of the reference arm, where rank 0 alone runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(dist)
        m = bench.max_over_ranks(dist, 10.0 + rank)          # rank times 10 ms, 11 ms
        ms, value = bench.aggregate(dist, world, 1000, 10.0 + rank)
        q.put((rank, m, ms, value))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, ms, value in out:
        assert m == 11.0 and ms == 11.0
        # 2 ranks x 1000 units in the slowest rank's 11 ms
        assert value == pytest.approx(2 * 1000 / 11e-3)


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched like the multi-GPU bench: one JSON
    line from rank 0, the other rank exits 0 without work."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1",
           "--workload", "conservative_64"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["value"] > 0 and rec["cpu_baseline"]["kind"] == "oracle"
    assert rec["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.parametrize("workload", ["ensemble", "twa_ensemble", "drive_sweep"])
def test_reference_arm_for_batched_workloads(workload):
    """The reference arm (the oracle, timed on the host) runs on a bounded
    sample of each batched workload and prints the contract's JSON line."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
           "--workload", workload]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    rec = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert rec["impl"] == "reference" and rec["config"]["workload"] == workload
    assert rec["value"] > 0 and rec["unit"] == "site-updates/s" and rec["higher_is_better"]
    # every host core runs a copy of the oracle, one process each
    assert rec["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert rec["e2e"]["d2h_bytes_per_step"] == 0
