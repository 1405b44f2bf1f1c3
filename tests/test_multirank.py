"""Multi-process (world size 2, gloo on CPU) coverage of the benchmark's rank logic.

The correlation shards by independent problems: each rank runs its own problem
and the only cross-rank operations are the timing barrier and the max-over-ranks
reduction.  These run here without a GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    got = bench.reduce_max(dist, 10.0 + rank, "cpu")
    with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
        f.write(repr(got))
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = 29511
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    assert vals == [11.0, 11.0]


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", "29513", "bench.py", "--impl",
           "reference", "--workload", "c2", "--steps", "1", "--warmup", "0",
           "--cpu-sample-n", "128"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_row_shards_cover_every_row_once():
    import paper_1808_00685_gb300 as pkg
    for n1 in (1, 127, 128, 129, 700, 32768):
        for world in (1, 2, 3, 4, 8):
            rows = []
            for rank in range(world):
                r0, cnt = pkg.shard_rows(n1, world, rank)
                assert r0 % 128 == 0 or cnt == 0
                rows.extend(range(r0, r0 + cnt))
            assert rows == list(range(n1))
