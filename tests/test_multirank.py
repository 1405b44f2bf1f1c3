"""Multi-process (world size 2, gloo on CPU) coverage of the multi-GPU logic.

Three ways to use several GPUs: independent problems per rank (the only
cross-rank operations are the timing barrier and the max-over-ranks
reduction), one problem split by output tiles (corr2d_compute_part: each rank
computes a balanced, contiguous part of the mirrored tile list and its
mirrored blocks; the parts cover the map exactly once), and one batch split by
problem (corr2d_plan_batch_part: a cost-balanced assignment, each rank running
corr2d_batch on its problems).  The partitions are host logic, so they are
checked here without a GPU: coverage and balance for many shapes, and two gloo
ranks that compute their parts with the oracle and gather the results."""
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


# ------------------------------------------------------- tile parts (one problem)

def _lib():
    import paper_1808_00685_gb300 as pkg
    pkg.load(pkg.build())
    return pkg


def _written(n1, n2, homo, tiles, mirror=True):
    """Boolean map of the outputs a part writes: each tile's block and, for an
    off-diagonal mirrored tile, the transposed block (a diagonal tile writes its
    whole block: its upper triangle and the mirror of it)."""
    import numpy as np
    w = np.zeros((n1, n2), np.int32)
    for ti, tj in tiles:
        w[ti * 128:(ti + 1) * 128, tj * 128:(tj + 1) * 128] += 1
        if homo and mirror and ti != tj:
            w[tj * 128:(tj + 1) * 128, ti * 128:(ti + 1) * 128] += 1
    return w


@pytest.mark.parametrize("n1,n2,homo", [(700, 700, True), (128, 128, True), (129, 129, True),
                                        (1000, 333, False), (4096, 4096, True)])
@pytest.mark.parametrize("nparts", [1, 2, 3, 5, 8])
def test_tile_parts_write_every_output_exactly_once(n1, n2, homo, nparts):
    """corr2d_plan_part (host only): the parts are disjoint, their blocks and mirrored
    blocks cover the n1 x n2 map exactly once, and their costs are balanced."""
    import numpy as np
    pkg = _lib()
    total = np.zeros((n1, n2), np.int32)
    costs = []
    for part in range(nparts):
        tiles = pkg.corr2d_plan_part(n1, n2, homo, 0, part, nparts)
        total += _written(n1, n2, homo, tiles)
        costs.append(sum(1 + (2 if homo and a != b else 1) for a, b in tiles))
    assert np.all(total == 1)
    nt = len(pkg.corr2d_plan_part(n1, n2, homo, 0, 0, 1))
    if nt >= 8 * nparts:  # balanced to within a few tiles' cost
        assert max(costs) - min(costs) <= 8
    # NO_MIRROR: every tile of the map, no mirrored blocks
    tiles = sum((pkg.corr2d_plan_part(n1, n2, homo, pkg.FLAG_NO_MIRROR, p, nparts)
                 for p in range(nparts)), [])
    assert np.all(_written(n1, n2, homo, tiles, mirror=False) == 1)


def _part_worker(rank, world, port, out):
    """One rank: its share of the tiles of a homo problem, each tile's block computed
    by the oracle from the stacks' columns of that block (every step before the
    cross product acts on one spectral variable at a time) and its mirror from the
    symmetry Phi(nu2, nu1) = Phi(nu1, nu2), Psi(nu2, nu1) = -Psi(nu1, nu2); the ranks'
    maps are gathered with gloo and rank 0 checks them against one full oracle call."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import oracle
    import paper_1808_00685_gb300 as pkg
    import workloads
    pkg.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, m = 300, 9
    y = workloads.random_stack(m, n, seed=77, offset=2.0)
    phi = np.full((n, n), np.nan)
    psi = np.full((n, n), np.nan)
    for ti, tj in pkg.corr2d_plan_part(n, n, True, 0, rank, world):
        r = np.arange(ti * 128, min(n, ti * 128 + 128))
        c = np.arange(tj * 128, min(n, tj * 128 + 128))
        bp, bq, _, _ = oracle.corr2d(np.ascontiguousarray(y[:, r]), np.ascontiguousarray(y[:, c]))
        phi[np.ix_(r, c)] = bp
        psi[np.ix_(r, c)] = bq
        if ti != tj:
            phi[np.ix_(c, r)] = bp.T
            psi[np.ix_(c, r)] = -bq.T
    parts = [torch.zeros((2, n, n), dtype=torch.float64) for _ in range(world)]
    dist.all_gather(parts, torch.from_numpy(np.stack([phi, psi])))
    if rank == 0:
        got = np.stack([p.numpy() for p in parts])  # world x 2 x n x n
        written = ~np.isnan(got)
        ok_once = bool(np.all(written.sum(axis=0) == 1))
        full = np.where(written, got, 0.0).sum(axis=0)
        ophi, opsi, _, _ = oracle.corr2d(y)
        with open(os.path.join(out, "result.txt"), "w") as f:
            f.write(repr((ok_once, bool(np.array_equal(full[0], ophi)),
                          bool(np.array_equal(full[1], opsi)))))
    dist.destroy_process_group()


def test_two_gloo_ranks_compute_their_tile_parts_and_gather_the_full_map(tmp_path):
    import torch.multiprocessing as mp
    _lib()
    mp.spawn(_part_worker, args=(2, 29517, str(tmp_path)), nprocs=2, join=True)
    assert open(tmp_path / "result.txt").read() == repr((True, True, True))


def _batch_cost(m, n1, n2, homo):
    """Cost of one problem in units of one output pair (the documented model)."""
    return n1 * (n1 if homo else n2) + 3 * m * (n1 if homo else n1 + n2)


@pytest.mark.parametrize("nparts", [1, 2, 3, 4, 8, 600])
def test_batch_parts_cover_every_problem_once_and_balance_cost(nparts):
    import workloads
    import paper_1808_00685_gb300 as pkg
    _lib()
    spec = workloads.c5_spec()
    shapes = [(p.m, p.n1, p.n2, p.homo) for p in spec.problems]
    parts = [pkg.plan_batch_part(shapes, r, nparts) for r in range(nparts)]
    flat = sorted(i for part in parts for i in part)
    assert flat == list(range(len(shapes)))  # every problem in exactly one part
    assert all(part == sorted(part) for part in parts)
    cost = [_batch_cost(*s) for s in shapes]
    loads = [sum(cost[i] for i in part) for part in parts]
    mean = sum(cost) / nparts
    assert max(loads) - mean < max(cost)  # greedy bound: less than one problem above the mean
    # the same shapes give the same split (every process computes it alone)
    assert parts == [pkg.plan_batch_part(shapes, r, nparts) for r in range(nparts)]


def test_batch_parts_follow_the_greedy_rule_on_a_small_list():
    """Costs 1000, 400, 250, 160 over 2 parts: by decreasing cost, each to the lighter
    part -> {0} and {1, 2, 3} (1000 against 810)."""
    import paper_1808_00685_gb300 as pkg
    _lib()
    # homo n1 = 10: cost = 100 + 30 m
    shapes = [(30, 10, 0, True), (10, 10, 0, True), (5, 10, 0, True), (2, 10, 0, True)]
    costs = [_batch_cost(*s) for s in shapes]
    assert costs == [1000, 400, 250, 160]
    assert pkg.plan_batch_part(shapes, 0, 2) == [0]
    assert pkg.plan_batch_part(shapes, 1, 2) == [1, 2, 3]
    # ties go to the lower index, then to the lower part
    same = [(4, 8, 0, True)] * 5
    assert pkg.plan_batch_part(same, 0, 2) == [0, 2, 4]
    assert pkg.plan_batch_part(same, 1, 2) == [1, 3]


def test_batch_part_arguments_are_checked():
    import paper_1808_00685_gb300 as pkg
    _lib()
    with pytest.raises(pkg.Corr2dError):
        pkg.plan_batch_part([(8, 10, 0, True)], 2, 2)  # part out of range
    with pytest.raises(pkg.Corr2dError):
        pkg.plan_batch_part([(1, 10, 0, True)], 0, 1)  # m < 2
    with pytest.raises(pkg.Corr2dError):
        pkg.plan_batch_part([(8, 0, 0, True)], 0, 1)  # n1 < 1
    assert pkg.plan_batch_part([], 0, 3) == []


def _batch_part_worker(rank, world, port, out):
    """One rank: the oracle on its problems of a small ragged batch; the ranks' results
    are gathered with gloo and rank 0 checks that every problem was computed once and
    equals one oracle call over the whole list."""
    import numpy as np
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import oracle
    import paper_1808_00685_gb300 as pkg
    import workloads
    pkg.load()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = workloads.c5_spec(count=9, seed=5, m_lo=3, m_hi=20, n_lo=8, n_hi=60)
    ins = workloads.batch_inputs(spec, nbands=3)
    shapes = [(p.m, p.n1, p.n2, p.homo) for p in spec.problems]
    mine = {}
    for i in pkg.plan_batch_part(shapes, rank, world):
        y1, y2 = ins[i]
        phi, psi, _, _ = oracle.corr2d(y1, y2)
        mine[i] = (phi.tolist(), psi.tolist())
    got = [None] * world
    dist.all_gather_object(got, mine)
    if rank == 0:
        merged = {}
        twice = False
        for d in got:
            for i, v in d.items():
                twice = twice or i in merged
                merged[i] = v
        ok = not twice and sorted(merged) == list(range(len(shapes)))
        for i, (y1, y2) in enumerate(ins):
            phi, psi, _, _ = oracle.corr2d(y1, y2)
            ok = ok and np.array_equal(np.array(merged[i][0]), phi)
            ok = ok and np.array_equal(np.array(merged[i][1]), psi)
        with open(os.path.join(out, "result.txt"), "w") as f:
            f.write(repr(ok))
    dist.destroy_process_group()


def test_two_gloo_ranks_compute_their_batch_parts_and_gather_every_problem(tmp_path):
    import torch.multiprocessing as mp
    _lib()
    mp.spawn(_batch_part_worker, args=(2, 29519, str(tmp_path)), nprocs=2, join=True)
    assert open(tmp_path / "result.txt").read() == "True"
