"""The N > 1 host path of bench.py on CPU: two gloo ranks, no GPU.

bench.py runs one process per GPU.  By default there is no data-path
collective (each rank searches its own resident copy: weak scaling); the only
communication is a barrier and the max-reduction of the elapsed time, and the
reference arm runs on rank 0 only.  With --shard each rank searches its shard
of one database and the score slices are all-gathered inside the end-to-end
step; here the CPU oracle stands in for each rank's GPU search."""

import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import io
    import sys
    from contextlib import redirect_stdout
    from types import SimpleNamespace

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    from workload import make_workload

    args = SimpleNamespace(impl="reference", gpus=world, steps=1, warmup=0)
    world_, rank_, local_, pg = bench.dist_setup(args)
    assert (world_, rank_) == (world, rank)
    bench.barrier(pg)
    t = bench.max_over_ranks(pg, 1.0 + rank)
    res = {"max": t}
    pg.destroy_process_group()
    # reference arm: rank 0 prints one JSON line, the others return silently
    w = make_workload("one_query_vs_2k", n_db=40)
    os.environ.update(MASTER_PORT=str(port + 1))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, w)
    res["stdout"] = buf.getvalue()
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["max"] == r1["max"] == 2.0
    line = json.loads(r0["stdout"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GCUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert r1["stdout"] == ""


def _shard_worker(rank, world, port, outdir):
    import sys

    import numpy as np
    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2412_08308_gb300.shard import partition
    from workload import make_workload
    from workload.matrices import BLOSUM62

    w = make_workload("one_query_vs_2k", n_db=150)
    parts = partition(w["db"].lengths, world)
    shard = w["db"].subset(parts[rank])
    full = bench.sharded_e2e_step(lambda: oracle.scores(w["queries"], shard, BLOSUM62, 10, 2), parts, dist)
    np.save(os.path.join(outdir, f"sharded{rank}.npy"), full)
    dist.destroy_process_group()


def test_sharded_bench_step_gathers_in_caller_order(tmp_path):
    import numpy as np

    import oracle
    from workload import make_workload
    from workload.matrices import BLOSUM62

    oracle.build()
    mp.start_processes(_shard_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    w = make_workload("one_query_vs_2k", n_db=150)
    exp = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"sharded{r}.npy"), exp)
