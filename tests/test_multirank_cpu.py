"""The N > 1 host path of bench.py on CPU: two gloo ranks, no GPU.

bench.py runs one process per GPU with no data-path collective (each rank
searches its own resident copy: weak scaling).  The only communication is a
barrier and the max-reduction of the elapsed time; the reference arm runs on
rank 0 only."""

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
