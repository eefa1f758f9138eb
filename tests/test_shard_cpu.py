"""Database sharding across ranks (host logic, no GPU): the partition, the
shard extraction and the gather of score slices over two gloo ranks, with the
CPU oracle standing in for each rank's GPU search."""

import os
import socket

import numpy as np
import torch.multiprocessing as mp

import oracle
from paper_2412_08308_gb300.shard import gather_scores, partition, subset
from workload import from_list, make_workload
from workload.matrices import BLOSUM62


def test_partition_covers_balances_and_stratifies():
    w = make_workload("one_query_vs_2k")
    lengths = w["db"].lengths
    for n in (1, 2, 3, 8):
        parts = partition(lengths, n)
        allidx = np.concatenate(parts)
        assert np.array_equal(np.sort(allidx), np.arange(lengths.size))    # every sequence exactly once
        assert max(map(len, parts)) - min(map(len, parts)) <= 1
        res = [int(lengths[p].sum()) for p in parts]
        assert max(res) - min(res) <= int(lengths.max())                  # residue-balanced
        med = [float(np.median(lengths[p])) for p in parts]
        assert max(med) - min(med) <= 0.05 * float(np.median(lengths))    # same length mix


def test_subset_round_trip():
    rng = np.random.Generator(np.random.PCG64(5))
    seqs = [rng.integers(0, 20, size=int(n)).astype(np.uint8) for n in (0, 5, 1, 30, 0, 7)]
    db = from_list(seqs)
    idx = np.array([3, 0, 5, 1])
    res, off = subset(db.residues, db.offsets, idx)
    for k, i in enumerate(idx):
        assert np.array_equal(res[off[k]:off[k + 1]], seqs[i])
    res0, off0 = subset(db.residues, db.offsets, np.array([], dtype=np.int64))
    assert res0.size == 0 and off0.tolist() == [0]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = make_workload("one_query_vs_2k", n_db=120)
    db, q = w["db"], w["queries"]
    parts = partition(db.lengths, world)
    res, off = subset(db.residues, db.offsets, parts[rank])
    local = oracle.scores(q, from_list([res[off[k]:off[k + 1]] for k in range(off.size - 1)]), BLOSUM62, 10, 2)
    full = gather_scores(local, parts, dist)
    np.save(os.path.join(outdir, f"full{rank}.npy"), full)
    dist.destroy_process_group()


def test_two_ranks_gather_the_full_score_matrix(tmp_path):
    oracle.build()
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    w = make_workload("one_query_vs_2k", n_db=120)
    exp = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2)
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"full{r}.npy"), exp)
