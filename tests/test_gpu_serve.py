"""Serving path: continuous batching over a resident database.

Requests arrive while earlier batches are still on the GPU; each result must
equal the same query searched alone (and the CPU oracle)."""

import threading
import time

import numpy as np
import pytest

import oracle
from workload import make_workload, random_sequences, sample_indices
from workload.matrices import BLOSUM62

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_08308_gb300 import api as _api
    from paper_2412_08308_gb300 import build

    build()
    oracle.build()
    return _api


@pytest.mark.parametrize("mode,prestage", [("packed", True), ("int32", True), ("packed", False)])
def test_results_same_alone_and_in_the_mix(api, mode, prestage):
    # prestage: the next batch is planned while every slot is busy
    from paper_2412_08308_gb300.serve import Server

    db_s = random_sequences(71, 3000, 300, 0.5, 20, 1000)
    qs = random_sequences(72, 40, 300, 0.5, 30, 1500)
    db = api.Database.from_sequences(db_s)
    alone = [api.search(db, qs[i], np.array([0, len(qs[i])]), BLOSUM62, 10, 2, mode)[0] for i in range(len(qs))]
    srv = Server(db, BLOSUM62, 10, 2, mode, max_batch=6, n_streams=3, prestage=prestage)
    futs = []
    # bursts from two client threads, so batches overlap on the device
    def client(lo, hi):
        for i in range(lo, hi):
            futs.append((i, srv.submit(qs[i])))
            if i % 7 == 0:
                time.sleep(0.002)
    t1 = threading.Thread(target=client, args=(0, 20))
    t2 = threading.Thread(target=client, args=(20, 40))
    t1.start(); t2.start(); t1.join(); t2.join()
    got = {i: f.result(timeout=120) for i, f in futs}
    srv.close()
    exp = oracle.scores(qs, db_s, BLOSUM62, 10, 2)
    for i in range(len(qs)):
        np.testing.assert_array_equal(got[i], alone[i])
        np.testing.assert_array_equal(got[i], exp[i])
    st = srv.latency_stats()
    assert st["requests"] == len(qs) and st["p99_ms"] >= st["p50_ms"] > 0
    assert 0 < st["plan_ms_p50"] < st["p50_ms"] and 0 < st["plan_share_of_p50"] < 1
    db.close()


def test_sharded_database_shards_on_one_gpu(api):
    # every rank's shard of a 3-way split, searched on this GPU one after the
    # other and put back in caller order, equals the whole search
    from paper_2412_08308_gb300.shard import ShardedDatabase

    db_s = random_sequences(75, 900, 300, 0.5, 20, 1000)
    qs = random_sequences(76, 4, 300, 0.5, 30, 800)
    full = np.zeros((len(qs), len(db_s)), dtype=np.int32)
    for rank in range(3):
        sh = ShardedDatabase(db_s.residues, db_s.offsets, rank, 3)
        full[:, sh.mine] = api.search(sh.db, qs.residues, qs.offsets, BLOSUM62, 10, 2, "packed")
        sh.close()
    np.testing.assert_array_equal(full, oracle.scores(qs, db_s, BLOSUM62, 10, 2))
    one = ShardedDatabase(db_s.residues, db_s.offsets, 0, 1)
    np.testing.assert_array_equal(one.search(qs.residues, qs.offsets, BLOSUM62, 10, 2), full)
    one.close()


def test_serving_500k_in_the_mix_matches_oracle(api):
    # the serving workload's database at full size (500,000 proteins, ~180M
    # residues) resident in HBM; 16 of its queries (30..3,000 residues, the
    # longest included) submitted by two client threads at its arrival
    # times, so that batches overlap on the device; every result on a seeded
    # 300-sequence sample equals the oracle's
    from paper_2412_08308_gb300.serve import Server

    w = make_workload("serving_500k")
    ql = w["queries"].lengths
    qi = set(sample_indices(len(ql), 14, seed=4103).tolist()) | {int(np.argmin(ql)), int(np.argmax(ql))}
    qi = sorted(qi)
    q = w["queries"].subset(qi)
    di = sample_indices(len(w["db"]), 300, seed=4104)
    exp = oracle.scores(q, w["db"], BLOSUM62, 10, 2, subset=di)
    db = api.Database.from_sequences(w["db"])
    srv = Server(db, BLOSUM62, 10, 2, "packed", max_batch=2, n_streams=2)
    arrivals = np.cumsum(np.full(len(qi), 0.02))
    t0 = time.perf_counter()
    futs = []

    def client(lo, step):
        for i in range(lo, len(qi), step):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            futs.append((i, srv.submit(q[i])))

    t1 = threading.Thread(target=client, args=(0, 2))
    t2 = threading.Thread(target=client, args=(1, 2))
    t1.start(); t2.start(); t1.join(); t2.join()
    got = {i: f.result(timeout=300) for i, f in futs}
    srv.close()
    assert len(got) == len(qi)
    for i in range(len(qi)):
        np.testing.assert_array_equal(got[i][di], exp[i], err_msg=f"query {qi[i]} of {ql[qi[i]]} residues")
    db.close()
