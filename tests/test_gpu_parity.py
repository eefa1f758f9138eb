"""GPU parity: every kernel form against the CPU oracle, bit-exact.

The GPU path is reached only through the C-ABI (paper_2412_08308_gb300.api ->
ctypes -> libswgb.so).  Scores are int32; the bar is exact equality.
"""

import numpy as np
import pytest

import oracle
from workload import from_list, make_config, random_sequences, sample_indices
from workload.matrices import BLOSUM62

pytestmark = pytest.mark.gpu

MODES = ["int32", "packed"]


@pytest.fixture(scope="module")
def api():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_08308_gb300 import api as _api
    from paper_2412_08308_gb300 import build

    build()
    oracle.build()
    return _api


def _search(api, db_seqs, q_seqs, mode, sm=BLOSUM62, go=10, ge=2):
    db = api.Database.from_sequences(db_seqs)
    try:
        return api.search(db, q_seqs.residues, q_seqs.offsets, sm, go, ge, mode)
    finally:
        db.close()


def _assert_equal(got, exp):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        i, j = bad[0]
        raise AssertionError(f"{len(bad)} mismatches; first at query {i}, sequence {j}: got {got[i, j]}, "
                             f"expected {exp[i, j]}")


@pytest.mark.parametrize("mode", MODES)
def test_config1_full(api, mode):
    # 1 query of 144 residues against 2,000 synthetic proteins
    w = make_config(1)
    got = _search(api, w["db"], w["queries"], mode)
    _assert_equal(got, oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2))


def _ragged(seed, n_db, n_q, qmax):
    rng = np.random.Generator(np.random.PCG64(seed))
    edge = [0, 1, 2, 15, 16, 17, 31, 32, 33, 47, 48, 49, 127, 128, 129]
    dl = list(edge) + list(rng.integers(1, 400, size=n_db - len(edge)))
    rng.shuffle(dl)
    db = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in dl])
    ql = [0, 1, 3] + list(rng.integers(4, qmax, size=n_q - 3))
    q = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in ql])
    return db, q


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("R,L", [(16, 0), (8, 4), (12, 5), (24, 13), (16, 32), (8, 31)])
def test_ragged_tiles(api, monkeypatch, mode, R, L):
    # database lengths straddling every padding boundary, empty and 1-residue
    # sequences, queries from 0 residues to several chunks of L*R rows
    monkeypatch.setenv("SWGB_R", str(R))
    monkeypatch.setenv("SWGB_L", str(L))
    db, q = _ragged(10 + R + L, 301, 9, 900)
    got = _search(api, db, q, mode)
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("go,ge", [(0, 1), (3, 1), (25, 1), (1, 12), (0, 0)])
def test_gap_parameters(api, mode, go, ge):
    db, q = _ragged(77, 120, 5, 300)
    got = _search(api, db, q, mode, go=go, ge=ge)
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, go, ge))


@pytest.mark.parametrize("mode", MODES)
def test_extreme_asymmetric_matrix(api, mode):
    rng = np.random.Generator(np.random.PCG64(5))
    sm = rng.integers(-64, 64, size=(20, 20)).astype(np.int8)
    sm[0, 0], sm[1, 2] = 63, -64
    db, q = _ragged(78, 150, 6, 400)
    got = _search(api, db, q, mode, sm=sm, go=7, ge=3)
    _assert_equal(got, oracle.scores(q, db, sm, 7, 3))


def test_packed_overflow_is_rescued_exactly(api):
    # identity-like matrix with +60 matches: a 700-residue self match scores
    # 42000 > 32767, so the 16-bit lanes saturate and the int32 rescue must
    # reproduce the exact score; unrelated pairs stay in the packed path.
    rng = np.random.Generator(np.random.PCG64(9))
    sm = np.full((20, 20), -5, dtype=np.int8)
    np.fill_diagonal(sm, 60)
    base = rng.integers(0, 20, size=700).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(50, 500))).astype(np.uint8) for _ in range(200)]
    for pos in (3, 4, 100, 199):
        seqs[pos] = base.copy() if pos != 100 else base[:600].copy()
    db = from_list(seqs)
    q = from_list([base, base[:100], rng.integers(0, 20, size=300).astype(np.uint8)])
    exp = oracle.scores(q, db, sm, 10, 2)
    assert exp.max() > 32767
    pq = api.PreparedQueries(api.Database.from_sequences(db), q.residues, q.offsets, sm, 10, 2, "packed")
    got = pq.search().cpu().numpy()
    rescued = pq.status()
    _assert_equal(got, exp)
    assert rescued >= 4
    pq.close()


@pytest.mark.parametrize("mode", MODES)
def test_config3_precision_path(api, mode):
    # config 1's database plus 10 planted ~8,000-residue homologs of an
    # 8,000-residue query; their int16 scores overflow and are rescued
    w = make_config(3)
    exp = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2)
    assert exp[1, w["homolog_ids"]].min() > 32767
    db = api.Database.from_sequences(w["db"])
    pq = api.PreparedQueries(db, w["queries"].residues, w["queries"].offsets, BLOSUM62, 10, 2, mode)
    got = pq.search().cpu().numpy()
    rescued = pq.status()
    _assert_equal(got, exp)
    if mode == "packed":
        assert rescued >= len(w["homolog_ids"])
    pq.close()
    db.close()


@pytest.mark.parametrize("mode", MODES)
def test_config2_sampled(api, mode):
    # 20 queries (144..5478) against 200,000 sequences; every score of a
    # seeded 300-sequence sample is compared with the oracle
    w = make_config(2)
    got = _search(api, w["db"], w["queries"], mode)
    idx = sample_indices(len(w["db"]), 300)
    exp = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2, subset=idx)
    _assert_equal(got[:, idx], exp)
    assert got.min() >= 0


def test_config4_sampled(api):
    # 1,000 queries against 50,000 sequences (packed); a sample of 12 queries
    # x 150 sequences is checked
    w = make_config(4)
    got = _search(api, w["db"], w["queries"], "packed")
    qi = sample_indices(len(w["queries"]), 12, seed=4101)
    di = sample_indices(len(w["db"]), 150, seed=4102)
    exp = oracle.scores(w["queries"].subset(qi), w["db"], BLOSUM62, 10, 2, subset=di)
    _assert_equal(got[np.ix_(qi, di)], exp)


def test_prepared_repeat_and_device_output(api):
    import torch

    db_s = random_sequences(31, 999, 250, 0.5, 1, 700)
    q_s = random_sequences(32, 7, 200, 0.6, 1, 900)
    db = api.Database.from_sequences(db_s)
    pq = api.PreparedQueries(db, q_s.residues, q_s.offsets, BLOSUM62, 10, 2, "packed")
    a = pq.search().cpu().numpy()
    b = pq.search().cpu().numpy()
    dev = torch.empty((len(q_s), len(db_s)), dtype=torch.int32, device="cuda")
    api.search(db, q_s.residues, q_s.offsets, BLOSUM62, 10, 2, "int32", out=dev)
    c = dev.cpu().numpy()
    exp = oracle.scores(q_s, db_s, BLOSUM62, 10, 2)
    _assert_equal(a, exp)
    _assert_equal(b, exp)
    _assert_equal(c, exp)
    pq.close()
    db.close()


def test_empty_inputs(api):
    empty_q = from_list([])
    db_s = random_sequences(33, 10, 50, 0.5, 1, 100)
    db = api.Database.from_sequences(db_s)
    out = api.search(db, empty_q.residues, empty_q.offsets, BLOSUM62, 10, 2, "packed")
    assert out.shape == (0, 10)
    db.close()
    edb = api.Database.from_sequences(from_list([]))
    q = random_sequences(34, 3, 50, 0.5, 1, 100)
    out = api.search(edb, q.residues, q.offsets, BLOSUM62, 10, 2, "packed")
    assert out.shape == (3, 0)
    edb.close()


def test_invalid_arguments_rejected(api):
    from paper_2412_08308_gb300._native import SW_EINVAL, SwError

    db_s = random_sequences(35, 10, 50, 0.5, 1, 100)
    db = api.Database.from_sequences(db_s)
    q = random_sequences(36, 2, 50, 0.5, 1, 100)
    with pytest.raises(SwError) as e:
        api.search(db, q.residues, q.offsets, BLOSUM62, -1, 2, "packed")
    assert e.value.code == SW_EINVAL
    bad = q.residues.copy()
    bad[0] = 20
    with pytest.raises(SwError):
        api.search(db, bad, q.offsets, BLOSUM62, 10, 2, "packed")
    sm = BLOSUM62.copy()
    sm[0, 0] = 100
    with pytest.raises(SwError):
        api.search(db, q.residues, q.offsets, sm, 10, 2, "packed")
    db.close()
