"""GPU parity: every kernel form against the CPU oracle, bit-exact.

The GPU path is reached only through the C-ABI (paper_2412_08308_gb300.api ->
ctypes -> libswgb.so).  Scores are int32; the bar is exact equality.
"""

import numpy as np
import pytest

import oracle
from workload import from_list, make_workload, random_sequences, sample_indices
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


def _search(api, db_seqs, q_seqs, mode, sm=BLOSUM62, go=10, ge=2, opts=None):
    db = api.Database.from_sequences(db_seqs)
    try:
        if opts is None:
            return api.search(db, q_seqs.residues, q_seqs.offsets, sm, go, ge, mode)
        pq = api.PreparedQueries(db, q_seqs.residues, q_seqs.offsets, sm, go, ge, mode, opts=opts)
        out = pq.search().cpu().numpy()
        pq.status()
        pq.close()
        return out
    finally:
        db.close()


def _assert_equal(got, exp):
    if not np.array_equal(got, exp):
        bad = np.argwhere(got != exp)
        i, j = bad[0]
        raise AssertionError(f"{len(bad)} mismatches; first at query {i}, sequence {j}: got {got[i, j]}, "
                             f"expected {exp[i, j]}")


@pytest.mark.parametrize("mode", MODES)
def test_one_query_vs_2k_full(api, mode):
    # 1 query of 144 residues against 2,000 synthetic proteins
    w = make_workload("one_query_vs_2k")
    got = _search(api, w["db"], w["queries"], mode)
    _assert_equal(got, oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2))


@pytest.mark.parametrize("mode", MODES)
def test_one_query_batch_of_256(api, mode):
    # 256 requests shaped like the single query (144 residues) searched
    # together against the same 2,000 proteins: every query against a
    # seeded sample of 300 of them
    from workload import query_batch_144

    w = make_workload("one_query_vs_2k")
    q = query_batch_144(256)
    idx = sample_indices(len(w["db"]), 300)
    got = _search(api, w["db"], q, mode)
    _assert_equal(got[:, idx], oracle.scores(q, w["db"].subset(idx), BLOSUM62, 10, 2))


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
@pytest.mark.parametrize("R,L", [(16, 0), (8, 4), (12, 5), (24, 13), (16, 32), (8, 31), (4, 9), (4, 0)])
def test_ragged_tiles(api, mode, R, L):
    # database lengths straddling every padding boundary, empty and 1-residue
    # sequences, queries from 0 residues to several chunks of L*R rows
    db, q = _ragged(10 + R + L, 301, 9, 900)
    got = _search(api, db, q, mode, opts=api.options(rows_per_lane=R, lanes_per_chain=L, band_stream="never"))
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


@pytest.mark.parametrize("scale,go,ge", [(2, 20, 4), (3, 8, 1)])
def test_wider_matrices_and_gap_schemes(api, scale, go, ge):
    # other substitution matrices and gap schemes than BLOSUM62 10/2: a matrix
    # scale x BLOSUM62 has entries up to 11 * scale, so the 16-bit threshold
    # (32767 - max SM) and the overflow bound max(SM) * min(m, n) move with it.
    # A 3,000-residue query and database copies of 1,200 and 2,400 of its
    # residues: at scale 3 the 2,400-residue copy scores ~40,000 and is
    # rescued (cutover 4096: inter-task) or computed in int32 (cutover 1000:
    # intra-task).  Every form and plan, exact against the oracle.
    rng = np.random.Generator(np.random.PCG64(60 + scale))
    sm = (BLOSUM62.astype(np.int32) * scale).astype(np.int8)
    base = rng.integers(0, 20, size=3000).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(10, 700))).astype(np.uint8) for _ in range(240)]
    seqs[3] = base[:1200].copy()
    seqs[100] = base[500:2900].copy()
    db = from_list(seqs)
    q = from_list([base, base[:400].copy(), rng.integers(0, 20, size=390).astype(np.uint8),
                   rng.integers(0, 20, size=150).astype(np.uint8)])
    exp = oracle.scores(q, db, sm, go, ge)
    if scale == 3:
        assert exp.max() > 32767
    for mode in MODES:
        for cutover in (1000, 4096):
            for band in ("never", "always"):
                got = _search(api, db, q, mode, sm=sm, go=go, ge=ge, opts=api.options(cutover=cutover, band_stream=band))
                _assert_equal(got, exp)


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
    pq = api.PreparedQueries(api.Database.from_sequences(db), q.residues, q.offsets, sm, 10, 2, "packed",
                             opts=api.options(band_stream="never"))
    got = pq.search().cpu().numpy()
    rescued = pq.status()
    _assert_equal(got, exp)
    assert rescued >= 4
    pq.close()
    # the same batch with the 700-residue query on band-stream jobs: its
    # saturating pairs run in int32 there, exact without a rescue
    _assert_equal(_search(api, db, q, "packed", sm=sm, opts=api.options(band_stream="always")), exp)


def _prepared(api, db_seqs, q_seqs, mode, sm=BLOSUM62, go=10, ge=2, opts=None):
    db = api.Database.from_sequences(db_seqs)
    pq = api.PreparedQueries(db, q_seqs.residues, q_seqs.offsets, sm, go, ge, mode, opts=opts)
    try:
        out = pq.search().cpu().numpy()
        pq.status()
        return out, pq.info()
    finally:
        pq.close()
        db.close()


@pytest.mark.parametrize("cutover", [0, 300])
def test_query_pairs(api, cutover):
    # packed mode runs queries in pairs, one per 16-bit half of a chain (one
    # database sequence per chain): each half runs a track of queries laid end
    # to end chunk by chunk.  Lengths from 0 to 700 residues; with this small
    # database the planner spreads the queries over several track plans.
    # cutover=300 also sends the longest units to the intra-task kernel.
    rng = np.random.Generator(np.random.PCG64(31))
    db, _ = _ragged(33, 401, 3, 10)
    ql = [300, 290, 281, 250, 700, 100, 96, 55, 0, 0, 17, 16]
    q = from_list([rng.integers(0, 20, size=L).astype(np.uint8) for L in ql])
    exp = oracle.scores(q, db, BLOSUM62, 10, 2)
    on, _ = _prepared(api, db, q, "packed", opts=api.options(cutover=cutover, band_stream="never"))
    off, _ = _prepared(api, db, q, "packed", opts=api.options(cutover=cutover, query_pairs=False, band_stream="never"))
    _assert_equal(on, exp)
    _assert_equal(off, exp)


def test_query_pairs_only_where_no_lane_can_overflow(api):
    # +60 matches: 3,000-residue queries can pass 32767 against the 1,500-
    # residue database units, so they stay in the rescued two-sequence form;
    # the 40-residue pair cannot and is paired.  Scores stay exact.
    rng = np.random.Generator(np.random.PCG64(12))
    sm = np.full((20, 20), -5, dtype=np.int8)
    np.fill_diagonal(sm, 60)
    base = rng.integers(0, 20, size=3000).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(20, 300))).astype(np.uint8) for _ in range(150)]
    seqs[7] = base[:1500].copy()
    seqs[8] = base[1000:2500].copy()
    db = from_list(seqs)
    q = from_list([base, base[::-1].copy(), base[:40].copy(), rng.integers(0, 20, size=38).astype(np.uint8)])
    exp = oracle.scores(q, db, sm, 10, 2)
    assert exp.max() > 32767
    got, info = _prepared(api, db, q, "packed", sm=sm, opts=api.options(cutover=4096, band_stream="never"))
    _assert_equal(got, exp)
    # the track plan adds its profile build and its inter-task launch
    _, info_off = _prepared(api, db, q, "packed", sm=sm,
                            opts=api.options(cutover=4096, query_pairs=False, band_stream="never"))
    assert info[3] == info_off[3] + 2


@pytest.mark.parametrize("R,L", [(4, 0), (8, 0), (24, 0), (4, 4), (12, 7), (16, 0), (16, 32), (24, 32), (8, 5)])
def test_query_pairs_tiles(api, R, L):
    # tracks at several rows-per-lane instances; with 4 x 4 rows per chunk a
    # track switches queries many times (restarting its half from the matrix
    # top boundary) and queries span up to 57 chunks.  R = 8, 16, 24 run split
    # lanes (two half-chains a column apart; 32 lanes: a 63-column chain lag),
    # R = 4 and 12 one chain per lane
    db, _ = _ragged(40 + R + L, 257, 3, 10)
    rng = np.random.Generator(np.random.PCG64(R + L))
    q = from_list([rng.integers(0, 20, size=n).astype(np.uint8) for n in (900, 880, 333, 300, 5, 4, 17, 16, 1)])
    got = _search(api, db, q, "packed", opts=api.options(rows_per_lane=R, lanes_per_chain=L, band_stream="never"))
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


@pytest.fixture(scope="module")
def homologs():
    w = make_workload("homologs_8k")
    w["expected"] = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2)
    assert w["expected"][1, w["homolog_ids"]].min() > 32767
    return w


@pytest.mark.parametrize("mode,cutover,band", [("int32", 0, "never"), ("packed", 0, "never"),
                                               ("packed", 16384, "never"), ("int32", 0, "auto"),
                                               ("packed", 0, "auto"), ("packed", 16384, "auto")])
def test_homologs_precision_path(api, homologs, mode, cutover, band):
    # the 2,000-protein database plus 10 planted ~8,000-residue homologs of an
    # 8,000-residue query, whose scores exceed the 16-bit range.  Without
    # band-stream jobs: with the default cutover the homologs run in the
    # intra-task kernel, which takes them straight to int32 (their bound
    # max(SM)*min(m, n) passes the 16-bit threshold); with cutover 16384 they
    # run packed in the inter-task kernel, saturate, are flagged and rescued
    # exactly.  With them (the default for this small batch): the
    # 8,000-residue query runs in 16 bands of 512 rows against every unit
    # (the homologs in int32, in 32 bands of 256 rows; the others two per
    # word), the 144-residue query transposed against row tracks of every
    # sequence.
    w = homologs
    db = api.Database.from_sequences(w["db"])
    pq = api.PreparedQueries(db, w["queries"].residues, w["queries"].offsets, BLOSUM62, 10, 2, mode,
                             opts=api.options(cutover=cutover, band_stream=band))
    got = pq.search().cpu().numpy()
    rescued = pq.status()
    _assert_equal(got, w["expected"])
    if mode == "packed" and cutover == 16384 and band == "never":
        assert rescued >= len(w["homolog_ids"])
    pq.close()
    db.close()


@pytest.mark.parametrize("mode", MODES)
def test_twenty_queries_vs_200k_sampled(api, mode):
    # 20 queries (144..5478) against 200,000 sequences; every score of a
    # seeded 300-sequence sample is compared with the oracle
    w = make_workload("twenty_queries_vs_200k")
    got = _search(api, w["db"], w["queries"], mode)
    idx = sample_indices(len(w["db"]), 300)
    exp = oracle.scores(w["queries"], w["db"], BLOSUM62, 10, 2, subset=idx)
    _assert_equal(got[:, idx], exp)
    assert got.min() >= 0


@pytest.fixture(scope="module")
def thousand():
    w = make_workload("thousand_queries_vs_50k")
    qi = sample_indices(len(w["queries"]), 12, seed=4101)
    di = sample_indices(len(w["db"]), 150, seed=4102)
    w["sample"] = (qi, di, oracle.scores(w["queries"].subset(qi), w["db"], BLOSUM62, 10, 2, subset=di))
    return w


@pytest.mark.parametrize("mode", MODES)
def test_thousand_queries_vs_50k_sampled(api, thousand, mode):
    # 1,000 queries against 50,000 sequences in one batch, both forms; a
    # sample of 12 queries x 150 sequences is checked against the oracle
    w = thousand
    got = _search(api, w["db"], w["queries"], mode)
    qi, di, exp = w["sample"]
    _assert_equal(got[np.ix_(qi, di)], exp)
    assert got.min() >= 0


def serving_sample(w, k=16):
    """About k seeded queries of the serving workload, its shortest and its
    longest among them, and a seeded 300-sequence sample of its database."""
    ql = w["queries"].lengths
    qi = set(sample_indices(len(ql), k - 2, seed=4103).tolist()) | {int(np.argmin(ql)), int(np.argmax(ql))}
    qi = np.array(sorted(qi), dtype=np.int64)
    di = sample_indices(len(w["db"]), 300, seed=4104)
    return qi, di


@pytest.fixture(scope="module")
def serving_500k():
    w = make_workload("serving_500k")
    qi, di = serving_sample(w)
    q = w["queries"].subset(qi)
    assert q.lengths.max() == w["queries"].lengths.max() and q.lengths.min() == w["queries"].lengths.min()
    return w, q, di, oracle.scores(q, w["db"], BLOSUM62, 10, 2, subset=di)


@pytest.mark.parametrize("mode", MODES)
def test_serving_500k_sampled(api, serving_500k, mode):
    # the serving database at its full size (500,000 proteins, ~180M
    # residues, resident) against 16 of its queries (30..3,000 residues,
    # the longest included) in one batch; every score of a seeded
    # 300-sequence sample is compared with the oracle
    w, q, di, exp = serving_500k
    got = _search(api, w["db"], q, mode)
    _assert_equal(got[:, di], exp)
    assert got.min() >= 0


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


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("intra_rows", [8, 16])
def test_intra_task_kernel(api, mode, intra_rows):
    # database sequences from 1 to ~5,000 residues with the cutover at 1,000:
    # the long ones go to the multi-warp intra-task kernel, concurrently with
    # the inter-task kernel; queries up to 9,000 residues span several chunks
    # of 32 * 16 * intra_rows rows
    rng = np.random.Generator(np.random.PCG64(40 + intra_rows))
    lens = [1, 15, 16, 17, 999, 1000, 1001, 1007, 2048, 4999] + list(rng.integers(1, 5000, size=40))
    db = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in lens])
    ql = [0, 1, 33, 511, 512, 513, 3000, 4097, 9000]
    q = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in ql])
    got = _search(api, db, q, mode, opts=api.options(cutover=1000, intra_rows=intra_rows, band_stream="never"))
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


@pytest.mark.parametrize("mode", MODES)
def test_everything_intra(api, mode):
    # cutover 1: every unit goes through the intra-task kernel
    db, q = _ragged(91, 60, 5, 700)
    got = _search(api, db, q, mode, opts=api.options(cutover=1, band_stream="never"))
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


def test_intra_saturating_units_exact(api):
    # long self-matches above the 16-bit range on intra-task units (routed to
    # int32) next to short ones that saturate in the packed inter-task kernel
    rng = np.random.Generator(np.random.PCG64(17))
    sm = np.full((20, 20), -5, dtype=np.int8)
    np.fill_diagonal(sm, 40)
    base = rng.integers(0, 20, size=3000).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(100, 3000))).astype(np.uint8) for _ in range(30)]
    seqs[5], seqs[6], seqs[20] = base.copy(), base[:2500].copy(), base[500:].copy()
    seqs[21], seqs[22] = base[:900].copy(), base[1000:1950].copy()
    db = from_list(seqs)
    q = from_list([base, base[:1000]])
    exp = oracle.scores(q, db, sm, 10, 2)
    assert exp.max() > 32767
    dbh = api.Database.from_sequences(db)
    pq = api.PreparedQueries(dbh, q.residues, q.offsets, sm, 10, 2, "packed",
                             opts=api.options(cutover=1000, band_stream="never"))
    got = pq.search().cpu().numpy()
    rescued = pq.status()
    _assert_equal(got, exp)
    assert rescued >= 2  # the two short self-matches (900 and 950 residues x 40 > 32767)
    pq.close()
    dbh.close()


def test_bad_options_rejected(api):
    from paper_2412_08308_gb300._native import SW_EINVAL, SwError

    db_s = random_sequences(37, 10, 50, 0.5, 1, 100)
    q = random_sequences(38, 2, 50, 0.5, 1, 100)
    db = api.Database.from_sequences(db_s)
    bad_band = api.options()
    bad_band.band_stream = 3
    for opts in (api.options(rows_per_lane=7), api.options(lanes_per_chain=3), api.options(intra_rows=12), bad_band,
                 api.options(band_rows=12)):
        with pytest.raises(SwError) as e:
            api.PreparedQueries(db, q.residues, q.offsets, BLOSUM62, 10, 2, "packed", opts=opts)
        assert e.value.code == SW_EINVAL
    db.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("band", ["never", "always"])
def test_graph_replay_matches(api, mode, band):
    # the whole search captured in a CUDA graph (long units included, so the
    # side-stream fork/join is captured too) and replayed twice, then again
    # into a different output buffer (re-capture); with the inter- and
    # intra-task kernels, and with the small-batch plan (band-stream jobs on
    # the side stream for the 1,100-residue query, transposed jobs beside)
    import torch

    rng = np.random.Generator(np.random.PCG64(61))
    lens = list(rng.integers(1, 600, size=120)) + [2500, 3100]
    db_s = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in lens])
    q_s = from_list(random_sequences(62, 5, 300, 0.5, 1, 1500).as_list() +
                    [rng.integers(0, 20, size=1100).astype(np.uint8)])
    exp = oracle.scores(q_s, db_s, BLOSUM62, 10, 2)
    db = api.Database.from_sequences(db_s)
    pq = api.PreparedQueries(db, q_s.residues, q_s.offsets, BLOSUM62, 10, 2, mode,
                             opts=api.options(cutover=2048, band_stream=band))
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        out = torch.full((len(q_s), len(db_s)), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            pq.search_graph(out, stream=st)
            st.synchronize()
            _assert_equal(out.cpu().numpy(), exp)
            out.fill_(-1)
        out2 = torch.full_like(out, -1)
        pq.search_graph(out2, stream=st)
        st.synchronize()
        _assert_equal(out2.cpu().numpy(), exp)
    assert pq.status(stream=st) >= 0
    pq.close()
    db.close()


def test_autotuner_picks_a_correct_plan(api, tmp_path):
    from paper_2412_08308_gb300 import tune

    db_s = random_sequences(81, 4000, 300, 0.5, 20, 1000)
    q_s = random_sequences(82, 12, 350, 0.5, 50, 2000)
    db = api.Database.from_sequences(db_s)
    cache = str(tmp_path / "tune.json")
    opts, table = tune.tune(db, db_s.lengths, q_s.residues, q_s.offsets, BLOSUM62, rows=(4, 16), cutovers=(512, 2048),
                            reps=1, cache_path=cache)
    assert len(table) == 4 and all(g > 0 for _, _, g in table)
    assert (opts.rows_per_lane, opts.cutover) in [(r, c) for r, c, _ in table]
    again, table2 = tune.tune(db, db_s.lengths, q_s.residues, q_s.offsets, BLOSUM62, rows=(4, 16),
                              cutovers=(512, 2048), reps=1, cache_path=cache)
    assert (again.rows_per_lane, again.cutover) == (opts.rows_per_lane, opts.cutover)  # from the cache
    got = _search(api, db_s, q_s, "packed", opts=opts)
    _assert_equal(got, oracle.scores(q_s, db_s, BLOSUM62, 10, 2))
    db.close()


def _band_db(seed, n, long_lens):
    rng = np.random.Generator(np.random.PCG64(seed))
    edge = [0, 1, 2, 15, 16, 17, 47, 48, 49, 127, 128, 129]
    lens = edge + list(long_lens) + list(rng.integers(1, 700, size=n - len(edge) - len(long_lens)))
    rng.shuffle(lens)
    return from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in lens])


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("band,rows", [("auto", 0), ("always", 8), ("always", 16)])
def test_band_stream_ragged(api, mode, band, rows):
    # band-stream jobs (k_band.cu): queries across the band edges (8 rows a
    # lane: 256-row bands, 511/512/513, 768/769 rows; 16 rows a lane: 512-row
    # bands, 1023/1024/1025) and up to 12 bands, against a database with every
    # padding edge and sequences at and past the cutover of 2,048 residues
    # (the queries below two bands meet those long units in one band each;
    # the others every unit in their own band pipelines)
    db = _band_db(511, 260, [2047, 2048, 2049, 3001, 5000])
    rng = np.random.Generator(np.random.PCG64(512))
    ql = [0, 1, 144, 255, 256, 257, 511, 512, 513, 768, 769, 1023, 1024, 1025, 1500, 3000]
    q = from_list([rng.integers(0, 20, size=L).astype(np.uint8) for L in ql])
    got = _search(api, db, q, mode, opts=api.options(band_stream=band, band_rows=rows))
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("rows", [8, 16])
def test_band_stream_saturating_and_asymmetric(api, mode, rows):
    # an asymmetric matrix with +60 matches: the band pipelines' pairs that
    # can pass 32767 (a 3,000-residue query against copies of 700 to 2,400 of
    # its residues) run in int32 -- the units wider than a job's share of
    # columns in bands of half the height --, the others two sequences per
    # word; all exact
    rng = np.random.Generator(np.random.PCG64(513))
    sm = rng.integers(-20, 6, size=(20, 20)).astype(np.int8)
    np.fill_diagonal(sm, 60)
    base = rng.integers(0, 20, size=3000).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(10, 900))).astype(np.uint8) for _ in range(180)]
    seqs[4], seqs[50], seqs[51], seqs[120] = base[:700].copy(), base[200:2600].copy(), base[:1500].copy(), base[::2]
    db = from_list(seqs)
    q = from_list([base, base[:600].copy(), base[2000:].copy(), rng.integers(0, 20, size=90).astype(np.uint8)])
    exp = oracle.scores(q, db, sm, 9, 3)
    assert exp.max() > 32767
    got = _search(api, db, q, mode, sm=sm, go=9, ge=3,
                  opts=api.options(band_stream="always", cutover=1000, band_rows=rows))
    _assert_equal(got, exp)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("with_band_query", [False, True])
def test_transposed_jobs_int32_tracks_and_long_rows(api, mode, with_band_query):
    # transposed jobs (short queries: the database sequences are the rows):
    # with 512-row bands the queries below 1,024 residues run transposed; a
    # +60 identity-like matrix lets a 700-residue query pass the 16-bit range
    # against its copies, so in packed mode the sequences that could
    # saturate against it go to int32 row tracks, the others two per word.
    # Copies of 5,000 residues span ten bands of one track (a pipeline); the
    # empty and one-residue sequences score 0 and the SM of query residue x
    # database residue is asymmetric.  with_band_query: a 1,100-residue query
    # runs as band-stream jobs beside them, and the transposed jobs take
    # 8-row lanes (256-row bands)
    rng = np.random.Generator(np.random.PCG64(514))
    sm = rng.integers(-9, 4, size=(20, 20)).astype(np.int8)
    np.fill_diagonal(sm, 60)
    base = rng.integers(0, 20, size=5000).astype(np.uint8)
    seqs = [rng.integers(0, 20, size=int(rng.integers(1, 400))).astype(np.uint8) for _ in range(200)]
    seqs[3], seqs[40], seqs[41], seqs[90] = base.copy(), base[:700].copy(), base[100:900].copy(), base[4000:]
    seqs[5], seqs[6] = np.zeros(0, np.uint8), base[:1].copy()
    db = from_list(seqs)
    ql = [base[:700].copy(), base[50:200].copy(), rng.integers(0, 20, size=33).astype(np.uint8), np.zeros(0, np.uint8)]
    if with_band_query:
        ql.append(base[1000:2100].copy())
    q = from_list(ql)
    exp = oracle.scores(q, db, sm, 10, 2)
    assert exp.max() > 32767
    got = _search(api, db, q, mode, sm=sm, opts=api.options(band_stream="always", band_rows=16))
    _assert_equal(got, exp)


@pytest.mark.parametrize("seed", range(8))
def test_small_batch_plans_random(api, seed):
    # random small batches through the small-batch plan (band-stream and
    # transposed jobs, forced): database and query lengths from 0 to a few
    # thousand (some databases with copies of a query, so that pairs pass the
    # 16-bit range), random asymmetric matrices with a strong diagonal,
    # random gap costs and both band heights; both forms, exact
    rng = np.random.Generator(np.random.PCG64(9000 + seed))
    sm = rng.integers(-8, 5, size=(20, 20)).astype(np.int8)
    np.fill_diagonal(sm, rng.integers(4, 61, size=20))
    go, ge = int(rng.integers(0, 16)), int(rng.integers(0, 5))
    nq = int(rng.integers(1, 6))
    qs = [rng.integers(0, 20, size=int(L)).astype(np.uint8)
          for L in rng.choice([0, 1, 40, 144, 300, 700, 1100, 1700, 2600], size=nq)]
    nd = int(rng.integers(1, 260))
    seqs = [rng.integers(0, 20, size=int(min(3000, rng.lognormal(np.log(250), 0.9)))).astype(np.uint8)
            for _ in range(nd)]
    long_q = max(qs, key=len)
    for k in range(min(3, nd)):  # copies of parts of the longest query
        a = int(rng.integers(0, max(1, len(long_q))))
        seqs[int(rng.integers(0, nd))] = long_q[a:a + int(rng.integers(1, 2500))].copy()
    db, q = from_list(seqs), from_list(qs)
    exp = oracle.scores(q, db, sm, go, ge)
    rows = int(rng.choice([8, 16]))
    for mode in MODES:
        got = _search(api, db, q, mode, sm=sm, go=go, ge=ge, opts=api.options(band_stream="always", band_rows=rows))
        _assert_equal(got, exp)


@pytest.mark.parametrize("mode", MODES)
def test_transposed_24_row_lanes_edges(api, mode):
    # one short query against ~2,000 proteins, the shape for which the
    # packed plan takes 24-row lanes (768-row bands, one per SM
    # sub-partition), with sequences at the lane and band edges of both
    # heights (16/24-row lanes, 512/768-row bands) and longer than a band
    rng = np.random.Generator(np.random.PCG64(515))
    db_s = random_sequences(516, 1990, 300, 0.5, 20, 1000).as_list()
    for L in (1, 15, 16, 17, 23, 24, 25, 47, 48, 49, 511, 512, 513, 767, 768, 769, 1023, 1024, 1025, 1536, 1537,
              2300, 3000):
        db_s.append(rng.integers(0, 20, size=L).astype(np.uint8))
    rng.shuffle(db_s)
    db = from_list(db_s)
    q = from_list([rng.integers(0, 20, size=144).astype(np.uint8)])
    got = _search(api, db, q, mode)
    _assert_equal(got, oracle.scores(q, db, BLOSUM62, 10, 2))


def test_searches_from_several_threads(api):
    # plans and searches from four host threads at once on one database
    # (per-thread planner tables, the shared occupancy cache, the memory
    # pool and the database's unit statistics), small-batch and inter-task
    # plans, each result exact
    import threading

    db_s = random_sequences(91, 1500, 300, 0.5, 1, 1200)
    db = api.Database.from_sequences(db_s)
    cases = [random_sequences(92 + i, n, 250, 0.6, 1, 1400) for i, n in enumerate((1, 3, 2, 9))]
    exp = [oracle.scores(q, db_s, BLOSUM62, 10, 2) for q in cases]
    got = [None] * len(cases)
    errors = []

    def run(i):
        try:
            import torch

            with torch.cuda.stream(torch.cuda.Stream()):
                for mode in ("packed", "int32"):
                    r = api.search(db, cases[i].residues, cases[i].offsets, BLOSUM62, 10, 2, mode)
                    got[i] = r if mode == "packed" else got[i]
                    if not np.array_equal(r, exp[i]):
                        errors.append((i, mode))
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=run, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    db.close()
    assert not errors, errors


def test_kept_track_layouts(api):
    # small batches of transposed jobs against one database: the first
    # search of each lane height and 16-bit / int32 routing builds a lane
    # table the database keeps (its device bytes grow), a repeat reuses it,
    # and beyond eight kept tables a plan builds its own.  The routing cut
    # moves with the largest substitution score: a 700-residue query under
    # matrices whose largest entry is 52..63 sends sequences longer than
    # (32767 - max) / max (629..519 residues) to int32 tracks.  Every score
    # against the oracle.
    rng = np.random.Generator(np.random.PCG64(8808))
    lens = [int(x) for x in rng.integers(20, 480, size=180)] + [int(x) for x in rng.integers(480, 700, size=100)]
    lens += [0, 1, 513, 900, 1100, 1700]
    db_s = from_list([rng.integers(0, 20, size=L).astype(np.uint8) for L in lens])
    db = api.Database.from_sequences(db_s)
    q144 = from_list([rng.integers(0, 20, size=144).astype(np.uint8)])
    q700 = from_list([rng.integers(0, 20, size=700).astype(np.uint8), rng.integers(0, 20, size=90).astype(np.uint8)])
    mixed = from_list([rng.integers(0, 20, size=1100).astype(np.uint8), rng.integers(0, 20, size=60).astype(np.uint8)])

    def run(q, sm, mode, opts=None):
        pq = api.PreparedQueries(db, q.residues, q.offsets, sm, 10, 2, mode, opts=opts)
        got = pq.search().cpu().numpy()
        pq.status()
        pq.close()
        _assert_equal(got, oracle.scores(q, db_s, sm, 10, 2))
        return db.stats()[2]

    try:
        b0 = db.stats()[2]
        b1 = run(q144, BLOSUM62, "packed")
        assert b1 > b0
        assert run(q144, BLOSUM62, "packed") == b1  # reused
        b2 = run(q144, BLOSUM62, "int32")
        assert b2 > b1
        sizes = []
        for top in range(52, 64):
            sm = BLOSUM62.copy()
            sm[3, 3] = top
            sizes.append(run(q700, sm, "packed"))
        kept = [b2] + sizes
        grown = sum(1 for a, b in zip(kept, kept[1:]) if b > a)
        assert grown == 6, sizes  # eight tables kept in all, then none
        assert run(mixed, BLOSUM62, "packed", api.options(band_stream="always")) == sizes[-1]
        assert run(mixed, BLOSUM62, "int32", api.options(band_stream="always")) == sizes[-1]
    finally:
        db.close()
