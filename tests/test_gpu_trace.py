"""GPU traceback (sw_traceback) against the CPU oracle's alignment.

Both sides recompute the pair's matrix and walk back from the first cell, in
row-major order, that holds the score, with the same order of preference
(the zero floor, the diagonal, E, F; a gap opening before an extension), so
the alignments must be identical; each one is also checked on its own (its
score recomputed from the operations, its coordinates, aligned ends).
"""

import numpy as np
import pytest

import oracle
from tests import _pins
from workload import from_list, make_dna_pair
from workload.matrices import BLOSUM62, DNA_SUBMAT

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


def _check(api, db_seqs, q_seqs, hits, sm, go, ge):
    db = api.Database.from_sequences(db_seqs)
    try:
        got = api.traceback(db, q_seqs.residues, q_seqs.offsets, hits, sm, go, ge)
    finally:
        db.close()
    for (qi, ti), g in zip(hits, got):
        q, d = q_seqs[qi], db_seqs[ti]
        exp = oracle.align(q, d, sm, go, ge)
        assert g == exp, (qi, ti, g[:5], exp[:5])
        s, qb, qe, tb, te, ops = g
        total, i, j = _pins.alignment_score(q, d, sm, go, ge, qb, tb, ops)
        assert total == s and (i, j) == (qe, te)
    return got


def test_hits_of_a_search(api):
    # the three best hits of each query of a search plus zero-score pairs;
    # queries up to 1,300 residues (three 512-row chunks), database sequences
    # of 0..900 residues, some holding stretches of a query
    rng = np.random.Generator(np.random.PCG64(90))
    ql = [1300, 700, 513, 512, 100, 7, 0]
    qs = [rng.integers(0, 20, size=n).astype(np.uint8) for n in ql]
    seqs = [rng.integers(0, 20, size=int(rng.integers(0, 900))).astype(np.uint8) for _ in range(120)]
    for k, qi in enumerate((0, 1, 2, 0)):
        src = qs[qi]
        a = int(rng.integers(0, len(src) // 2))
        seqs[10 * k + 3] = np.concatenate([seqs[10 * k + 3][:20], src[a:a + 300], seqs[10 * k + 3][20:]])
    db_seqs, q_seqs = from_list(seqs), from_list(qs)
    scores = oracle.scores(q_seqs, db_seqs, BLOSUM62, 10, 2)
    hits = []
    for qi in range(len(ql)):
        hits += [(qi, int(t)) for t in np.argsort(-scores[qi], kind="stable")[:3]]
    hits += [(5, 1), (6, 2), (0, 0)]
    got = _check(api, db_seqs, q_seqs, hits, BLOSUM62, 10, 2)
    for (qi, ti), g in zip(hits, got):
        assert g[0] == scores[qi, ti]


@pytest.mark.parametrize("go,ge", [(5, 2), (0, 1), (20, 0)])
def test_dna_hits_with_indels(api, go, ge):
    # diverged DNA copies (substitutions and indels): long gapped paths
    q, t = make_dna_pair(m=1500, n=1400, seed=91)
    rng = np.random.Generator(np.random.PCG64(92))
    seqs = [t, t[200:900], rng.integers(0, 4, size=300).astype(np.uint8), q[::-1].copy()]
    _check(api, from_list(seqs), from_list([q, q[100:700]]), [(0, 0), (0, 1), (0, 2), (0, 3), (1, 0), (1, 1)],
           DNA_SUBMAT, go, ge)


def test_many_hits_and_repeats(api):
    # 200 hits in one call (one CTA each), the same pair several times
    rng = np.random.Generator(np.random.PCG64(93))
    seqs = [rng.integers(0, 20, size=int(rng.integers(1, 300))).astype(np.uint8) for _ in range(50)]
    qs = [rng.integers(0, 20, size=int(rng.integers(1, 300))).astype(np.uint8) for _ in range(8)]
    hits = [(int(rng.integers(0, 8)), int(rng.integers(0, 50))) for _ in range(197)] + [(1, 2)] * 3
    _check(api, from_list(seqs), from_list(qs), hits, BLOSUM62, 10, 2)


@pytest.mark.parametrize("with_short", [False, True])
def test_long_queries_several_rounds(api, with_short):
    # queries of 18 and 9 chunks of 512 rows: 8 warps per hit take the chunks
    # in rounds, the last warp's rows passing to the first through the
    # strip; with_short: hits of a 1,500-residue query too (3 chunks, one
    # round, five warps of its CTA idle), listed between the others
    rng = np.random.Generator(np.random.PCG64(95))
    q0 = rng.integers(0, 20, size=9000).astype(np.uint8)
    q1 = rng.integers(0, 20, size=4100).astype(np.uint8)
    q2 = rng.integers(0, 20, size=1500).astype(np.uint8)
    t0 = np.concatenate([rng.integers(0, 20, size=100).astype(np.uint8), q0[2000:3200], q0[6000:6300]])
    t0[300:900:7] = (t0[300:900:7] + 3) % 20
    t1 = np.concatenate([q1[3500:4100], rng.integers(0, 20, size=50).astype(np.uint8), q1[:400], q2[700:1100]])
    t2 = rng.integers(0, 20, size=777).astype(np.uint8)
    hits = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 0), (1, 2)]
    if with_short:
        hits = [(2, 1), (0, 0), (2, 0), (0, 1), (0, 2), (2, 2), (1, 1), (1, 0), (1, 2)]
    _check(api, from_list([t0, t1, t2]), from_list([q0, q1, q2]), hits, BLOSUM62, 10, 2)


def test_invalid_hits(api):
    from paper_2412_08308_gb300._native import SW_EINVAL, SwError

    rng = np.random.Generator(np.random.PCG64(94))
    db_seqs = from_list([rng.integers(0, 20, size=50).astype(np.uint8) for _ in range(4)])
    q = from_list([rng.integers(0, 20, size=30).astype(np.uint8)])
    db = api.Database.from_sequences(db_seqs)
    try:
        for hits in ([(1, 0)], [(0, 4)], [(-1, 0)], [(0, -1)]):
            with pytest.raises(SwError) as e:
                api.traceback(db, q.residues, q.offsets, hits, BLOSUM62, 10, 2)
            assert e.value.code == SW_EINVAL
        assert api.traceback(db, q.residues, q.offsets, [], BLOSUM62, 10, 2) == []
    finally:
        db.close()
