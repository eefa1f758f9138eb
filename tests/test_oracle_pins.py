"""Pins for the CPU oracle (Sec. 2.2, Eqs. 1-3; Algorithm 1).

Every check here compares the oracle with something other than itself:
brute-force enumeration of alignments, closed forms, invariants, special
cases that reduce to other textbook algorithms, and hand-derived gap-cost
cases (tests/golden/gap_cost_cases.json).
"""

import itertools
import json
import os

import numpy as np
import pytest

from tests import _pins
from workload import encode, random_sequences
from workload.matrices import ALPHABET, BLOSUM62, ROBINSON_FREQS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_seq(rng, n, alphabet=20):
    return rng.integers(0, alphabet, size=n).astype(np.uint8)


# --------------------------------------------------------------------------
# the scoring data entered from the literature
# --------------------------------------------------------------------------

def test_blosum62_shape_and_published_properties():
    B = BLOSUM62.astype(int)
    assert B.shape == (20, 20)
    assert (B == B.T).all()
    diag = np.diag(B)
    assert diag.min() == 4 and diag.max() == 11
    assert B[ALPHABET.index("W"), ALPHABET.index("W")] == 11
    assert diag.sum() == 116
    off = B[~np.eye(20, dtype=bool)]
    assert off.min() == -4 and off.max() == 3


def test_background_frequencies():
    f = ROBINSON_FREQS
    assert (f > 0).all()
    assert abs(f.sum() - 1.0) < 1e-4
    # a log-odds matrix has a negative expected score under its background
    assert float(f @ BLOSUM62.astype(float) @ f) < 0


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(40))
def test_oracle_equals_brute_force_random(oracle_mod, seed):
    rng = _rng(100 + seed)
    m, n = int(rng.integers(0, 7)), int(rng.integers(0, 7))
    q, d = _rand_seq(rng, m), _rand_seq(rng, n)
    go, ge = [(10, 2), (3, 1), (0, 4), (5, 0), (1, 1)][seed % 5]
    assert oracle_mod.score(q, d, BLOSUM62, go, ge) == _pins.brute_force(q, d, BLOSUM62, go, ge)


@pytest.mark.parametrize("seed", range(12))
def test_oracle_equals_brute_force_asymmetric_matrix(oracle_mod, seed):
    # an asymmetric matrix catches a transposed substitution lookup
    rng = _rng(300 + seed)
    sm = rng.integers(-6, 9, size=(20, 20)).astype(np.int8)
    q, d = _rand_seq(rng, int(rng.integers(1, 7)), 6), _rand_seq(rng, int(rng.integers(1, 7)), 6)
    assert oracle_mod.score(q, d, sm, 4, 1) == _pins.brute_force(q, d, sm, 4, 1)


def test_oracle_equals_brute_force_exhaustive_small_alphabet(oracle_mod):
    # every pair of sequences up to length 3 over a 3-letter sub-alphabet
    sm = np.full((20, 20), -3, dtype=np.int8)
    sm[0, 0], sm[1, 1], sm[2, 2] = 5, 4, 6
    sm[0, 1], sm[1, 0], sm[2, 0] = 1, -1, 2
    seqs = [np.array(s, dtype=np.uint8) for L in range(4) for s in itertools.product(range(3), repeat=L)]
    for q in seqs:
        for d in seqs:
            for go, ge in ((2, 1), (0, 3)):
                assert oracle_mod.score(q, d, sm, go, ge) == _pins.brute_force(q, d, sm, go, ge), (q, d, go, ge)


# --------------------------------------------------------------------------
# hand-derived gap costs (golden)
# --------------------------------------------------------------------------

def _id10():
    sm = np.full((20, 20), -30, dtype=np.int8)
    np.fill_diagonal(sm, 10)
    return sm


def test_gap_cost_golden_cases(oracle_mod):
    with open(os.path.join(GOLDEN, "gap_cost_cases.json")) as f:
        spec = json.load(f)
    assert spec["matrix"] == "id10"
    sm = _id10()
    for case in spec["cases"]:
        q, d = encode(case["q"]), encode(case["d"])
        got = oracle_mod.score(q, d, sm, case["gap_open"], case["gap_extend"])
        assert got == case["expected"], case
        # the same case, database and query swapped (symmetric matrix)
        assert oracle_mod.score(d, q, sm, case["gap_open"], case["gap_extend"]) == case["expected"]


def test_gap_convention_maps_to_literal_equations(oracle_mod):
    # Eqs. 2-3 charge Go for the first gap position and Ge for each further
    # one; this library's (gap_open, gap_extend) = (Go - Ge, Ge).
    rng = _rng(7)
    for _ in range(10):
        q, d = _rand_seq(rng, 12), _rand_seq(rng, 15)
        assert oracle_mod.score(q, d, BLOSUM62, 10, 2) == _pins.literal_gotoh(q, d, BLOSUM62, 12, 2)
        assert oracle_mod.score(q, d, BLOSUM62, 8, 2) == _pins.literal_gotoh(q, d, BLOSUM62, 10, 2)


# --------------------------------------------------------------------------
# closed forms and special cases
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_self_score_is_diagonal_sum(oracle_mod, seed):
    # BLOSUM62: every off-diagonal entry (<= 3) is below half the sum of the
    # two diagonal entries (>= 4 each) and gaps cost > 0, so the identity
    # alignment is optimal and S(Q, Q) = sum_i SM(q_i, q_i).
    rng = _rng(500 + seed)
    q = _rand_seq(rng, int(rng.integers(1, 400)))
    expected = int(sum(int(BLOSUM62[c, c]) for c in q))
    assert oracle_mod.score(q, q, BLOSUM62, 10, 2) == expected


@pytest.mark.parametrize("seed", range(10))
def test_single_residue_query(oracle_mod, seed):
    rng = _rng(600 + seed)
    q = _rand_seq(rng, 1)
    d = _rand_seq(rng, int(rng.integers(0, 60)))
    expected = max([0] + [int(BLOSUM62[q[0], c]) for c in d])
    assert oracle_mod.score(q, d, BLOSUM62, 10, 2) == expected


@pytest.mark.parametrize("seed", range(8))
def test_prohibitive_gaps_reduce_to_ungapped_kadane(oracle_mod, seed):
    rng = _rng(700 + seed)
    q, d = _rand_seq(rng, int(rng.integers(1, 40))), _rand_seq(rng, int(rng.integers(1, 40)))
    go = 11 * min(len(q), len(d)) + 1  # no gap can ever pay for itself
    assert oracle_mod.score(q, d, BLOSUM62, go, 1) == _pins.ungapped_best(q, d, BLOSUM62)


@pytest.mark.parametrize("seed", range(8))
def test_zero_open_reduces_to_linear_gap_sw(oracle_mod, seed):
    rng = _rng(800 + seed)
    q, d = _rand_seq(rng, int(rng.integers(1, 35))), _rand_seq(rng, int(rng.integers(1, 35)))
    g = int(rng.integers(1, 6))
    assert oracle_mod.score(q, d, BLOSUM62, 0, g) == _pins.linear_gap_sw(q, d, BLOSUM62, g)


def test_all_negative_scores_give_zero(oracle_mod):
    sm = np.full((20, 20), -1, dtype=np.int8)
    rng = _rng(9)
    assert oracle_mod.score(_rand_seq(rng, 50), _rand_seq(rng, 70), sm, 10, 2) == 0


def test_empty_sequences_score_zero(oracle_mod):
    z = np.zeros(0, np.uint8)
    one = np.array([5], np.uint8)
    assert oracle_mod.score(z, z, BLOSUM62, 10, 2) == 0
    assert oracle_mod.score(z, one, BLOSUM62, 10, 2) == 0
    assert oracle_mod.score(one, z, BLOSUM62, 10, 2) == 0


def test_invalid_codes_rejected(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.score(np.array([20], np.uint8), np.array([1], np.uint8), BLOSUM62, 10, 2)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(10))
def test_swap_symmetry_and_bounds(oracle_mod, seed):
    rng = _rng(1000 + seed)
    q, d = _rand_seq(rng, int(rng.integers(1, 300))), _rand_seq(rng, int(rng.integers(1, 300)))
    s = oracle_mod.score(q, d, BLOSUM62, 10, 2)
    assert s == oracle_mod.score(d, q, BLOSUM62, 10, 2)
    assert 0 <= s <= 11 * min(len(q), len(d))


@pytest.mark.parametrize("seed", range(6))
def test_monotone_under_extension(oracle_mod, seed):
    rng = _rng(1100 + seed)
    q, d = _rand_seq(rng, 80), _rand_seq(rng, 120)
    s = oracle_mod.score(q, d, BLOSUM62, 10, 2)
    ext = np.concatenate([d, _rand_seq(rng, 5)])
    pre = np.concatenate([_rand_seq(rng, 5), d])
    assert oracle_mod.score(q, ext, BLOSUM62, 10, 2) >= s
    assert oracle_mod.score(q, pre, BLOSUM62, 10, 2) >= s
    assert oracle_mod.score(q, d[10:90], BLOSUM62, 10, 2) <= s


@pytest.mark.parametrize("seed", range(10))
def test_boundary_init_zero_equals_neginf(oracle_mod, seed):
    # The paper initialises E and F with 0 on the first row/column; the
    # textbook uses -infinity.  E, F <= 0 never lift H above its 0 floor, so
    # both give the same score.
    rng = _rng(1200 + seed)
    q, d = _rand_seq(rng, int(rng.integers(1, 100))), _rand_seq(rng, int(rng.integers(1, 100)))
    go, ge = [(10, 2), (0, 1), (3, 7)][seed % 3]
    a = oracle_mod.score_init(q, d, BLOSUM62, go, ge, "zero")
    b = oracle_mod.score_init(q, d, BLOSUM62, go, ge, "neginf")
    assert a == b


def test_batch_matches_single_calls(oracle_mod):
    db = random_sequences(42, 60, 80, 0.5, 5, 200)
    qs = random_sequences(43, 4, 50, 0.5, 0, 120)
    all_scores = oracle_mod.scores(qs, db, BLOSUM62, 10, 2, threads=3)
    for i in range(len(qs)):
        for j in range(len(db)):
            assert all_scores[i, j] == oracle_mod.score(qs[i], db[j], BLOSUM62, 10, 2)
    sub = np.array([5, 0, 59, 17], dtype=np.int64)
    part = oracle_mod.scores(qs, db, BLOSUM62, 10, 2, subset=sub, threads=2)
    assert (part == all_scores[:, sub]).all()


# --- the DNA scoring of the pairwise workload (+1 / -3, gaps 5 + 2k) ---------

def test_dna_matrix_is_the_papers_scoring():
    from workload.matrices import DNA_GAP_EXTEND, DNA_GAP_OPEN, DNA_SUBMAT
    assert DNA_SUBMAT.shape == (20, 20)
    assert (np.diag(DNA_SUBMAT) == 1).all()
    assert (DNA_SUBMAT[~np.eye(20, dtype=bool)] == -3).all()
    assert (DNA_GAP_OPEN, DNA_GAP_EXTEND) == (5, 2)


@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_dna_identity_scores_its_length(oracle_mod, n):
    # with +1 matches, every mismatch or gap only lowers a path, so the full
    # diagonal of X against itself is optimal: S(X, X) = |X|
    from workload.matrices import DNA_SUBMAT
    x = np.random.Generator(np.random.PCG64(n)).integers(0, 4, size=n).astype(np.uint8)
    assert oracle_mod.score(x, x, DNA_SUBMAT, 5, 2) == n


@pytest.mark.parametrize("n,p", [(40, 0), (40, 1), (40, 20), (40, 38), (40, 39), (9, 4), (3, 1)])
def test_dna_one_substitution_closed_form(oracle_mod, n, p):
    # X against X with base p changed: the full diagonal scores (n - 1) - 3,
    # the two unchanged flanks p and n - 1 - p; a detour around the mismatch
    # needs a gap in each sequence (>= 2 x 7 > 4), so
    # S = max(n - 4, p, n - 1 - p)
    from workload.matrices import DNA_SUBMAT
    x = np.random.Generator(np.random.PCG64(100 + n)).integers(0, 4, size=n).astype(np.uint8)
    y = x.copy()
    y[p] = (y[p] + 1) % 4
    assert oracle_mod.score(x, y, DNA_SUBMAT, 5, 2) == max(n - 4, p, n - 1 - p)


def test_dna_brute_force(oracle_mod):
    from workload.matrices import DNA_SUBMAT
    rng = np.random.Generator(np.random.PCG64(77))
    for _ in range(40):
        a = rng.integers(0, 4, size=int(rng.integers(0, 6))).astype(np.uint8)
        b = rng.integers(0, 4, size=int(rng.integers(0, 6))).astype(np.uint8)
        assert oracle_mod.score(a, b, DNA_SUBMAT, 5, 2) == _pins.brute_force(a, b, DNA_SUBMAT, 5, 2)


# --- one optimal alignment (traceback) ----------------------------------------

def _check_alignment(oracle_mod, q, d, sm, go, ge):
    s, qb, qe, tb, te, ops = oracle_mod.align(q, d, sm, go, ge)
    assert s == oracle_mod.score(q, d, sm, go, ge)
    total, i, j = _pins.alignment_score(q, d, sm, go, ge, qb, tb, ops)
    assert total == s and (i, j) == (qe, te)
    if s > 0:
        assert ops[0] == "M" and ops[-1] == "M"  # a local alignment starts and ends on aligned pairs
    else:
        assert ops == "" and qb == qe and tb == te
    return s, ops


@pytest.mark.parametrize("seed", range(6))
def test_alignment_reproduces_the_score(oracle_mod, seed):
    rng = np.random.Generator(np.random.PCG64(500 + seed))
    sm = BLOSUM62 if seed % 2 == 0 else rng.integers(-8, 9, size=(20, 20)).astype(np.int8)
    for _ in range(20):
        q = rng.integers(0, 20, size=int(rng.integers(0, 40))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(0, 40))).astype(np.uint8)
        if rng.random() < 0.5 and len(q) > 4:
            d = np.concatenate([d[:5], q[2:-2], d[5:]]).astype(np.uint8)  # a shared stretch
        _check_alignment(oracle_mod, q, d, sm, int(rng.integers(0, 12)), int(rng.integers(0, 4)))


def test_alignment_brute_force_small(oracle_mod):
    rng = np.random.Generator(np.random.PCG64(501))
    for _ in range(60):
        q = rng.integers(0, 20, size=int(rng.integers(0, 6))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(0, 6))).astype(np.uint8)
        s, _ = _check_alignment(oracle_mod, q, d, BLOSUM62, 3, 1)
        assert s == _pins.brute_force(q, d, BLOSUM62, 3, 1)


def test_alignment_of_a_gapped_copy(oracle_mod):
    # a query and a copy with 3 extra residues in the middle: with cheap gaps
    # the optimum bridges them with one D run of length 3
    from workload.matrices import DNA_SUBMAT
    rng = np.random.Generator(np.random.PCG64(502))
    x = rng.integers(0, 4, size=80).astype(np.uint8)
    y = np.concatenate([x[:40], rng.integers(0, 4, size=3).astype(np.uint8), x[40:]]).astype(np.uint8)
    s, ops = _check_alignment(oracle_mod, x, y, DNA_SUBMAT, 2, 1)
    assert s == 80 - (2 + 3 * 1) and ops.count("D") == 3 and ops.count("I") == 0
