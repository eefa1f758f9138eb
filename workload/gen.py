"""Seeded synthetic protein workloads.

These inputs stand in for the paper's protein benchmark (Env. NR 2021_04 as
the database, 20 Swiss-Prot queries of 144-5478 residues, BLOSUM62, gaps
10/2; Sec. 4.1), which is not available here.  Recipe:

* sequence lengths: ``L = clip(round(exp(ln(median) + sigma * N(0,1))), lo, hi)``;
* residues: i.i.d. draws from the Robinson & Robinson background law over the
  20 standard amino acids (``workload.matrices.ROBINSON_FREQS``);
* planted homologs: per position a substitution with probability ``p_sub`` (a
  background draw different from the original) and an indel event with
  probability ``p_indel`` (insertion or deletion with equal odds, length
  ``Geometric(0.5)`` on 1, 2, ...);
* every generator is driven by ``numpy.random.PCG64`` with a fixed seed.

The module holds input generation only: no part of the alignment method.
It is the one module that both the CPU oracle's tests and the GPU path use.
"""

from dataclasses import dataclass

import numpy as np

from .matrices import ROBINSON_FREQS


@dataclass
class Sequences:
    """A set of sequences as one concatenated uint8 code array plus offsets.

    ``offsets`` has ``len + 1`` entries; sequence ``i`` is
    ``residues[offsets[i]:offsets[i+1]]``.
    """

    residues: np.ndarray
    offsets: np.ndarray

    def __post_init__(self):
        self.residues = np.ascontiguousarray(self.residues, dtype=np.uint8)
        self.offsets = np.ascontiguousarray(self.offsets, dtype=np.int64)

    def __len__(self):
        return len(self.offsets) - 1

    def __getitem__(self, i):
        return self.residues[self.offsets[i]:self.offsets[i + 1]]

    @property
    def lengths(self):
        return np.diff(self.offsets)

    @property
    def total(self):
        return int(self.offsets[-1])

    def subset(self, idx):
        return from_list([self[int(i)] for i in idx])

    def as_list(self):
        return [self[i] for i in range(len(self))]


def from_list(seqs):
    seqs = [np.asarray(s, dtype=np.uint8) for s in seqs]
    offsets = np.zeros(len(seqs) + 1, dtype=np.int64)
    if seqs:
        offsets[1:] = np.cumsum([len(s) for s in seqs])
        res = np.concatenate(seqs) if offsets[-1] > 0 else np.zeros(0, np.uint8)
    else:
        res = np.zeros(0, np.uint8)
    return Sequences(res, offsets)


def lognormal_lengths(rng, n, median, sigma, lo, hi):
    z = rng.standard_normal(n)
    lengths = np.rint(np.exp(np.log(median) + sigma * z))
    return np.clip(lengths, lo, hi).astype(np.int64)


def random_residues(rng, total):
    """``total`` i.i.d. residue codes from the background law."""
    cdf = np.cumsum(ROBINSON_FREQS)
    cdf /= cdf[-1]
    out = np.empty(total, dtype=np.uint8)
    step = 1 << 24
    for s in range(0, total, step):
        e = min(total, s + step)
        out[s:e] = np.searchsorted(cdf, rng.random(e - s), side="right")
    np.minimum(out, 19, out=out)
    return out


def random_sequences(seed, n, median, sigma, lo, hi):
    rng = np.random.Generator(np.random.PCG64(seed))
    lengths = lognormal_lengths(rng, n, median, sigma, lo, hi)
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    return Sequences(random_residues(rng, int(offsets[-1])), offsets)


def random_sequence(rng, length):
    return random_residues(rng, int(length))


def mutate(rng, seq, p_sub=0.10, p_indel=0.01):
    """A homolog of ``seq`` under the substitution + indel model above."""
    cdf = np.cumsum(ROBINSON_FREQS)
    cdf /= cdf[-1]
    out = []
    i = 0
    n = len(seq)
    while i < n:
        if rng.random() < p_indel:
            k = int(rng.geometric(0.5))
            if rng.random() < 0.5:  # insertion of k background residues
                out.extend(int(min(19, np.searchsorted(cdf, rng.random(), side="right"))) for _ in range(k))
            else:  # deletion of k residues
                i += k
                continue
        c = int(seq[i])
        if rng.random() < p_sub:
            while True:
                r = int(min(19, np.searchsorted(cdf, rng.random(), side="right")))
                if r != c:
                    c = r
                    break
        out.append(c)
        i += 1
    return np.array(out, dtype=np.uint8)


# ---------------------------------------------------------------------------
# The five benchmark workloads, by name.
# ---------------------------------------------------------------------------

DB_SEED = 1000
QUERY_SEED = 2000
ARRIVAL_SEED = 3000
SAMPLE_SEED = 4000

WORKLOADS = {
    "one_query_vs_2k": "1 query of 144 residues x 2,000 proteins (~1e8 cells)",
    "twenty_queries_vs_200k": "20 queries of 144..5478 residues (log-uniform) x 200,000 proteins (~67.5M residues)",
    "homologs_8k": "2,000 proteins + 10 planted ~8,000-residue homologs of an 8,000-residue query; "
                   "queries: the 144-residue query and the 8,000-residue source",
    "thousand_queries_vs_50k": "1,000 queries (median 350, 50..2000) x 50,000 proteins",
    "serving_500k": "500,000 proteins (~180M residues); 10,000 queries (median 400, 30..3000) arriving "
                    "as a Poisson process at 50/s",
}


def twenty_query_lengths():
    """20 query lengths spread log-uniformly over 144..5478 residues."""
    return [int(round(144 * (5478 / 144) ** (k / 19))) for k in range(20)]


def make_workload(name, n_db=None, n_queries=None):
    """Build a named workload (see WORKLOADS).

    Returns a dict with ``db`` (Sequences), ``queries`` (Sequences) and, where
    the workload has them, ``homolog_ids`` (homologs_8k) or ``arrivals``
    (serving_500k, seconds).  ``n_db`` / ``n_queries`` shrink it (tests only).
    Seeds: database 1000 + k, queries 2000 + k, k = 1..5 in the order above.
    """
    if name not in WORKLOADS:
        raise ValueError(f"unknown workload {name!r}; one of {sorted(WORKLOADS)}")
    out = {"name": name}
    if name in ("one_query_vs_2k", "homologs_8k"):
        db = random_sequences(DB_SEED + 1, n_db or 2000, 300, 0.5, 20, 1000)
        rng = np.random.Generator(np.random.PCG64(QUERY_SEED + 1))
        q144 = random_sequence(rng, 144)
        if name == "one_query_vs_2k":
            out.update(db=db, queries=from_list([q144]))
            return out
        rng3 = np.random.Generator(np.random.PCG64(QUERY_SEED + 3))
        src = random_sequence(rng3, 8000)
        n_hom = max(1, round(0.005 * len(db)))
        homologs = [mutate(rng3, src) for _ in range(n_hom)]
        seqs = db.as_list()
        pos = np.sort(rng3.choice(len(seqs) + n_hom, size=n_hom, replace=False))
        merged, hi, si = [], 0, 0
        for p in range(len(seqs) + n_hom):
            if hi < n_hom and pos[hi] == p:
                merged.append(homologs[hi])
                hi += 1
            else:
                merged.append(seqs[si])
                si += 1
        out.update(db=from_list(merged), queries=from_list([q144, src]), homolog_ids=pos.astype(np.int64))
        return out
    if name == "twenty_queries_vs_200k":
        db = random_sequences(DB_SEED + 2, n_db or 200_000, 300, 0.5, 20, 1000)
        rng = np.random.Generator(np.random.PCG64(QUERY_SEED + 2))
        lens = twenty_query_lengths()
        if n_queries:
            lens = lens[:n_queries]
        out.update(db=db, queries=from_list([random_sequence(rng, m) for m in lens]))
        return out
    if name == "thousand_queries_vs_50k":
        db = random_sequences(DB_SEED + 4, n_db or 50_000, 300, 0.5, 20, 1000)
        q = random_sequences(QUERY_SEED + 4, n_queries or 1000, 350, 0.5, 50, 2000)
        out.update(db=db, queries=q)
        return out
    db = random_sequences(DB_SEED + 5, n_db or 500_000, 300, 0.65, 20, 1000)
    nq = n_queries or 10_000
    q = random_sequences(QUERY_SEED + 5, nq, 400, 0.5, 30, 3000)
    rng = np.random.Generator(np.random.PCG64(ARRIVAL_SEED))
    arrivals = np.cumsum(rng.exponential(1.0 / 50.0, size=nq))
    out.update(db=db, queries=q, arrivals=arrivals)
    return out


def query_batch_144(n, seed=QUERY_SEED + 6):
    """n seeded queries of 144 residues (the single query's length), drawn
    like every other query: a batch of requests shaped like the one-query
    workload, searched together against its 2,000 proteins."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return from_list([random_sequence(rng, 144) for _ in range(n)])


# ---------------------------------------------------------------------------
# DNA pairs (the paper's pairwise workload, Sec. 4.1, Table 3): the genome
# pairs are not available; each stand-in pair is a uniform random target of
# the database sequence's size and a query of the query sequence's size that
# is a diverged copy of the target (10% substitutions, indel events at 1% of
# positions, insertion or deletion with equal odds, length Geometric(0.5)),
# extended with random bases when the query is the longer one.
# ---------------------------------------------------------------------------

DNA_SEED = 5000
DNA_PAIRS = {  # name: (query length, target length), the sizes of the paper's five pairs
    "dna_162k_x_172k": (162_000, 172_000),
    "dna_543k_x_536k": (543_000, 536_000),
    "dna_1m_x_1m": (1_000_000, 1_000_000),
    "dna_3m_x_3m": (3_000_000, 3_000_000),
    "dna_7m_x_5m": (7_000_000, 5_000_000),
}


def diverge_dna(rng, seq, p_sub=0.10, p_indel=0.01):
    """A diverged copy of a DNA code array (codes 0..3), vectorised: each
    position is substituted by one of the three other bases with probability
    p_sub; indel events start before a position with probability p_indel."""
    seq = np.asarray(seq, dtype=np.uint8)
    n = seq.size
    sub = rng.random(n) < p_sub
    out = seq.copy()
    out[sub] = (out[sub] + rng.integers(1, 4, size=int(sub.sum()))) % 4
    ev = np.flatnonzero(rng.random(n) < p_indel)
    if ev.size == 0:
        return out
    lens = rng.geometric(0.5, size=ev.size)
    ins = rng.random(ev.size) < 0.5
    pieces, start = [], 0
    for pos, k, is_ins in zip(ev.tolist(), lens.tolist(), ins.tolist()):
        if pos < start:
            continue  # inside a deletion
        pieces.append(out[start:pos])
        if is_ins:
            pieces.append(rng.integers(0, 4, size=k).astype(np.uint8))
            start = pos
        else:
            start = pos + k
    pieces.append(out[start:])
    return np.concatenate(pieces).astype(np.uint8)


def make_dna_pair(name=None, m=None, n=None, seed=DNA_SEED):
    """(query, target) uint8 code arrays: a named pair of DNA_PAIRS, or sizes
    m, n.  The query has about m codes (indels change it slightly)."""
    if name is not None:
        m, n = DNA_PAIRS[name]
        seed = DNA_SEED + list(DNA_PAIRS).index(name) + 1
    rng = np.random.Generator(np.random.PCG64(seed))
    target = rng.integers(0, 4, size=n).astype(np.uint8)
    common = min(m, n)
    query = diverge_dna(rng, target[:common])
    if m > common:
        query = np.concatenate([query, rng.integers(0, 4, size=m - common).astype(np.uint8)])
    return query, target


def sample_indices(n, k, seed=SAMPLE_SEED):
    """A seeded sample of ``k`` distinct subject indices out of ``n`` (sorted)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(k, n), replace=False)).astype(np.int64)
