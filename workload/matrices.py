"""Scoring data used as *inputs* by every workload: the 20-letter protein
alphabet, the BLOSUM62 substitution matrix and the Robinson & Robinson
amino-acid background frequencies.

This module holds data only; it computes nothing of the alignment method.

* BLOSUM62: Henikoff S. & Henikoff J.G. (1992), "Amino acid substitution
  matrices from protein blocks", PNAS 89:10915-10919, the 62% clustering
  matrix in half-bit units, restricted to the 20 standard amino acids.  The
  paper scores its protein search with it (Sec. 4.1, experimental design).
* Background frequencies: Robinson A.B. & Robinson L.R. (1991), "Distribution
  of glutamine and asparagine residues and their near neighbors in peptides
  and proteins", PNAS 88:8880-8884 (the amino-acid composition widely used as
  the protein background law).

Residue codes are the positions in ``ALPHABET`` (0..19).
"""

import numpy as np

ALPHABET = "ARNDCQEGHILKMFPSTWYV"

_BLOSUM62_ROWS = """
 4 -1 -2 -2  0 -1 -1  0 -2 -1 -1 -1 -1 -2 -1  1  0 -3 -2  0
-1  5  0 -2 -3  1  0 -2  0 -3 -2  2 -1 -3 -2 -1 -1 -3 -2 -3
-2  0  6  1 -3  0  0  0  1 -3 -3  0 -2 -3 -2  1  0 -4 -2 -3
-2 -2  1  6 -3  0  2 -1 -1 -3 -4 -1 -3 -3 -1  0 -1 -4 -3 -3
 0 -3 -3 -3  9 -3 -4 -3 -3 -1 -1 -3 -1 -2 -3 -1 -1 -2 -2 -1
-1  1  0  0 -3  5  2 -2  0 -3 -2  1  0 -3 -1  0 -1 -2 -1 -2
-1  0  0  2 -4  2  5 -2  0 -3 -3  1 -2 -3 -1  0 -1 -3 -2 -2
 0 -2  0 -1 -3 -2 -2  6 -2 -4 -4 -2 -3 -3 -2  0 -2 -2 -3 -3
-2  0  1 -1 -3  0  0 -2  8 -3 -3 -1 -2 -1 -2 -1 -2 -2  2 -3
-1 -3 -3 -3 -1 -3 -3 -4 -3  4  2 -3  1  0 -3 -2 -1 -3 -1  3
-1 -2 -3 -4 -1 -2 -3 -4 -3  2  4 -2  2  0 -3 -2 -1 -2 -1  1
-1  2  0 -1 -3  1  1 -2 -1 -3 -2  5 -1 -3 -1  0 -1 -3 -2 -2
-1 -1 -2 -3 -1  0 -2 -3 -2  1  2 -1  5  0 -2 -1 -1 -1 -1  1
-2 -3 -3 -3 -2 -3 -3 -3 -1  0  0 -3  0  6 -4 -2 -2  1  3 -1
-1 -2 -2 -1 -3 -1 -1 -2 -2 -3 -3 -1 -2 -4  7 -1 -1 -4 -3 -2
 1 -1  1  0 -1  0  0  0 -1 -2 -2  0 -1 -2 -1  4  1 -3 -2 -2
 0 -1  0 -1 -1 -1 -1 -2 -2 -1 -1 -1 -1 -2 -1  1  5 -2 -2  0
-3 -3 -4 -4 -2 -2 -3 -2 -2 -3 -2 -3 -1  1 -4 -3 -2 11  2 -3
-2 -2 -2 -3 -2 -1 -2 -3  2 -1 -1 -2 -1  3 -3 -2 -2  2  7 -1
 0 -3 -3 -3 -1 -2 -2 -3 -3  3  1 -2  1 -1 -2 -2  0 -3 -1  4
"""

BLOSUM62 = np.array([[int(v) for v in row.split()] for row in _BLOSUM62_ROWS.strip().splitlines()],
                    dtype=np.int8)

# Robinson & Robinson (1991) composition, in ALPHABET order.
ROBINSON_FREQS = np.array([
    0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377, 0.02199, 0.05142,
    0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120, 0.05841, 0.01330, 0.03216, 0.06441,
], dtype=np.float64)

# Scoring used throughout the paper's protein benchmark: BLOSUM62 with gap
# penalties 10/2.  In this library a gap run of length k costs
# gap_open + k * gap_extend = 10 + 2k.
GAP_OPEN = 10
GAP_EXTEND = 2


# Scoring of the paper's DNA pairwise alignments (Sec. 4.1): +1 for a match,
# -3 for a mismatch, gap penalties 5/2 (read like the protein ones: a gap run
# of length k costs 5 + 2k).  Nucleotides use codes 0..3 (A, C, G, T); the
# matrix spans the library's 20-code alphabet with the same rule.
DNA_ALPHABET = "ACGT"
DNA_MATCH = 1
DNA_MISMATCH = -3
DNA_GAP_OPEN = 5
DNA_GAP_EXTEND = 2
DNA_SUBMAT = np.full((20, 20), DNA_MISMATCH, dtype=np.int8)
np.fill_diagonal(DNA_SUBMAT, DNA_MATCH)


def encode(text):
    """Map a protein string over ``ALPHABET`` to uint8 codes."""
    lut = {c: i for i, c in enumerate(ALPHABET)}
    return np.array([lut[c] for c in text], dtype=np.uint8)


def decode(codes):
    return "".join(ALPHABET[int(c)] for c in codes)
