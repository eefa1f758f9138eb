"""Seeded synthetic inputs (sequences, scoring data) shared by the oracle's
tests, the GPU tests and the benchmark.  Input generation only."""

from .matrices import ALPHABET, BLOSUM62, ROBINSON_FREQS, GAP_OPEN, GAP_EXTEND, encode, decode  # noqa: F401
from .matrices import DNA_SUBMAT, DNA_GAP_OPEN, DNA_GAP_EXTEND  # noqa: F401
from .gen import Sequences, from_list, make_workload, WORKLOADS, random_sequences, sample_indices, mutate  # noqa: F401
from .gen import query_batch_144  # noqa: F401
from .gen import DNA_PAIRS, make_dna_pair, diverge_dna  # noqa: F401
