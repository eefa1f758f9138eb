"""GPU parity of the long-pair band kernel (sw_align_pair) against the CPU oracle.

The kernel cuts the query rows into bands, one per warp, and runs them as a
pipeline across all warps; the options below shrink the bands, cap the warps
and the boundary rings so that small pairs still span many bands, several
bands per warp, full rings and every kind of boundary.  Scores are int32; the
bar is equality.
"""

import numpy as np
import pytest

import oracle
from workload import make_dna_pair
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


@pytest.mark.parametrize("warps,rows,ctas,ring", [(1, 8, 0, 0), (1, 8, 3, 0), (2, 16, 2, 0), (3, 8, 1, 0),
                                                 (16, 24, 0, 0), (16, 16, 0, 256), (2, 24, 1, 256), (1, 8, 1, 256),
                                                 (8, 8, 1, 256), (4, 4, 2, 256)])
def test_related_dna_pair(api, warps, rows, ctas, ring):
    # a diverged copy: bands of 128..768 rows, one per warp; with one or a few
    # warps in the grid each warp takes many bands in turn (every band then
    # follows the band above it on another warp or on the same one), and
    # 256-column boundary rings make every band wait for room
    q, t = make_dna_pair(m=3000, n=2900, seed=11)
    exp = oracle.score(q, t, DNA_SUBMAT, 5, 2)
    got = api.align_pair(q, t, DNA_SUBMAT, 5, 2, opts=api.pair_options(warps, rows, ctas, ring))
    assert got == exp


def test_many_bands_several_rounds(api):
    # 20,000 x 20,000 cells in 79 bands of 256 rows on 5 warps: 16 rounds of
    # the warp pipeline, rings of 4,096 columns reused every 6 bands
    q, t = make_dna_pair(m=20000, n=20000, seed=12)
    exp = oracle.score(q, t, DNA_SUBMAT, 5, 2)
    got = api.align_pair(q, t, DNA_SUBMAT, 5, 2, opts=api.pair_options(1, 8, 5, 4096))
    assert got == exp


@pytest.mark.parametrize("m,n", [(1, 1), (1, 100), (100, 1), (15, 17), (257, 15), (4097, 33), (300, 5000)])
def test_ragged_shapes(api, m, n):
    rng = np.random.Generator(np.random.PCG64(m * 7 + n))
    q = rng.integers(0, 4, size=m).astype(np.uint8)
    t = rng.integers(0, 4, size=n).astype(np.uint8)
    t[: min(m, n) // 2] = q[: min(m, n) // 2]
    exp = oracle.score(q, t, DNA_SUBMAT, 5, 2)
    for opts in (None, api.pair_options(1, 8, 2)):
        assert api.align_pair(q, t, DNA_SUBMAT, 5, 2, opts=opts) == exp


def test_empty_sequences(api):
    x = np.zeros(10, dtype=np.uint8)
    assert api.align_pair(x[:0], x, DNA_SUBMAT, 5, 2) == 0
    assert api.align_pair(x, x[:0], DNA_SUBMAT, 5, 2) == 0


def test_protein_pair(api):
    # the kernel takes any 20x20 matrix: two 5,000-residue proteins with a
    # shared core, BLOSUM62, gaps 10 + 2k
    rng = np.random.Generator(np.random.PCG64(13))
    q = rng.integers(0, 20, size=5000).astype(np.uint8)
    t = rng.integers(0, 20, size=4800).astype(np.uint8)
    t[1000:3000] = q[1500:3500]
    exp = oracle.score(q, t, BLOSUM62, 10, 2)
    assert api.align_pair(q, t, BLOSUM62, 10, 2, opts=api.pair_options(4, 16, 0)) == exp
    assert api.align_pair(q, t, BLOSUM62, 10, 2) == exp


def test_identity_at_full_size(api):
    # beyond the oracle: S(X, X) = |X| with +1 matches (pinned on the oracle
    # for small X); a million-residue pair, default bands over all SMs
    x = np.random.Generator(np.random.PCG64(14)).integers(0, 4, size=1_000_000).astype(np.uint8)
    assert api.align_pair(x, x, DNA_SUBMAT, 5, 2) == 1_000_000


def test_one_substitution_at_full_size(api):
    # S = max(n - 4, p, n - 1 - p) (pinned on the oracle for small n)
    n = 300_000
    x = np.random.Generator(np.random.PCG64(15)).integers(0, 4, size=n).astype(np.uint8)
    for p in (5, 150_000, n - 3):
        y = x.copy()
        y[p] = (y[p] + 2) % 4
        assert api.align_pair(x, y, DNA_SUBMAT, 5, 2) == max(n - 4, p, n - 1 - p)


def test_invalid_arguments(api):
    from paper_2412_08308_gb300._native import SW_EINVAL, SwError

    x = np.zeros(10, dtype=np.uint8)
    bad = x.copy()
    bad[3] = 20
    for call in (lambda: api.align_pair(bad, x, DNA_SUBMAT, 5, 2),
                 lambda: api.align_pair(x, bad, DNA_SUBMAT, 5, 2),
                 lambda: api.align_pair(x, x, DNA_SUBMAT, -1, 2),
                 lambda: api.align_pair(x, x, DNA_SUBMAT, 5, 2, opts=api.pair_options(17, 0, 0)),
                 lambda: api.align_pair(x, x, DNA_SUBMAT, 5, 2, opts=api.pair_options(0, 12, 0)),
                 lambda: api.align_pair(x, x, DNA_SUBMAT, 5, 2, opts=api.pair_options(0, 0, 0, 128))):
        with pytest.raises(SwError) as e:
            call()
        assert e.value.code == SW_EINVAL


def test_score_bound(api):
    # scores must stay below 2^31 - Go: max(SM) = 63 and 35M residues could
    # reach 63 x 35M > 2^31, refused before any device work
    from paper_2412_08308_gb300._native import SW_EINVAL, SwError

    sm = np.full((20, 20), -3, dtype=np.int8)
    np.fill_diagonal(sm, 63)
    x = np.zeros(35_000_000, dtype=np.uint8)
    with pytest.raises(SwError) as e:
        api.align_pair(x, x, sm, 5, 2)
    assert e.value.code == SW_EINVAL
