"""sw_search_noalloc: the allocation-free single-query entry point.

Callers that cannot allocate device memory while they search (a service that
fixes its memory budget at start-up, a real-time loop in which a cudaMalloc
may synchronise the device and stall every stream, a host that runs the
library inside an arena it does not control) use this entry point; its
scratch is a static device array inside the library.  Its scores must equal
the CPU oracle's and those of the regular entry point (sw_search) exactly,
call after call, although every call reuses the same scratch.

The queries cover both plans of the entry point (16 rows per lane up to 512
residues, 24 rows above, as its header states): the empty query, 1 residue,
512 and 513 residues (the two sides of the switch), 700 and the maximum, 768
(32 lanes x 24 rows: the profile chunk then fills its whole slot of the
scratch).  The database holds empty, one-residue and padding-edge sequences
and sequences beyond the regular path's inter/intra-task cutover of 2,048
residues (the regular path runs them in the intra-task kernel, this entry
point in the inter-task kernel).  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

import oracle
from workload import from_list, random_sequences
from workload.matrices import BLOSUM62

pytestmark = pytest.mark.gpu


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _database():
    rng = np.random.Generator(np.random.PCG64(93))
    base = random_sequences(91, 2500, 300, 0.5, 1, 1000).as_list()
    extra = [rng.integers(0, 20, size=L).astype(np.uint8) for L in (0, 1, 15, 16, 17, 2049, 2600, 4100)]
    seqs = base + extra
    order = rng.permutation(len(seqs))
    return from_list([seqs[i] for i in order])


def _queries():
    rng = np.random.Generator(np.random.PCG64(92))
    lens = [0, 1, 118, 512, 513, 700, 768]
    return from_list([rng.integers(0, 20, size=L).astype(np.uint8) for L in lens])


def test_noalloc_matches_oracle_and_regular_entry_point():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_08308_gb300 import _native as N
    from paper_2412_08308_gb300 import api, build

    build()
    oracle.build()
    db_s = _database()
    qs = _queries()
    assert max(db_s.lengths) > 2048
    exp = oracle.scores(qs, db_s, BLOSUM62, 10, 2)
    db = api.Database.from_sequences(db_s)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sm = np.ascontiguousarray(BLOSUM62)
    out = torch.full((len(db_s),), -1, dtype=torch.int32, device="cuda")
    # calls in a row with different plans, then the largest and the first again
    for i in (3, 4, 6, 0, 5, 1, 2, 6, 3):
        q = np.ascontiguousarray(qs[i])
        regular = api.search(db, q, np.array([0, len(q)], dtype=np.int64), sm, 10, 2, "int32")[0]
        out.fill_(-1)
        N.sw_search_noalloc(db.handle, _ptr(q), len(q), _ptr(sm), 10, 2, ctypes.c_void_p(out.data_ptr()), stream)
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, exp[i], err_msg=f"query of {len(q)} residues vs the oracle")
        np.testing.assert_array_equal(got, regular, err_msg=f"query of {len(q)} residues vs sw_search")
    assert exp[qs.lengths == 0].max() == 0 and exp.max() > 0
    # sizes beyond the stated maximum are rejected, not truncated
    long_q = np.zeros(769, dtype=np.uint8)
    with pytest.raises(N.SwError) as e:
        N.sw_search_noalloc(db.handle, _ptr(long_q), 769, _ptr(sm), 10, 2, ctypes.c_void_p(out.data_ptr()), stream)
    assert e.value.code == N.SW_EINVAL and "768" in str(e.value)
    db.close()
