"""Failure detection without a GPU fault: the bounded device waits give up on
a condition that nothing fulfils, report SW_ETIMEOUT, and the context stays
usable for the next search."""

import time

import numpy as np
import pytest

import oracle
from workload import random_sequences
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


def test_bounded_waits_give_up_and_the_context_stays_usable(api):
    import ctypes

    import torch

    from paper_2412_08308_gb300 import _native as N

    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a counter nothing raises: ~1 ms of clock cycles, then SW_ETIMEOUT
    assert N.sw_selftest_wait(0, 2_000_000, s) == N.SW_ETIMEOUT
    # an mbarrier phase nothing completes, with the kernels' own ~1 s budget
    t0 = time.perf_counter()
    assert N.sw_selftest_wait(1, 0, s) == N.SW_ETIMEOUT
    assert time.perf_counter() - t0 < 30
    # the same process searches on
    db_s = random_sequences(81, 200, 300, 0.5, 20, 600)
    q = random_sequences(82, 3, 200, 0.5, 30, 400)
    db = api.Database.from_sequences(db_s)
    got = api.search(db, q.residues, q.offsets, BLOSUM62, 10, 2, "packed")
    db.close()
    np.testing.assert_array_equal(got, oracle.scores(q, db_s, BLOSUM62, 10, 2))


def test_invalid_selftest_arguments(api):
    import ctypes

    from paper_2412_08308_gb300 import _native as N

    for which, budget in ((2, 1000), (0, 0), (0, 1 << 33)):
        with pytest.raises(N.SwError) as e:
            N.sw_selftest_wait(which, budget, ctypes.c_void_p(0))
        assert e.value.code == N.SW_EINVAL
