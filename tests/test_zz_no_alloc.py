"""sw_search_noalloc: the allocation-free single-query entry point.

Callers that cannot allocate device memory while they search (a fixed memory
budget, a real-time loop where an allocation may stall the device, an arena
the caller does not control) use this entry point; its scratch is a static
device array inside the library.  Its scores must equal those of the regular
entry point (sw_search) exactly, call after call, although every call reuses
the same scratch.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from workload import random_sequences
from workload.matrices import BLOSUM62

pytestmark = pytest.mark.gpu


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def test_noalloc_matches_regular_entry_point_twice():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2412_08308_gb300 import api, build
    from paper_2412_08308_gb300 import _native as N

    build()
    db_s = random_sequences(91, 5000, 300, 0.5, 1, 1000)
    qs = random_sequences(92, 3, 400, 0.5, 30, 768)
    db = api.Database.from_sequences(db_s)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    sm = np.ascontiguousarray(BLOSUM62)
    out = torch.full((len(db_s),), -1, dtype=torch.int32, device="cuda")
    for i in (0, 1, 2, 0):  # calls in a row, different query lengths, then the first again
        q = np.ascontiguousarray(qs[i])
        expected = api.search(db, q, np.array([0, len(q)], dtype=np.int64), sm, 10, 2, "int32")[0]
        out.fill_(-1)
        N.sw_search_noalloc(db.handle, _ptr(q), len(q), _ptr(sm), 10, 2, ctypes.c_void_p(out.data_ptr()), stream)
        np.testing.assert_array_equal(out.cpu().numpy(), expected)
    # sizes beyond the stated maximum are rejected, not truncated
    long_q = np.zeros(769, dtype=np.uint8)
    with pytest.raises(N.SwError) as e:
        N.sw_search_noalloc(db.handle, _ptr(long_q), 769, _ptr(sm), 10, 2, ctypes.c_void_p(out.data_ptr()), stream)
    assert e.value.code == N.SW_EINVAL and "768" in str(e.value)
    db.close()
