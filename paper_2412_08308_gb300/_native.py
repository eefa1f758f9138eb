"""ctypes binding of the C-ABI in include/swgb.h (argument marshalling only).

Every function here has the name of the C entry point it wraps and forwards
plain pointers and sizes; all work happens in libswgb.so.  There is no
fallback: if the library is missing, importing the binding raises.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libswgb.so")

SW_OK, SW_EINVAL, SW_ENOMEM, SW_ECUDA, SW_ETIMEOUT = 0, 1, 2, 3, 4
SW_MODE_INT32, SW_MODE_PACKED = 0, 1

# every symbol include/swgb.h declares, with (restype, argtypes)
_p, _i64, _i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
_pp = ctypes.POINTER(ctypes.c_void_p)
_pi64 = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = {
    "sw_db_prepare": (ctypes.c_int, [_p, _p, _i64, _p, _pp]),
    "sw_db_free": (ctypes.c_int, [_p]),
    "sw_db_stats": (ctypes.c_int, [_p, _pi64, _pi64, _pi64]),
    "sw_queries_prepare": (ctypes.c_int, [_p, _p, _p, _i64, _p, _i32, _i32, _i32, _p, _p, _pp]),
    "sw_queries_free": (ctypes.c_int, [_p]),
    "sw_search_prepared": (ctypes.c_int, [_p, _p, _p, _p]),
    "sw_queries_status": (ctypes.c_int, [_p, _p, _pi64]),
    "sw_search_graph": (ctypes.c_int, [_p, _p, _p, _p]),
    "sw_search": (ctypes.c_int, [_p, _p, _p, _i64, _p, _i32, _i32, _i32, _p, _p]),
    "sw_queries_set_timing": (ctypes.c_int, [_p, _i32]),
    "sw_queries_kernel_ms": (ctypes.c_int, [_p, _p, ctypes.POINTER(ctypes.c_float)]),
    "sw_queries_info": (ctypes.c_int, [_p, _pi64, _pi64, _pi64, _pi64]),
    "sw_search_noalloc": (ctypes.c_int, [_p, _p, _i64, _p, _i32, _i32, _p, _p]),
    "sw_align_pair": (ctypes.c_int, [_p, _i64, _p, _i64, _p, _i32, _i32, _p, _p, _p, _p]),
    "sw_traceback": (ctypes.c_int, [_p, _p, _p, _i64, _p, _i64, _p, _i32, _i32, _p, _p, _i64, _p]),
    "sw_selftest_wait": (ctypes.c_int, [_i32, _i64, ctypes.POINTER(ctypes.c_int32), _p]),
    "sw_last_error": (ctypes.c_char_p, []),
}


class SwOptions(ctypes.Structure):
    """Mirror of sw_options (include/swgb.h); zero fields take defaults."""

    _fields_ = [("cutover", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32), ("lanes_per_chain", ctypes.c_int32),
                ("intra_rows", ctypes.c_int32), ("query_pairs", ctypes.c_int32), ("band_stream", ctypes.c_int32),
                ("band_rows", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


class SwError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"swgb error {code}: {msg}")
        self.code = code


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built; run paper_2412_08308_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def use_library(path):
    """Bind every entry point of this module to the library at `path` (the
    checked build libswgb_check.so, say) instead of libswgb.so.  Must come
    before the first call in the process."""
    global _lib
    if _lib is not None:
        raise RuntimeError("the library is already loaded in this process")
    _lib = load(path)


def check(rc):
    if rc != SW_OK:
        raise SwError(rc, lib().sw_last_error().decode())
    return rc


def sw_last_error():
    return lib().sw_last_error().decode()


def sw_db_prepare(residues_ptr, offsets_ptr, n_seqs, stream):
    h = ctypes.c_void_p()
    check(lib().sw_db_prepare(residues_ptr, offsets_ptr, n_seqs, stream, ctypes.byref(h)))
    return h


def sw_db_free(h):
    return check(lib().sw_db_free(h))


def sw_db_stats(h):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().sw_db_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sw_queries_prepare(db, q_ptr, qoff_ptr, n_queries, submat_ptr, gap_open, gap_extend, mode, opts, stream):
    """opts: an SwOptions or None for defaults."""
    h = ctypes.c_void_p()
    check(lib().sw_queries_prepare(db, q_ptr, qoff_ptr, n_queries, submat_ptr, gap_open, gap_extend, mode,
                                   ctypes.byref(opts) if opts is not None else None, stream, ctypes.byref(h)))
    return h


def sw_queries_free(h):
    return check(lib().sw_queries_free(h))


def sw_search_prepared(db, qh, scores_dev_ptr, stream):
    return check(lib().sw_search_prepared(db, qh, scores_dev_ptr, stream))


def sw_queries_status(qh, stream):
    r = ctypes.c_int64()
    check(lib().sw_queries_status(qh, stream, ctypes.byref(r)))
    return r.value


def sw_search(db, q_ptr, qoff_ptr, n_queries, submat_ptr, gap_open, gap_extend, mode, scores_ptr, stream):
    return check(lib().sw_search(db, q_ptr, qoff_ptr, n_queries, submat_ptr, gap_open, gap_extend, mode,
                                 scores_ptr, stream))


def sw_queries_set_timing(qh, enable):
    return check(lib().sw_queries_set_timing(qh, int(enable)))


def sw_queries_kernel_ms(qh, stream):
    v = ctypes.c_float()
    check(lib().sw_queries_kernel_ms(qh, stream, ctypes.byref(v)))
    return v.value


def sw_queries_info(qh):
    a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    check(lib().sw_queries_info(qh, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return a.value, b.value, c.value, d.value


def sw_search_graph(db, qh, scores_dev_ptr, stream):
    return check(lib().sw_search_graph(db, qh, scores_dev_ptr, stream))


def sw_search_noalloc(db, q_ptr, m, submat_ptr, gap_open, gap_extend, scores_dev_ptr, stream):
    return check(lib().sw_search_noalloc(db, q_ptr, m, submat_ptr, gap_open, gap_extend, scores_dev_ptr, stream))


class SwPairOptions(ctypes.Structure):
    """Mirror of sw_pair_options (include/swgb.h); zero fields take defaults."""

    _fields_ = [("band_warps", ctypes.c_int32), ("rows_per_lane", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("ring_columns", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


def sw_align_pair(q_ptr, m, t_ptr, n, submat_ptr, gap_open, gap_extend, opts, stream):
    """Returns (score, band kernel milliseconds)."""
    score = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    check(lib().sw_align_pair(q_ptr, m, t_ptr, n, submat_ptr, gap_open, gap_extend,
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(score),
                              ctypes.byref(ms), stream))
    return score.value, ms.value


class SwHit(ctypes.Structure):
    """Mirror of sw_hit (include/swgb.h)."""

    _fields_ = [("query", ctypes.c_int32), ("target", ctypes.c_int32)]


class SwAlignment(ctypes.Structure):
    """Mirror of sw_alignment (include/swgb.h)."""

    _fields_ = [("score", ctypes.c_int32), ("q_begin", ctypes.c_int32), ("q_end", ctypes.c_int32),
                ("t_begin", ctypes.c_int32), ("t_end", ctypes.c_int32), ("n_ops", ctypes.c_int32),
                ("ops_offset", ctypes.c_int64)]


def sw_traceback(db, q_ptr, qoff_ptr, n_queries, hits, submat_ptr, gap_open, gap_extend, ops_buf, stream):
    """hits: a ctypes array of SwHit; ops_buf: a writable numpy uint8 array.  Returns the SwAlignment array."""
    out = (SwAlignment * len(hits))()
    check(lib().sw_traceback(db, q_ptr, qoff_ptr, n_queries, hits, len(hits), submat_ptr, gap_open, gap_extend,
                             out, ops_buf.ctypes.data_as(ctypes.c_void_p) if ops_buf.size else None, ops_buf.size,
                             stream))
    return out


def sw_selftest_wait(which, budget_cycles, stream):
    st = ctypes.c_int32(-1)
    check(lib().sw_selftest_wait(int(which), int(budget_cycles), ctypes.byref(st), stream))
    return st.value
