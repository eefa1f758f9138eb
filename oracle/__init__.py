"""CPU oracle for score-only Smith-Waterman / Gotoh (Sec. 2.2, Eqs. 1-3;
Algorithm 1) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The GPU
library never imports, links or calls it, and the two share no code.

``sw_oracle.c`` holds the scalar int32 DP (threaded across pairs only, never
inside one matrix); this module compiles it with gcc, loads it with ctypes and
exposes:

* ``score(q, d, submat, gap_open, gap_extend)``         -- one pair
* ``score_init(..., init="zero"|"neginf")``            -- boundary-init variant
* ``scores(queries, db, submat, gap_open, gap_extend)`` -- all pairs, int32 [nq, nd]
* ``align(q, d, submat, gap_open, gap_extend)``          -- one optimal alignment (traceback)

Gap convention: a run of k gap positions costs ``gap_open + k * gap_extend``.
"""

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sw_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile ``liboracle.so`` next to its source (plain gcc, -O2)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-pthread", _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        p = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int32
        lib.oracle_sw_score_init.argtypes = [p, i64, p, i64, p, i32, i32, i32]
        lib.oracle_sw_score_init.restype = i32
        lib.oracle_sw_score.argtypes = [p, i64, p, i64, p, i32, i32]
        lib.oracle_sw_score.restype = i32
        lib.oracle_sw_batch.argtypes = [p, p, i64, p, p, i64, p, i64, p, i32, i32, p, i32]
        lib.oracle_sw_batch.restype = i32
        lib.oracle_sw_align.argtypes = [p, i64, p, i64, p, i32, i32, p, p, p]
        lib.oracle_sw_align.restype = i64
        _lib = lib
    return _lib


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def _sm(submat):
    sm = np.ascontiguousarray(np.asarray(submat, dtype=np.int8))
    if sm.shape != (20, 20):
        raise ValueError("submat must be 20x20")
    return sm


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a.size else None


def score_init(q, d, submat, gap_open, gap_extend, init="zero"):
    lib = _load()
    q, d, sm = _u8(q), _u8(d), _sm(submat)
    mode = {"zero": 0, "neginf": 1}[init]
    s = lib.oracle_sw_score_init(_ptr(q), q.size, _ptr(d), d.size, _ptr(sm), int(gap_open), int(gap_extend), mode)
    if s < 0:
        raise ValueError("invalid input to oracle")
    return int(s)


def score(q, d, submat, gap_open, gap_extend):
    return score_init(q, d, submat, gap_open, gap_extend, "zero")


def align(q, d, submat, gap_open, gap_extend):
    """One optimal local alignment: (score, q_begin, q_end, t_begin, t_end, ops),
    ops a str over M (aligned pair), I (query residue against a gap), D
    (database residue against a gap); coordinates 0-based, ends exclusive."""
    lib = _load()
    q, d, sm = _u8(q), _u8(d), _sm(submat)
    sc = ctypes.c_int32(0)
    coords = np.zeros(4, dtype=np.int64)
    ops = np.zeros(max(1, q.size + d.size), dtype=np.uint8)
    k = lib.oracle_sw_align(_ptr(q), q.size, _ptr(d), d.size, _ptr(sm), int(gap_open), int(gap_extend),
                            ctypes.byref(sc), coords.ctypes.data_as(ctypes.c_void_p), _ptr(ops))
    if k < 0:
        raise ValueError("invalid input to oracle")
    return (int(sc.value), int(coords[0]), int(coords[1]), int(coords[2]), int(coords[3]),
            bytes(ops[:k]).decode())


def default_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def scores(queries, db, submat, gap_open, gap_extend, subset=None, threads=None):
    """int32 scores [n_queries, n_db] (or [n_queries, len(subset)]).

    ``queries`` and ``db`` are ``workload.Sequences``-like objects with
    ``residues`` and ``offsets`` arrays.
    """
    lib = _load()
    qres, qoff = _u8(queries.residues), np.ascontiguousarray(queries.offsets, dtype=np.int64)
    dres, doff = _u8(db.residues), np.ascontiguousarray(db.offsets, dtype=np.int64)
    sm = _sm(submat)
    nq, nd = len(qoff) - 1, len(doff) - 1
    sel = None
    ncols = nd
    if subset is not None:
        sel = np.ascontiguousarray(subset, dtype=np.int64)
        if sel.size and (sel.min() < 0 or sel.max() >= nd):
            raise ValueError("subset index out of range")
        ncols = sel.size
    out = np.zeros((nq, ncols), dtype=np.int32)
    if nq == 0 or ncols == 0:
        return out
    rc = lib.oracle_sw_batch(_ptr(qres), _ptr(qoff), nq, _ptr(dres), _ptr(doff), nd,
                             _ptr(sel) if sel is not None else None, ncols if sel is not None else 0,
                             _ptr(sm), int(gap_open), int(gap_extend), _ptr(out),
                             int(threads or default_threads()))
    if rc != 0:
        raise ValueError("invalid input to oracle")
    return out
