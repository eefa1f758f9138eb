"""The oracle's pins must catch plausible mistakes.

Each mutant below is the oracle's C source with one deliberate error (a wrong
penalty, a dropped term, a wrong neighbour, a transposed lookup, ...).  The
mutant is compiled into a temporary library on the CPU and run through a
subset of the pins of test_oracle_pins.py; every mutant must fail at least one.
"""

import ctypes
import json
import os
import subprocess

import numpy as np
import pytest

from tests import _pins
from workload import encode
from workload.matrices import BLOSUM62

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "sw_oracle.c")

MUTANTS = {
    "E extends with Go": ("int32_t E1 = El - Ge;", "int32_t E1 = El - Go;"),
    "E opens with Ge": ("int32_t E2 = Hl - Go;", "int32_t E2 = Hl - Ge;"),
    "F extends with Go": ("int32_t F1 = Fup[j] - Ge;", "int32_t F1 = Fup[j] - Go;"),
    "diagonal taken from above": ("int32_t H = Hul + row[D[j - 1]];", "int32_t H = Hup[j] + row[D[j - 1]];"),
    "E term dropped": ("H = max2(H, E);", ";"),
    "F term dropped": ("H = max2(H, F);", ";"),
    "zero floor dropped": ("H = max2(H, 0);", ";"),
    "gap open convention": ("const int32_t Go = gap_open + gap_extend;", "const int32_t Go = gap_open;"),
    "score is last cell": ("S = max2(H, S);", "S = H;"),
    "substitution transposed": ("int32_t H = Hul + row[D[j - 1]];",
                                "int32_t H = Hul + SM[(size_t)D[j - 1] * ORACLE_ALPHABET + Q[i - 1]];"),
    "E carried from above": ("El = E;", "El = Fup[j];"),
}

# mistakes in the traceback walk (one optimal alignment): caught by the
# alignment pins (the score recomputed from the operations, the coordinates)
TRACEBACK_MUTANTS = {
    "walk opens E with Ge": ("state = (E[c] == H[c - 1] - Go) ? 0 : 1;", "state = (E[c] == H[c - 1] - Ge) ? 0 : 1;"),
    "walk opens F from the left": ("state = (F[c] == H[c - W] - Go) ? 0 : 2;",
                                   "state = (F[c] == H[c - 1] - Go) ? 0 : 2;"),
    "walk swaps I and D": ("ops[k++] = 'D';", "ops[k++] = 'I';"),
    "walk ignores E": ("} else if (H[c] == E[c]) {", "} else if (0) {"),
    "walk drops the substitution": ("if (H[c] == H[c - W - 1] + SM[(size_t)Q[i - 1] * ORACLE_ALPHABET + D[j - 1]]) {",
                                    "if (H[c] == H[c - W - 1]) {"),
}

_ALIGN_MARK = "/* ---- one optimal local alignment"


def _build_mutant(tmp_path, name, old, new, in_align=False):
    """Compile the oracle with `old` replaced by `new` in the score functions
    (the text before the traceback function) or, in_align, in the traceback."""
    src = open(SRC).read()
    cut = src.index(_ALIGN_MARK)
    head, tail = src[:cut], src[cut:]
    part = tail if in_align else head
    assert part.count(old) == 1, f"mutation anchor not unique: {old}"
    part = part.replace(old, new)
    path = tmp_path / "mut.c"
    path.write_text(head + part if in_align else part + tail)
    lib = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-pthread", str(path), "-o", str(lib)])
    L = ctypes.CDLL(str(lib))
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    L.oracle_sw_score.argtypes = [p, i64, p, i64, p, i32, i32]
    L.oracle_sw_score.restype = i32
    L.oracle_sw_align.argtypes = [p, i64, p, i64, p, i32, i32, p, p, p]
    L.oracle_sw_align.restype = i64

    def score(q, d, sm, go, ge):
        q = np.ascontiguousarray(q, dtype=np.uint8)
        d = np.ascontiguousarray(d, dtype=np.uint8)
        sm = np.ascontiguousarray(sm, dtype=np.int8)
        return int(L.oracle_sw_score(q.ctypes.data_as(p) if q.size else None, q.size,
                                     d.ctypes.data_as(p) if d.size else None, d.size,
                                     sm.ctypes.data_as(p), go, ge))

    def align(q, d, sm, go, ge):
        q = np.ascontiguousarray(q, dtype=np.uint8)
        d = np.ascontiguousarray(d, dtype=np.uint8)
        sm = np.ascontiguousarray(sm, dtype=np.int8)
        sc = ctypes.c_int32(0)
        coords = np.zeros(4, dtype=np.int64)
        ops = np.zeros(max(1, q.size + d.size), dtype=np.uint8)
        k = L.oracle_sw_align(q.ctypes.data_as(p) if q.size else None, q.size,
                              d.ctypes.data_as(p) if d.size else None, d.size, sm.ctypes.data_as(p), go, ge,
                              ctypes.byref(sc), coords.ctypes.data_as(p), ops.ctypes.data_as(p))
        return int(sc.value), [int(c) for c in coords], bytes(ops[:k]).decode()

    return (align if in_align else score)


def _pins_fail(score):
    """True as soon as one pin disagrees with ``score``."""
    rng = np.random.Generator(np.random.PCG64(5))
    asym = rng.integers(-6, 9, size=(20, 20)).astype(np.int8)
    for k in range(30):
        q = rng.integers(0, 20, size=int(rng.integers(1, 7))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(1, 7))).astype(np.uint8)
        for sm in (BLOSUM62, asym):
            for go, ge in ((10, 2), (3, 1), (0, 4)):
                if score(q, d, sm, go, ge) != _pins.brute_force(q, d, sm, go, ge):
                    return True
    sm = np.full((20, 20), -30, dtype=np.int8)
    np.fill_diagonal(sm, 10)
    with open(os.path.join(HERE, "golden", "gap_cost_cases.json")) as f:
        for case in json.load(f)["cases"]:
            if score(encode(case["q"]), encode(case["d"]), sm, case["gap_open"], case["gap_extend"]) != case["expected"]:
                return True
    q = rng.integers(0, 20, size=50).astype(np.uint8)
    if score(q, q, BLOSUM62, 10, 2) != int(sum(int(BLOSUM62[c, c]) for c in q)):
        return True
    return False


def test_unmutated_source_passes(tmp_path):
    score = _build_mutant(tmp_path, "none", "S = max2(H, S);", "S = max2(H, S);")
    assert not _pins_fail(score)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    score = _build_mutant(tmp_path, name, old, new)
    assert _pins_fail(score), f"pins did not catch mutant: {name}"


def _alignment_pins_fail(align):
    """True as soon as an alignment disagrees with its own score, coordinates
    or local ends (the pins of test_oracle_pins.py)."""
    rng = np.random.Generator(np.random.PCG64(6))
    for k in range(60):
        q = rng.integers(0, 20, size=int(rng.integers(1, 30))).astype(np.uint8)
        d = rng.integers(0, 20, size=int(rng.integers(1, 30))).astype(np.uint8)
        if k % 2 and len(q) > 6:
            d = np.concatenate([d[:4], q[1:4], d[4:7], q[4:-1], d[7:]]).astype(np.uint8)
        for go, ge in ((10, 2), (3, 1), (0, 4)):
            s, (qb, qe, tb, te), ops = align(q, d, BLOSUM62, go, ge)
            try:
                total, i, j = _pins.alignment_score(q, d, BLOSUM62, go, ge, qb, tb, ops)
            except (ValueError, IndexError):
                return True
            if total != s or (i, j) != (qe, te) or (s > 0 and (ops[:1] != "M" or ops[-1:] != "M")):
                return True
    return False


def test_unmutated_traceback_passes(tmp_path):
    old = "ops[k++] = 'M';"
    align = _build_mutant(tmp_path, "none", old, old, in_align=True)
    assert not _alignment_pins_fail(align)


@pytest.mark.parametrize("name", sorted(TRACEBACK_MUTANTS))
def test_traceback_mutant_is_caught(tmp_path, name):
    old, new = TRACEBACK_MUTANTS[name]
    align = _build_mutant(tmp_path, name, old, new, in_align=True)
    assert _alignment_pins_fail(align), f"alignment pins did not catch mutant: {name}"
