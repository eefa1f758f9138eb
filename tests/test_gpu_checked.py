"""The checked build (-DSW_CHECK) on small parity cases.

libswgb_check.so tests every index into a packed residue buffer, a query
profile, a boundary strip or ring and the score matrix before the access; an
index outside its buffer records a device status that the host call turns
into an error (SW_ECUDA, "an index left its buffer") and the access is
skipped, without a trap.  It stands in for a memory checker.  Each case below
runs in a fresh process bound to that library and must match the CPU oracle
with no index reported: the inter-task kernel (int32, two sequences per word,
query pairs, several chunks, rescue), the intra-task kernel, the band-stream
kernel and the allocation-free entry point.
"""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import ctypes, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2412_08308_gb300 import build
import paper_2412_08308_gb300._native as N
N.use_library(build(checked=True))
import torch
from paper_2412_08308_gb300 import api
import oracle
from workload import from_list, make_workload, random_sequences
from workload.matrices import BLOSUM62
oracle.build()

def check(db_s, q_s, mode, sm=BLOSUM62, opts=None, what=""):
    db = api.Database.from_sequences(db_s)
    pq = api.PreparedQueries(db, q_s.residues, q_s.offsets, sm, 10, 2, mode, opts=opts)
    got = pq.search().cpu().numpy()
    pq.status()                     # raises on a reported index
    exp = oracle.scores(q_s, db_s, sm, 10, 2)
    assert np.array_equal(got, exp), what + " " + mode
    pq.close()
    db.close()

rng = np.random.Generator(np.random.PCG64(7))
edge = [0, 1, 15, 16, 17, 127, 128, 129]
db_s = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8)
                  for L in edge + list(rng.integers(1, 600, size=150))])
q_s = from_list([rng.integers(0, 20, size=int(L)).astype(np.uint8) for L in (0, 1, 40, 144, 300, 900)])
for mode in ("int32", "packed"):
    check(db_s, q_s, mode, opts=api.options(band_stream="never"), what="inter-task, several chunks")
    check(db_s, q_s, mode, opts=api.options(rows_per_lane=8, lanes_per_chain=5, band_stream="never"),
          what="inter-task, short chains")
    check(db_s, q_s, mode, opts=api.options(band_stream="always"), what="band-stream")
long_db = from_list(db_s.as_list()[:40] + [rng.integers(0, 20, size=L).astype(np.uint8) for L in (1000, 1500, 2100)])
for mode in ("int32", "packed"):
    check(long_db, q_s, mode, opts=api.options(cutover=1000, band_stream="never"), what="intra-task")
    check(long_db, q_s, mode, opts=api.options(cutover=1000, band_stream="always", band_rows=16),
          what="band-stream, long units")
# query pairs (12 queries of similar lengths) and the rescue of saturated pairs
qq = from_list([rng.integers(0, 20, size=L).astype(np.uint8) for L in (300, 290, 281, 250, 100, 96, 55, 17, 16, 0)])
check(db_s, qq, "packed", opts=api.options(band_stream="never"), what="query pairs")
sm = np.full((20, 20), -5, dtype=np.int8)
np.fill_diagonal(sm, 60)
base = rng.integers(0, 20, size=700).astype(np.uint8)
sat_db = from_list(db_s.as_list()[:60] + [base, base[:650].copy()])
check(sat_db, from_list([base, base[:100].copy()]), "packed", sm=sm, opts=api.options(band_stream="never"),
      what="rescue")
# the allocation-free entry point
db = api.Database.from_sequences(long_db)
out = torch.full((len(long_db),), -1, dtype=torch.int32, device="cuda")
q = np.ascontiguousarray(q_s[4])
smc = np.ascontiguousarray(BLOSUM62)
N.sw_search_noalloc(db.handle, ctypes.c_void_p(q.ctypes.data), q.size, ctypes.c_void_p(smc.ctypes.data), 10, 2,
                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
assert np.array_equal(out.cpu().numpy(), oracle.scores(from_list([q]), long_db, BLOSUM62, 10, 2)[0]), "noalloc"
db.close()
print("checked build: all cases exact, no index reported")
'''


def test_checked_build_small_parity():
    env = dict(os.environ)
    r = subprocess.run([sys.executable, "-c", SCRIPT.replace("ROOT", repr(ROOT), 1)], capture_output=True,
                       text=True, timeout=1800, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "no index reported" in r.stdout
