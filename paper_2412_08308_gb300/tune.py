"""Autotuner for the search plan.

Sweeps the tuning knobs of sw_options -- query rows per lane of the
inter-task kernel (the residues each thread holds) and the length cutover
between the inter-task and the intra-task kernels (SW# likewise splits database
sequences between a short and a long kernel by length, Sec. 3.1) -- on the real
query batch, timing each point with CUDA events around graph launches of the
whole search, and returns the fastest options.  Results are cached in a JSON
file keyed by the GPU name and fingerprints of the database and the batch.
"""

import hashlib
import json
import os

import numpy as np

from . import api

ROWS = (4, 8, 16, 24)
CUTOVERS = (512, 1024, 2048, 4096)


def _fingerprint(lengths):
    L = np.asarray(lengths, dtype=np.int64)
    if L.size == 0:
        return "empty"
    q = np.percentile(L, [0, 10, 50, 90, 99, 100]).astype(np.int64).tolist()
    h = hashlib.sha1(np.sort(L).tobytes()).hexdigest()[:12]
    return f"n{L.size}-s{int(L.sum())}-q{'-'.join(map(str, q))}-{h}"


def cache_key(gpu_name, db_lengths, q_lengths, mode, gap_open, gap_extend):
    return "|".join([gpu_name, _fingerprint(db_lengths), _fingerprint(q_lengths), str(mode),
                     f"{gap_open}/{gap_extend}"])


def tune(db, db_lengths, residues, offsets, submat, gap_open=10, gap_extend=2, mode="packed", rows=ROWS,
         cutovers=CUTOVERS, reps=2, cache_path=None):
    """Return (best sw_options, table of (rows, cutover, GCUPS)) for this batch.

    ``db`` is an api.Database, ``db_lengths`` its sequence lengths (host),
    ``residues`` / ``offsets`` the query batch.
    """
    import torch

    offsets = np.asarray(offsets, dtype=np.int64)
    q_lengths = np.diff(offsets)
    key = cache_key(torch.cuda.get_device_name(), db_lengths, q_lengths, mode, gap_open, gap_extend)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except ValueError:
            cache = {}
    if key in cache:
        c = cache[key]
        return api.options(cutover=c["cutover"], rows_per_lane=c["rows_per_lane"]), c["table"]

    cells = float(offsets[-1]) * float(np.sum(db_lengths))
    stream = torch.cuda.Stream()
    out = torch.empty((len(q_lengths), db.n), dtype=torch.int32, device="cuda")
    table = []
    best = None
    with torch.cuda.stream(stream):
        for r in rows:
            for c in cutovers:
                opts = api.options(cutover=c, rows_per_lane=r)
                pq = api.PreparedQueries(db, residues, offsets, submat, gap_open, gap_extend, mode, opts=opts,
                                         stream=stream)
                pq.search_graph(out, stream=stream)  # capture + first run
                stream.synchronize()
                ts = []
                for _ in range(reps):
                    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    s.record(stream)
                    pq.search_graph(out, stream=stream)
                    e.record(stream)
                    e.synchronize()
                    ts.append(s.elapsed_time(e) / 1e3)
                pq.status(stream=stream)
                pq.close()
                g = cells / min(ts) / 1e9
                table.append((r, c, round(g, 1)))
                if best is None or g > best[2]:
                    best = (r, c, g)
    if cache_path:
        cache[key] = {"rows_per_lane": best[0], "cutover": best[1], "table": table}
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return api.options(cutover=best[1], rows_per_lane=best[0]), table
