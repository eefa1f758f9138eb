"""Python front-end over the C-ABI: numpy arrays for host data, torch tensors
for device memory and streams.  Marshalling only; every step of the search
runs in libswgb.so."""

import ctypes

import numpy as np

from . import _native as N

MODES = {"int32": N.SW_MODE_INT32, "packed": N.SW_MODE_PACKED}


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a.size else None


def _stream(stream):
    import torch

    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _seqs(residues, offsets):
    res = np.ascontiguousarray(residues, dtype=np.uint8)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    if off.ndim != 1 or off.size < 1:
        raise ValueError("offsets must be a 1-D array with n+1 entries")
    return res, off


def _mode(mode):
    if isinstance(mode, str):
        return MODES[mode]
    return int(mode)


class Database:
    """A protein database packed and resident on the current CUDA device."""

    def __init__(self, residues, offsets, stream=None):
        res, off = _seqs(residues, offsets)
        self.n = off.size - 1
        self.lengths = np.diff(off)
        self.handle = N.sw_db_prepare(_ptr(res), _ptr(off), self.n, _stream(stream))

    @classmethod
    def from_sequences(cls, seqs, stream=None):
        return cls(seqs.residues, seqs.offsets, stream)

    def stats(self):
        return N.sw_db_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.sw_db_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BAND_STREAM = {"auto": 0, "never": 1, "always": 2}


def options(cutover=0, rows_per_lane=0, lanes_per_chain=0, intra_rows=0, query_pairs=True, band_stream="auto",
            band_rows=0):
    """Tuning knobs of a query batch (sw_options); 0 keeps the default.
    query_pairs=False keeps every packed query in the two-sequences-per-chain form;
    band_stream: "auto" (batches too small to fill the GPU), "never" or "always";
    band_rows: rows per lane of the band-stream kernel (8 or 16; 0 = 16)."""
    return N.SwOptions(int(cutover), int(rows_per_lane), int(lanes_per_chain), int(intra_rows),
                       0 if query_pairs else 1, BAND_STREAM[band_stream], int(band_rows))


class PreparedQueries:
    """A query batch uploaded and planned against one Database; search() is
    device-only and asynchronous (graph-capturable)."""

    def __init__(self, db, residues, offsets, submat, gap_open=10, gap_extend=2, mode="packed", opts=None,
                 stream=None):
        res, off = _seqs(residues, offsets)
        sm = np.ascontiguousarray(submat, dtype=np.int8)
        if sm.shape != (20, 20):
            raise ValueError("submat must be 20x20")
        self.db = db
        self.nq = off.size - 1
        self.handle = N.sw_queries_prepare(db.handle, _ptr(res), _ptr(off), self.nq, _ptr(sm), int(gap_open),
                                           int(gap_extend), _mode(mode), opts, _stream(stream))

    def search(self, out=None, stream=None):
        import torch

        if out is None:
            out = torch.empty((self.nq, self.db.n), dtype=torch.int32, device="cuda")
        if not (out.is_cuda and out.dtype == torch.int32 and out.is_contiguous() and out.numel() == self.nq * self.db.n):
            raise ValueError("out must be a contiguous int32 CUDA tensor of n_queries * n_db elements")
        N.sw_search_prepared(self.db.handle, self.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream))
        return out

    def search_graph(self, out=None, stream=None):
        """search() through a CUDA graph captured on the first call (needs a
        non-default stream; pass a torch.cuda.Stream or run under one)."""
        import torch

        if out is None:
            out = torch.empty((self.nq, self.db.n), dtype=torch.int32, device="cuda")
        if not (out.is_cuda and out.dtype == torch.int32 and out.is_contiguous() and out.numel() == self.nq * self.db.n):
            raise ValueError("out must be a contiguous int32 CUDA tensor of n_queries * n_db elements")
        N.sw_search_graph(self.db.handle, self.handle, ctypes.c_void_p(out.data_ptr()), _stream(stream))
        return out

    def set_timing(self, enable=True):
        N.sw_queries_set_timing(self.handle, enable)

    def kernel_ms(self, stream=None):
        """Duration (ms) of the main DP kernel in the last timed search."""
        return N.sw_queries_kernel_ms(self.handle, _stream(stream))

    def info(self):
        """(host->device bytes copied at prepare, device bytes held, DP tasks,
        kernel launches per search)."""
        return N.sw_queries_info(self.handle)

    def status(self, stream=None):
        """Synchronise; return the number of rescued (query, sequence) pairs."""
        return N.sw_queries_status(self.handle, _stream(stream))

    def close(self):
        if getattr(self, "handle", None) is not None:
            N.sw_queries_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def search(db, residues, offsets, submat, gap_open=10, gap_extend=2, mode="packed", out=None, stream=None):
    """One-call search through ``sw_search``.  Returns int32 scores
    [n_queries, n_db] in caller order: a numpy array by default, or ``out``
    (a numpy array or a CUDA int32 tensor) when given."""
    res, off = _seqs(residues, offsets)
    sm = np.ascontiguousarray(submat, dtype=np.int8)
    nq = off.size - 1
    if out is None:
        out = np.empty((nq, db.n), dtype=np.int32)
    if isinstance(out, np.ndarray):
        if out.dtype != np.int32 or not out.flags.c_contiguous or out.size != nq * db.n:
            raise ValueError("out must be a contiguous int32 array of n_queries * n_db elements")
        optr = _ptr(out)
    else:
        optr = ctypes.c_void_p(out.data_ptr())
    N.sw_search(db.handle, _ptr(res), _ptr(off), nq, _ptr(sm), int(gap_open), int(gap_extend), _mode(mode), optr,
                _stream(stream))
    return out


def pair_options(band_warps=0, rows_per_lane=0, max_ctas=0, ring_columns=0):
    """Knobs of sw_align_pair (sw_pair_options); 0 keeps the default."""
    return N.SwPairOptions(int(band_warps), int(rows_per_lane), int(max_ctas), int(ring_columns))


def align_pair(query, target, submat, gap_open=5, gap_extend=2, opts=None, stream=None, timed=False):
    """Score-only local alignment of two long sequences (residue codes 0..19) on
    the band-pipeline kernel; returns the score, or (score, kernel ms) if timed."""
    q = np.ascontiguousarray(query, dtype=np.uint8)
    t = np.ascontiguousarray(target, dtype=np.uint8)
    sm = np.ascontiguousarray(submat, dtype=np.int8)
    if sm.shape != (20, 20):
        raise ValueError("submat must be 20x20")
    score, ms = N.sw_align_pair(_ptr(q), q.size, _ptr(t), t.size, _ptr(sm), int(gap_open), int(gap_extend), opts,
                                _stream(stream))
    return (score, ms) if timed else score


def traceback(db, residues, offsets, hits, submat, gap_open=10, gap_extend=2, stream=None):
    """One optimal local alignment for each hit (query index, database index
    in the caller's order): a list of (score, q_begin, q_end, t_begin, t_end,
    ops) with ops a str over M (aligned pair), I (query residue against a gap)
    and D (database residue against a gap); coordinates 0-based, ends exclusive."""
    res, off = _seqs(residues, offsets)
    sm = np.ascontiguousarray(submat, dtype=np.int8)
    if sm.shape != (20, 20):
        raise ValueError("submat must be 20x20")
    hits = [(int(a), int(b)) for a, b in hits]
    arr = (N.SwHit * len(hits))(*[N.SwHit(a, b) for a, b in hits])
    qlen = np.diff(off)
    need = sum(int(qlen[a]) if 0 <= a < qlen.size else 0 for a, _ in hits) + sum(
        int(db.lengths[b]) if 0 <= b < len(db.lengths) else 0 for _, b in hits)
    ops = np.zeros(max(need, 1), dtype=np.uint8)
    out = N.sw_traceback(db.handle, _ptr(res), _ptr(off), off.size - 1, arr, _ptr(sm), int(gap_open),
                         int(gap_extend), ops, _stream(stream))
    result = []
    for o in out:
        seg = bytes(ops[o.ops_offset:o.ops_offset + o.n_ops]).decode()
        result.append((o.score, o.q_begin, o.q_end, o.t_begin, o.t_end, seg))
    return result

