"""Database sharding across GPUs, one process per GPU.

Alignments of different (query, database sequence) pairs are independent
(Fig. 1, inter-sequence parallelism), so a database splits into shards that
each GPU keeps resident: every rank searches all queries against its shard
and the int32 score slices are gathered into the caller's order, the only
exchange.  Shards are length-stratified and residue-balanced: sequences are
dealt longest first in a back-and-forth order over the ranks, so each shard
gets the same mix of lengths (the work of a sequence is proportional to its
length for every query) and residue totals that differ by at most the longest
sequence.

The scores travel through ``torch.distributed`` (NCCL with device tensors, or
gloo with host tensors); every search step still runs in libswgb.so.
"""

import numpy as np


def partition(lengths, n_shards):
    """Caller-order indices of the sequences of each shard (ascending)."""
    lengths = np.asarray(lengths)
    if n_shards < 1:
        raise ValueError("n_shards must be at least 1")
    order = np.argsort(-lengths, kind="stable")
    pos = np.arange(order.size)
    rnd, r = pos // n_shards, pos % n_shards
    shard_of = np.where(rnd % 2 == 0, r, n_shards - 1 - r)
    return [np.sort(order[shard_of == k]) for k in range(n_shards)]


def subset(residues, offsets, idx):
    """(residues, offsets) of the sequences idx, in that order."""
    residues = np.asarray(residues, dtype=np.uint8)
    offsets = np.asarray(offsets, dtype=np.int64)
    idx = np.asarray(idx, dtype=np.int64)
    lens = offsets[idx + 1] - offsets[idx]
    out_off = np.zeros(idx.size + 1, dtype=np.int64)
    np.cumsum(lens, out=out_off[1:])
    if idx.size == 0:
        return np.zeros(0, dtype=np.uint8), out_off
    starts = np.repeat(offsets[idx] - out_off[:-1], lens)
    return residues[np.arange(out_off[-1]) + starts], out_off


def gather_scores(local, parts, dist, device="cpu"):
    """Assemble the [n_queries, n_db] scores from every rank's slice.

    local: this rank's int32 scores [n_queries, len(parts[rank])] (numpy);
    parts: partition(); dist: an initialised torch.distributed module.  Slices
    are padded to the largest shard for the all-gather.  Returns the full
    matrix (numpy) on every rank."""
    import torch

    nq = local.shape[0]
    width = max(len(p) for p in parts)
    buf = torch.zeros((nq, width), dtype=torch.int32, device=device)
    buf[:, :local.shape[1]] = torch.from_numpy(np.ascontiguousarray(local)).to(device)
    slices = [torch.empty_like(buf) for _ in parts]
    dist.all_gather(slices, buf)
    n = sum(len(p) for p in parts)
    full = np.empty((nq, n), dtype=np.int32)
    for k, p in enumerate(parts):
        full[:, p] = slices[k][:, :len(p)].cpu().numpy()
    return full


class ShardedDatabase:
    """This rank's shard of a database, resident on its GPU.

    residues, offsets: the whole database (host, caller order); rank, world:
    this process and the number of processes (one per GPU).  ``search`` scores
    every query against the shard and returns the full score matrix in the
    caller's order on every rank."""

    def __init__(self, residues, offsets, rank, world, stream=None):
        from .api import Database

        offsets = np.asarray(offsets, dtype=np.int64)
        self.parts = partition(np.diff(offsets), world)
        self.rank, self.world = rank, world
        self.mine = self.parts[rank]
        self.db = Database(*subset(residues, offsets, self.mine), stream=stream)

    def search(self, residues, offsets, submat, gap_open=10, gap_extend=2, mode="packed", dist=None):
        import torch

        from .api import search

        local = search(self.db, residues, offsets, submat, gap_open, gap_extend, mode)
        if self.world == 1:
            return local  # the one shard is the whole database, in caller order
        if dist is None:
            raise ValueError("a sharded search over several ranks needs torch.distributed")
        device = f"cuda:{torch.cuda.current_device()}" if dist.get_backend() == "nccl" else "cpu"
        return gather_scores(local, self.parts, dist, device)

    def close(self):
        self.db.close()
