"""One batch over several processes (one per GPU): host orchestration only.

Instances are independent problems (Section 6.1), so a batch splits across
ranks with no collective on the data path.  ``native.shard`` (the library's
``vsbpp_shard``) assigns each instance to a rank, longest first by item count;
``local_part`` cuts this rank's instances out as a CSR batch of their own
(input order kept), which the rank packs on its GPU; ``gather`` collects the
per-rank CSR results on rank 0 in the batch's input order, once, after the
packing (torch.distributed, any backend).  No packing arithmetic here.
"""
from __future__ import annotations

import numpy as np

from . import instances as I
from . import native


def local_part(batch: I.Batch, rank_of: np.ndarray, rank: int):
    """(sub-batch, indices into the batch) of the instances `rank` packs."""
    idx = np.nonzero(np.asarray(rank_of) == rank)[0]
    return batch.subset(idx), idx


def split(batch: I.Batch, world: int, rank: int):
    """This rank's part of the batch under the library's split."""
    rank_of, _ = native.shard(batch.w_off, world)
    return local_part(batch, rank_of, rank)


def gather(batch: I.Batch, idx: np.ndarray, local, world: int, rank: int):
    """Assemble per-rank results on rank 0.  `local` holds this rank's CSR
    results over its sub-batch (status, bin_of_item, bin_type, num_bins,
    total as numpy arrays, e.g. oracle.BatchResult or DeviceResult.to_host()
    fields).  Returns (status, bin_of_item, bin_type, num_bins, total) for the
    whole batch, CSR-aligned with batch.w_off, on rank 0; None elsewhere."""
    import torch.distributed as dist
    mine = (np.asarray(idx, dtype=np.int64), np.asarray(local.status), np.asarray(local.bin_of_item),
            np.asarray(local.bin_type), np.asarray(local.num_bins), np.asarray(local.total))
    parts = [None] * world if rank == 0 else None
    if world > 1:
        dist.gather_object(mine, parts, dst=0)
    else:
        parts = [mine]
    if rank != 0:
        return None
    N, T = batch.N, batch.total_items
    st = np.zeros(N, dtype=np.int32)
    boi = np.full(T, -1, dtype=np.int32)
    bt = np.full(T, -1, dtype=np.int32)
    nb = np.zeros(N, dtype=np.int64)
    tot = np.zeros(N, dtype=np.int64)
    seen = np.zeros(N, dtype=np.int32)
    for (ix, s_, b_, t_, n_, o_) in parts:
        a_loc = 0
        for j, i in enumerate(ix.tolist()):
            a, e = int(batch.w_off[i]), int(batch.w_off[i + 1])
            m = e - a
            st[i], nb[i], tot[i] = s_[j], n_[j], o_[j]
            boi[a:e] = b_[a_loc:a_loc + m]
            bt[a:a + int(n_[j])] = t_[a_loc:a_loc + int(n_[j])]
            a_loc += m
            seen[i] += 1
    assert np.all(seen == 1), "an instance was packed by no rank or by several"
    return st, boi, bt, nb, tot
