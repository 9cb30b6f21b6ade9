"""Helpers for the GPU parity tests: run the CUDA path and the oracle on the
same seeded batch and compare element by element."""
import numpy as np

import oracle
from paper_1602_08735_gb300 import native


def run_batch(batch, heuristic=1, criterion=1, sublist_size=0, preopen=0, seed=0, plain=False,
              max_m=None, flags=0, max_open=0):
    import torch
    db = native.DeviceBatch.from_host(batch)
    out = native.DeviceResult.empty(db.N, db.total_items)
    fn = native.pack_plain if plain else native.pack_batch
    rc = fn(db, out, heuristic, criterion, sublist_size, preopen, seed, max_m=max_m, flags=flags,
            max_open=max_open)
    assert rc == 0, native.strerror(rc)
    torch.cuda.synchronize()
    st, boi, bt, nb, tot = out.to_host(db.N, db.total_items)
    return oracle.BatchResult(st, boi, bt, nb, tot)


def run_oracle(batch, heuristic=1, criterion=1, sublist_size=0, preopen=0, seed=0, flags=0, max_open=0):
    return oracle.pack_many(batch.w_all, batch.w_off, batch.B_all, batch.B_off, heuristic, criterion,
                            sublist_size, preopen, seed, flags, max_open=max_open)


def assert_same(batch, got, ref, what=""):
    """Bit-exact equality on status, assignment, bin types, bin count, total."""
    bad = np.nonzero(got.status != ref.status)[0]
    assert bad.size == 0, f"{what}: status differs at {bad[:5]}: {got.status[bad[:5]]} vs {ref.status[bad[:5]]}"
    for i in range(batch.N):
        if ref.status[i] != 0:
            continue
        a, b = int(batch.w_off[i]), int(batch.w_off[i + 1])
        nb = int(ref.num_bins[i])
        assert got.num_bins[i] == nb, f"{what}: instance {i} num_bins {got.num_bins[i]} vs {nb}"
        assert got.total[i] == ref.total[i], f"{what}: instance {i} total {got.total[i]} vs {ref.total[i]}"
        if not np.array_equal(got.bin_of_item[a:b], ref.bin_of_item[a:b]):
            j = int(np.nonzero(got.bin_of_item[a:b] != ref.bin_of_item[a:b])[0][0])
            raise AssertionError(f"{what}: instance {i} item {j}: bin {got.bin_of_item[a + j]} vs "
                                 f"{ref.bin_of_item[a + j]}")
        assert np.array_equal(got.bin_type[a:a + nb], ref.bin_type[a:a + nb]), \
            f"{what}: instance {i} bin types differ"
