"""Multi-process path on CPU: the library's batch split (vsbpp_shard, longest
processing time first) and the gather of per-rank results, over two gloo
ranks.  Instances are independent problems (Section 6.1), so any split packs
each instance exactly as the whole batch does; the test packs each rank's
part with the oracle (no GPU here) and compares the gathered result with the
oracle on the whole batch, element by element."""
import itertools
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

from paper_1602_08735_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_1602_08735_gb300 import build
    build.build()
    from paper_1602_08735_gb300 import native as nat
    nat.load()
    return nat


def _opt_makespan(ms, world):
    best = None
    for assign in itertools.product(range(world), repeat=len(ms)):
        loads = [0] * world
        for m, r in zip(ms, assign):
            loads[r] += m
        best = max(loads) if best is None else min(best, max(loads))
    return best


def test_split_properties(native):
    rng = np.random.default_rng(1)
    for t in range(200):
        N = int(rng.integers(0, 9))
        world = int(rng.integers(1, 4))
        ms = rng.integers(0, 50, size=N)
        w_off = np.concatenate([[0], np.cumsum(ms)]).astype(np.int64)
        rank_of, items = native.shard(w_off, world)
        assert rank_of.shape == (N,) and np.all((rank_of >= 0) & (rank_of < world))
        assert [int(ms[rank_of == r].sum()) for r in range(world)] == items.tolist()
        again, _ = native.shard(w_off, world)
        assert np.array_equal(rank_of, again)                 # every rank computes the same split
        if N:
            opt = _opt_makespan(ms.tolist(), world)
            # Graham's bound for longest processing time first
            assert 3 * world * int(items.max()) <= (4 * world - 1) * opt
    # one rank takes everything
    rank_of, items = native.shard(np.array([0, 3, 3, 9], dtype=np.int64), 1)
    assert rank_of.tolist() == [0, 0, 0] and items.tolist() == [9]
    # the longest first, each to the least loaded rank (lowest on ties): m =
    # 5, 7, 3, 4 -> 7 to rank 0, 5 to rank 1, 4 to rank 1 (5 < 7), 3 to rank 0
    rank_of, items = native.shard(np.array([0, 5, 12, 15, 19], dtype=np.int64), 2)
    assert rank_of.tolist() == [1, 0, 0, 1] and items.tolist() == [10, 9]


def test_split_rejects_bad_arguments(native):
    from paper_1602_08735_gb300.native import VsbppError
    for w_off, world in (([0, 3, 2], 2), ([0, 1], 0)):
        with pytest.raises(VsbppError):
            native.shard(np.array(w_off, dtype=np.int64), world)


CHILD = r"""
import os, sys, json
sys.path[:0] = [%r, %r]
import numpy as np
import torch.distributed as dist
import oracle
from paper_1602_08735_gb300 import instances as I, shard
dist.init_process_group("gloo")
ws, rank = dist.get_world_size(), dist.get_rank()
batch = I.config3(seed=7, N=48, m_hi=2000)
part, idx = shard.split(batch, ws, rank)
res = oracle.pack_many(part.w_all, part.w_off, part.B_all, part.B_off, 1, 1, nthreads=2)
full = shard.gather(batch, idx, res, ws, rank)
out = {"rank": rank, "instances": int(part.N), "items": int(part.total_items)}
if rank == 0:
    ref = oracle.pack_many(batch.w_all, batch.w_off, batch.B_all, batch.B_off, 1, 1, nthreads=2)
    st, boi, bt, nb, tot = full
    out["same"] = bool(np.array_equal(st, ref.status) and np.array_equal(nb, ref.num_bins)
                       and np.array_equal(tot, ref.total) and np.array_equal(boi, ref.bin_of_item))
    out["types_same"] = all(np.array_equal(bt[a:a + n], ref.bin_type[a:a + n])
                            for a, n in zip(batch.w_off[:-1].tolist(), ref.num_bins.tolist()))
    out["total_items"] = int(batch.total_items)
print(json.dumps(out))
dist.destroy_process_group()
""" % (ROOT, os.path.join(ROOT, "tests"))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_split_pack_gather(native):
    pytest.importorskip("torch")
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=300) for p in procs]
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    r0 = next(r for r in res if r["rank"] == 0)
    assert r0["same"] and r0["types_same"]
    assert sum(r["instances"] for r in res) == 48
    assert sum(r["items"] for r in res) == r0["total_items"]
    assert all(r["instances"] > 0 for r in res)
