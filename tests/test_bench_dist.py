"""The multi-rank path of bench.py on CPU: two gloo ranks rendezvous on
127.0.0.1, each takes its part of one global batch under the library's
split (no collective on the data), and the timing is reduced with max/sum
over ranks."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys, json
sys.path.insert(0, %r)
import numpy as np
import bench
from paper_1602_08735_gb300 import instances as I
ws, rank, local = bench.dist_setup()
assert ws == 2
mx = bench.max_over_ranks(float(rank + 1), ws)
sm = bench.sum_over_ranks(float(10 * (rank + 1)), ws)
bench.barrier(ws)
from paper_1602_08735_gb300 import native
native.load()
part = bench.rank_batch(native, I, 8, ws, rank)
whole = I.config3(seed=3, N=16)
print(json.dumps({"rank": rank, "max": mx, "sum": sm, "instances": part.N,
                  "items": part.total_items, "whole_items": whole.total_items}))
import torch.distributed as dist
dist.destroy_process_group()
""" % ROOT


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks():
    pytest.importorskip("torch")
    from paper_1602_08735_gb300 import build
    build.build()
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=180) for p in procs]
    import json
    res = []
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
        res.append(json.loads(o.strip().splitlines()[-1]))
    assert all(r["max"] == 2.0 for r in res)
    assert all(r["sum"] == 30.0 for r in res)
    assert res[0]["instances"] + res[1]["instances"] == 16
    assert res[0]["items"] + res[1]["items"] == res[0]["whole_items"]
