"""Write the oracle's per-instance results for the two full-size batched
workloads that are too slow to pack with the oracle inside a GPU test run:

  config4_digests.json     64 instances of 10^6 items, B = {1000, 800, 640,
                           500, 400, 300, 200}, w = 0.8*U[1,100] + 0.2*U[400,1000]
                           (seed 4); first heuristic, one membrane system per
                           instance, FF / BF / WF (Section 6.3, Rules 2-6)
  config3_h2_digests.json  4096 instances, m log-uniform in [100, 10^4]
                           (seed 3); second heuristic, sublists of 5 items,
                           FF / BF / WF / RANDOM (Section 6.4)

Every value comes from ``oracle`` (the plain CPU simulation) and from the
seeded input generator; nothing here calls the CUDA library.  Per instance the
file holds the bin count, the total capacity of the used bins, and SHA-256
digests (the first 128 bits, as 32 hex digits) of the item -> bin assignment
(int32 little-endian, m entries) and of the used bins' types (int32
little-endian, num_bins entries), one column per field, so a test can
compare every element of a GPU result without storing 512 MB of expected
output.  A digest of the inputs guards against a generator that draws
differently on another machine.

Usage:  python tests/golden/make_config_digests.py [--threads T] [--only config4|config3h2]

Config 4 costs about 10^13 flat-scan fit tests (WF dominates: ~7 minutes per
instance on one x86 core), so the script checkpoints after every chunk of
instances into ``<name>.partial.json`` and resumes from it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1602_08735_gb300 import instances as I  # noqa: E402

CRIT_NAMES = {oracle.FF: "FF", oracle.BF: "BF", oracle.WF: "WF", oracle.RANDOM: "RANDOM"}
RANDOM_SEED = 3          # seed of the RANDOM criterion's SplitMix64 stream (reading G12)


def sha256_i32(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def digest128(a: np.ndarray) -> str:
    """First 128 bits of the SHA-256 of an int32 array's little-endian bytes."""
    return sha256_i32(a)[:32]


def input_digest(b: I.Batch) -> dict:
    return {"w_all": sha256_i32(b.w_all),
            "w_off": hashlib.sha256(np.ascontiguousarray(b.w_off, dtype="<i8").tobytes()).hexdigest(),
            "B_all": sha256_i32(b.B_all),
            "B_off": sha256_i32(b.B_off)}


FIELDS = ("status", "num_bins", "total", "bin_of_item_sha256", "bin_type_sha256")


def append_records(cols: dict, b: I.Batch, res: oracle.BatchResult) -> None:
    """Append one entry per instance of the (sub-)batch b to each column; res
    is CSR-aligned with b."""
    for j in range(b.N):
        a, e = int(b.w_off[j]), int(b.w_off[j + 1])
        nb = int(res.num_bins[j])
        cols["status"].append(int(res.status[j]))
        cols["num_bins"].append(nb)
        cols["total"].append(int(res.total[j]))
        cols["bin_of_item_sha256"].append(digest128(res.bin_of_item[a:e]))
        cols["bin_type_sha256"].append(digest128(res.bin_type[a:a + nb]))


def write_doc(path: str, doc: dict) -> None:
    """JSON with one line per column (readable diffs, ~1 MB for 4096 x 4)."""
    head = {k: v for k, v in doc.items() if k != "passes"}
    lines = ["{"]
    for k, v in head.items():
        lines.append(f" {json.dumps(k)}: {json.dumps(v)},")
    lines.append(' "passes": {')
    names = list(doc["passes"])
    for pi, name in enumerate(names):
        cols = doc["passes"][name]
        lines.append(f"  {json.dumps(name)}: {{")
        for ci, k in enumerate(FIELDS):
            sep = "," if ci + 1 < len(FIELDS) else ""
            lines.append(f"   {json.dumps(k)}: {json.dumps(cols[k], separators=(',', ':'))}{sep}")
        lines.append("  }" + ("," if pi + 1 < len(names) else ""))
    lines.append(" }")
    lines.append("}")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


def run(name: str, b: I.Batch, heuristic: int, sublist_size: int, crits, threads: int,
        chunk: int, meta: dict):
    path = os.path.join(HERE, f"{name}.json")
    part = path.replace(".json", ".partial.json")
    doc = {"generated_by": "tests/golden/make_config_digests.py (oracle only)", **meta,
           "heuristic": heuristic, "sublist_size": sublist_size, "random_seed": RANDOM_SEED,
           "inputs_sha256": input_digest(b), "passes": {}}
    if os.path.exists(part):
        with open(part) as f:
            old = json.load(f)
        if old.get("inputs_sha256") == doc["inputs_sha256"]:
            doc["passes"] = old["passes"]
    for c in crits:
        cols = doc["passes"].setdefault(CRIT_NAMES[c], {k: [] for k in FIELDS})
        start = len(cols["status"])
        for lo in range(start, b.N, chunk):
            idx = list(range(lo, min(b.N, lo + chunk)))
            sub = b.subset(idx)
            t = time.time()
            res = oracle.pack_many(sub.w_all, sub.w_off, sub.B_all, sub.B_off, heuristic, c,
                                   sublist_size, 0, RANDOM_SEED, nthreads=threads)
            append_records(cols, sub, res)
            with open(part, "w") as f:
                json.dump(doc, f)
            print(f"{name} {CRIT_NAMES[c]} instances {lo}..{idx[-1]} in {time.time() - t:.1f}s",
                  flush=True)
    write_doc(path, doc)
    if os.path.exists(part):
        os.remove(part)
    print("wrote", path, flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", choices=["config4", "config3h2"], default=None)
    a = ap.parse_args()
    if a.only in (None, "config3h2"):
        b3 = I.config3()
        run("config3_h2_digests", b3, oracle.H2, 5,
            [oracle.FF, oracle.BF, oracle.WF, oracle.RANDOM], a.threads, 4096,
            {"workload": "config 3: 4096 instances, m log-uniform in [100, 10^4], n in {3,5,7}, "
                         "B distinct in [20,1000] descending, w ~ U[1,B_1], seed 3"})
    if a.only in (None, "config4"):
        b4 = I.config4()
        run("config4_digests", b4, oracle.H1, 0, [oracle.BF, oracle.FF, oracle.WF], a.threads,
            a.threads,
            {"workload": "config 4: 64 instances of 10^6 items, B = {1000,800,640,500,400,300,200}, "
                         "w = 0.8*U[1,100] + 0.2*U[400,1000], seed 4"})


if __name__ == "__main__":
    main()
