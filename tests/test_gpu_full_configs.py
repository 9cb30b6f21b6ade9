"""Full-size oracle parity for the batched workloads whose oracle run is too
slow for a test session, every instance and every element:

  config 4   64 membrane systems of 10^6 items (first heuristic, FF/BF/WF;
             Section 6.3 Rules 2-6), the global-memory path at full size
  config 3   4096 instances, second heuristic with sublists of 5 items
             (Section 6.4), FF/BF/WF/RANDOM

Expected values come from tests/golden/*_digests.json, written by
tests/golden/make_config_digests.py, which calls only the oracle and the
seeded input generator: per instance the status, bin count and total, and
SHA-256 digests (first 128 bits) of the item -> bin assignment and of the
used bins' types.  A GPU result equal in all five fields is the oracle's
result element by element.  The second heuristic is also compared element
by element with a live oracle run (BF), which names the first differing item
should a digest ever disagree."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import oracle_pins as P
from gpu_util import assert_same, run_batch, run_oracle
from paper_1602_08735_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1602_08735_gb300 import native  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CRIT = {"FF": native.FF, "BF": native.BF, "WF": native.WF, "RANDOM": native.RANDOM}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _d128(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()[:32]


def _check_inputs(b: I.Batch, doc: dict):
    want = doc["inputs_sha256"]
    got = {"w_all": hashlib.sha256(np.ascontiguousarray(b.w_all, dtype="<i4").tobytes()).hexdigest(),
           "w_off": hashlib.sha256(np.ascontiguousarray(b.w_off, dtype="<i8").tobytes()).hexdigest(),
           "B_all": hashlib.sha256(np.ascontiguousarray(b.B_all, dtype="<i4").tobytes()).hexdigest(),
           "B_off": hashlib.sha256(np.ascontiguousarray(b.B_off, dtype="<i4").tobytes()).hexdigest()}
    assert got == want, "the seeded generator drew different inputs than the stored oracle run"


def _compare(b: I.Batch, got, cols: dict, what: str):
    assert len(cols["status"]) == b.N
    st = np.asarray(cols["status"], dtype=np.int32)
    bad = np.nonzero(got.status != st)[0]
    assert bad.size == 0, f"{what}: status differs at {bad[:5]}"
    nb = np.asarray(cols["num_bins"], dtype=np.int64)
    tot = np.asarray(cols["total"], dtype=np.int64)
    bad = np.nonzero(got.num_bins != nb)[0]
    assert bad.size == 0, f"{what}: num_bins differs at {bad[:5]}: {got.num_bins[bad[:5]]} vs {nb[bad[:5]]}"
    bad = np.nonzero(got.total != tot)[0]
    assert bad.size == 0, f"{what}: total differs at {bad[:5]}"
    for i in range(b.N):
        a, e = int(b.w_off[i]), int(b.w_off[i + 1])
        assert _d128(got.bin_of_item[a:e]) == cols["bin_of_item_sha256"][i], f"{what}: instance {i} assignment"
        assert _d128(got.bin_type[a:a + int(nb[i])]) == cols["bin_type_sha256"][i], f"{what}: instance {i} types"


@pytest.mark.parametrize("crit", ["FF", "BF", "WF", "RANDOM"])
def test_config3_second_heuristic_full_batch(crit):
    doc = _load("config3_h2_digests.json")
    b = I.config3()
    _check_inputs(b, doc)
    got = run_batch(b, 2, CRIT[crit], doc["sublist_size"], seed=doc["random_seed"])
    _compare(b, got, doc["passes"][crit], f"cfg3 H2 {crit}")
    if crit == "BF":
        ref = run_oracle(b, 2, CRIT[crit], doc["sublist_size"], seed=doc["random_seed"])
        assert_same(b, got, ref, "cfg3 H2 BF live oracle")


@pytest.mark.parametrize("crit", ["BF", "FF", "WF"])
def test_config4_full_size_every_instance(crit):
    doc = _load("config4_digests.json")
    b = I.config4()
    _check_inputs(b, doc)
    got = run_batch(b, 1, CRIT[crit], seed=doc["random_seed"])
    _compare(b, got, doc["passes"][crit], f"cfg4 {crit}")
    for i in (0, b.N - 1):                        # invariants on the first and last system
        w, B = b.instance(i)
        a = int(b.w_off[i])
        nb = int(got.num_bins[i])
        P.check_packing(w, B, oracle.PackResult(0, got.bin_of_item[a:a + len(w)],
                                                got.bin_type[a:a + nb], nb, int(got.total[i])))
