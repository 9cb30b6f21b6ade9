"""The CPU oracle against its pins (no GPU).  See tests/oracle_pins.py."""
import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_1602_08735_gb300 import instances as I


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda p: p.__name__)
def test_pin(oracle_lib, pin):
    pin(oracle_lib)


def test_random_criterion_from_vectors():
    d = P.load_golden("splitmix64_vectors.json")
    crit = [int(v) % 3 for v in d["outputs"]]
    assert crit == [0, 1, 0, 1, 2]          # FF, BF, FF, BF, WF


def test_sublists_equal_independent_packs(oracle_lib):
    """First heuristic with sublists: each chunk is its own membrane system
    (Rule 2); ids are offset by the bins of earlier chunks; totals add."""
    rng = np.random.default_rng(21)
    for t in range(30):
        w, B = I.random_instance(rng, int(rng.integers(1, 80)), int(rng.integers(1, 6)), 200)
        s = int(rng.integers(1, 15))
        crit = int(rng.integers(0, 3))
        full = oracle_lib.pack(w, B, 1, crit, s)
        off, tot, boi, bty = 0, 0, [], []
        for a in range(0, len(w), s):
            r = oracle_lib.pack(w[a:a + s], B, 1, crit)
            boi += (r.bin_of_item + off).tolist()
            bty += r.bin_type.tolist()
            off += r.num_bins
            tot += r.total
        assert full.bin_of_item.tolist() == boi
        assert full.bin_type.tolist() == bty
        assert full.total == tot


@pytest.mark.parametrize("flags", [0, 1])
def test_determinism_and_pack_many(oracle_lib, flags):
    """The threaded batch driver gives each instance exactly the single call's
    result (flags = 1: the Remark 3 option of Rule 5)."""
    b = I.config3(N=24, m_hi=600)
    for crit in ((1,) if flags == 0 else (0, 1, 2)):
        many = oracle_lib.pack_many(b.w_all, b.w_off, b.B_all, b.B_off, 1, crit, flags=flags, nthreads=4)
        for i in range(b.N):
            w, B = b.instance(i)
            r = oracle_lib.pack(w, B, 1, crit, flags=flags)
            a = int(b.w_off[i])
            assert many.status[i] == 0
            assert many.total[i] == r.total
            assert many.bin_of_item[a:a + len(w)].tolist() == r.bin_of_item.tolist()
            assert many.bin_type[a:a + r.num_bins].tolist() == r.bin_type.tolist()


def test_group2_fixture_matches_table7_weights():
    d = P.load_golden("group2_multisets.json")
    for inst in d["instances"]:
        assert sum(c for _, c in inst["pairs"]) == 1000
        assert sum(w * c for w, c in inst["pairs"]) == inst["total_weight"]


def test_group2_second_heuristic_sane(oracle_lib):
    """Section 7 Table 7 reports H2 utilisations of 0.84-0.90 on these
    multisets; the item order is not printed, so only a band is checked."""
    d = P.load_golden("group2_multisets.json")
    rng = np.random.default_rng(7)
    for inst in d["instances"]:
        w = np.repeat([p[0] for p in inst["pairs"]], [p[1] for p in inst["pairs"]]).astype(np.int32)
        rng.shuffle(w)
        r = oracle_lib.pack(w, d["B"], 2, 1, 5)
        P.check_packing(w, d["B"], r)
        util = inst["total_weight"] / r.total
        assert 0.6 < util <= 1.0


def test_generators_are_seeded():
    a, b = I.config3(N=8), I.config3(N=8)
    assert np.array_equal(a.w_all, b.w_all) and np.array_equal(a.B_all, b.B_all)
    c1 = I.config1()
    w, B = c1.instance(0)
    assert len(w) == 100 and B.tolist() == [100, 70, 40] and w.min() >= 1 and w.max() <= 100
    c3 = I.config3(N=64)
    for i in range(c3.N):
        w, B = c3.instance(i)
        assert 100 <= len(w) <= 10_000 and len(B) in (3, 5, 7)
        assert np.all(np.diff(B) < 0) and B[-1] >= 20 and B[0] <= 1000
        assert w.min() >= 1 and w.max() <= B[0]
