"""CUDA path vs the CPU oracle, element by element (bit-exact integers)."""
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

H1_CRITERIA = [native.FF, native.BF, native.WF, native.RANDOM]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()
    cfg = native.get_config()
    yield
    native.set_config(**cfg)


def test_hand_examples_host_api():
    """Every hand-worked packing, the Remark 3, pre-sort and bounded-space
    ones included, through the host-memory call."""
    for ex in P.load_golden("hand_examples.json")["examples"]:
        r = native.pack(ex["w"], ex["B"], ex["heuristic"], ex["criterion"], ex["sublist_size"],
                        ex["preopen"], ex["seed"], ex.get("flags", 0), ex.get("max_open", 0))
        assert r.status == 0, ex["name"]
        assert r.bin_of_item.tolist() == ex["bin_of_item"], ex["name"]
        assert r.bin_type.tolist() == ex["bin_type"], ex["name"]
        assert r.total == ex["total"], ex["name"]


@pytest.mark.parametrize("crit", H1_CRITERIA)
def test_config1_h1(crit):
    b = I.config1()
    assert_same(b, run_batch(b, 1, crit, seed=99), run_oracle(b, 1, crit, seed=99), f"cfg1 H1 c{crit}")


@pytest.mark.parametrize("crit", H1_CRITERIA)
def test_config1_h2(crit):
    b = I.config1()
    assert_same(b, run_batch(b, 2, crit, 5, seed=7), run_oracle(b, 2, crit, 5, seed=7), f"cfg1 H2 c{crit}")


def test_config1_first10_vs_optimum():
    w, B = I.config1().instance(0)
    w10 = w[:10]
    opt = oracle.opt_bruteforce(w10, B)
    for h, s in ((1, 0), (2, 5)):
        for c in (native.FF, native.BF, native.WF):
            r = native.pack(w10, B, h, c, s)
            assert r.status == 0 and r.total >= opt


@pytest.mark.parametrize("variant", ["u", "m"])
@pytest.mark.parametrize("crit", H1_CRITERIA)
def test_config2_h1(variant, crit):
    b = I.config2(variant)
    assert_same(b, run_batch(b, 1, crit, seed=5), run_oracle(b, 1, crit, seed=5), f"cfg2{variant} H1 c{crit}")


@pytest.mark.parametrize("variant", ["u", "m"])
def test_config2_h2(variant):
    b = I.config2(variant)
    assert_same(b, run_batch(b, 2, native.BF, 5), run_oracle(b, 2, native.BF, 5), f"cfg2{variant} H2")


@pytest.mark.parametrize("crit", H1_CRITERIA)
def test_config3_full_batch(crit):
    b = I.config3()
    assert_same(b, run_batch(b, 1, crit, seed=3), run_oracle(b, 1, crit, seed=3), f"cfg3 H1 c{crit}")



def _fuzz_batch(seed, N=300, m_hi=400, cap_choices=(20, 100, 1000, 32767, 40000, 2**31 - 1)):
    rng = np.random.default_rng(seed)
    inst = []
    for _ in range(N):
        m = int(rng.integers(0, m_hi))
        n = int(rng.integers(1, 9))
        cap = int(rng.choice(cap_choices))
        inst.append(I.random_instance(rng, m, n, cap))
    return I.from_instances(inst)


@pytest.mark.parametrize("preopen", [0, 1])
@pytest.mark.parametrize("crit", H1_CRITERIA)
def test_fuzz_h1(crit, preopen):
    b = _fuzz_batch(100 + crit + 10 * preopen)
    assert_same(b, run_batch(b, 1, crit, 0, preopen, 17), run_oracle(b, 1, crit, 0, preopen, 17),
                f"fuzz H1 c{crit} p{preopen}")


@pytest.mark.parametrize("s", [1, 3, 10, 64])
def test_fuzz_h1_sublists(s):
    b = _fuzz_batch(200 + s)
    for crit in (native.BF, native.RANDOM):
        assert_same(b, run_batch(b, 1, crit, s, 0, 5), run_oracle(b, 1, crit, s, 0, 5), f"H1 s={s} c{crit}")


@pytest.mark.parametrize("s", [1, 2, 5, 6])
def test_fuzz_h2(s):
    b = _fuzz_batch(300 + s, N=120, m_hi=60)
    for crit in H1_CRITERIA:
        for pre in (0, 1):
            assert_same(b, run_batch(b, 2, crit, s, pre, 9), run_oracle(b, 2, crit, s, pre, 9),
                        f"H2 s={s} c{crit} p{pre}")


def test_plain_equals_batch_and_oracle():
    b = I.config3(N=64, m_hi=3000)
    ref = run_oracle(b, 1, native.BF)
    assert_same(b, run_batch(b, 1, native.BF, plain=True), ref, "plain")
    assert_same(b, run_batch(b, 1, native.BF), ref, "batch")


def test_batch_equals_single_calls():
    b = I.config3(N=12, m_hi=2000, seed=44)
    got = run_batch(b, 1, native.WF)
    for i in range(b.N):
        w, B = b.instance(i)
        r = native.pack(w, B, 1, native.WF)
        a = int(b.w_off[i])
        assert r.status == 0
        assert np.array_equal(r.bin_of_item, got.bin_of_item[a:a + len(w)])
        assert r.total == got.total[i]


@pytest.mark.parametrize("chunk", [32, 96, 4096])
def test_chunk_boundaries(chunk):
    saved = native.get_config()
    native.set_config(chunk=chunk)
    try:
        b = I.config3(N=40, m_hi=5000, seed=8)
        for crit in (native.FF, native.BF, native.WF):
            assert_same(b, run_batch(b, 1, crit), run_oracle(b, 1, crit), f"chunk {chunk} c{crit}")
    finally:
        native.set_config(**saved)


@pytest.mark.parametrize("warps", [1, 2, 4, 8, 16, 32])
def test_group_sizes(warps):
    saved = native.get_config()
    native.set_config(large_warps=warps, small_m=64)
    try:
        b = I.config3(N=40, m_hi=4000, seed=9)
        for crit in (native.BF, native.FF, native.WF, native.RANDOM):
            assert_same(b, run_batch(b, 1, crit, seed=1), run_oracle(b, 1, crit, seed=1), f"G={warps} c{crit}")
    finally:
        native.set_config(**saved)


@pytest.mark.parametrize("small_m", [0, 300, 3000])
def test_single_warp_class(small_m):
    saved = native.get_config()
    native.set_config(small_m=small_m)
    try:
        b = I.config3(N=60, m_hi=4000, seed=10)
        for crit in (native.BF, native.FF, native.WF, native.RANDOM):
            assert_same(b, run_batch(b, 1, crit, seed=2), run_oracle(b, 1, crit, seed=2),
                        f"small_m={small_m} c{crit}")
    finally:
        native.set_config(**saved)


def test_edge_cases():
    cases = [
        ([], [10]), ([5], [5]), ([1] * 50, [1]), ([7] * 33, [7, 3]),
        ([32767, 1, 32767], [32767]), ([32768, 2, 32767], [32768, 5]),
        ([2**31 - 1, 1, 5], [2**31 - 1, 3]), ([3, 3, 3], [6, 5, 4, 3, 2, 1]),
    ]
    for w, B in cases:
        for h, s in ((1, 0), (2, 0), (1, 2)):
            for c in (0, 1, 2, 3):
                r = native.pack(w, B, h, c, s, 0, 1)
                ref = oracle.pack(w, B, h, c, s, 0, 1)
                assert r.status == ref.status == 0, (w, B)
                assert r.bin_of_item.tolist() == ref.bin_of_item.tolist(), (w, B, h, c)
                assert r.bin_type.tolist() == ref.bin_type.tolist()
                assert r.total == ref.total


def test_errors():
    assert native.pack([1, 2], [50, 100]).status == native.EINVAL
    assert native.pack([0, 2], [50]).status == native.EINVAL
    assert native.pack([51], [50]).status == native.ETOOBIG
    assert native.pack([0, 99], [50]).status == native.EINVAL
    assert native.pack([99, 0], [50]).status == native.ETOOBIG
    assert native.pack([1], list(range(40, 7, -1))).status == native.EINVAL    # n = 33
    assert native.pack([1], [5], heuristic=3).status == native.EINVAL
    assert native.pack([1], [5], heuristic=2, sublist_size=13).status == native.EINVAL
    assert native.pack([1] * 8, [5], heuristic=2, sublist_size=8, preopen=1).status == native.EINVAL
    # mixed batch: bad instances flagged, good ones packed
    b = I.from_instances([([1, 2, 3], [5]), ([0], [5]), ([6], [5]), ([4, 4], [5, 4]), ([1], [3, 3])])
    got = run_batch(b, 1, native.BF)
    assert got.status.tolist() == [0, native.EINVAL, native.ETOOBIG, 0, native.EINVAL]
    ref = run_oracle(b, 1, native.BF)
    assert_same(b, got, ref, "mixed")


@pytest.mark.parametrize("pct", [50, 100])
def test_spill_and_rerun(pct):
    """Systems that outgrow their shared-memory slots are repacked at full
    size; the result must not change."""
    saved = native.get_config()
    native.set_config(slot_pct=pct)
    try:
        rng = np.random.default_rng(77)
        inst = [(rng.integers(51, 101, size=m).astype(np.int32), np.array([100, 60], dtype=np.int32))
                for m in (300, 2000, 19000)]            # ~2 bins per item: always spills
        inst += [I.config3(N=20, m_hi=5000, seed=78).instance(i) for i in range(20)]
        b = I.from_instances(inst)
        for crit in H1_CRITERIA:
            assert_same(b, run_batch(b, 1, crit, seed=3), run_oracle(b, 1, crit, seed=3), f"spill {pct} c{crit}")
            assert_same(b, run_batch(b, 1, crit, seed=3, plain=True), run_oracle(b, 1, crit, seed=3),
                        f"spill plain {pct} c{crit}")
    finally:
        native.set_config(**saved)


def test_second_heuristic_slot_forms():
    """The second heuristic's one-word slots hold capacities up to 2047 and
    16 types; B_1 = 2048 or a 17th type takes the wide slots.  Both sides of
    each boundary against the oracle, every criterion, sublists of 4-6."""
    rng = np.random.default_rng(61)
    def inst(B1, n, m):
        B = np.sort(rng.choice(np.arange(1, B1), size=n - 1, replace=False))[::-1]
        B = np.concatenate([[B1], B]).astype(np.int32)
        return rng.integers(1, B1 + 1, size=m).astype(np.int32), B
    b = I.from_instances([inst(2047, 5, 97), inst(2048, 5, 101), inst(900, 16, 64), inst(900, 17, 66),
                          inst(2047, 16, 40), inst(3000, 32, 55)])
    for s in (4, 5, 6):
        for crit in H1_CRITERIA:
            assert_same(b, run_batch(b, 2, crit, s, seed=8), run_oracle(b, 2, crit, s, seed=8), f"s={s} c{crit}")


@pytest.mark.parametrize("s", [7, 8, 9])
def test_exhaustive_second_heuristic(s):
    """Sublists of 7..12 items: every permutation searched across the GPU
    (Section 7's exhaustive comparison); equal to the oracle on several
    sublists per instance, ragged last sublists, all criteria, both paths."""
    rng = np.random.default_rng(80 + s)
    inst = [I.random_instance(rng, int(m), int(rng.integers(1, 6)), 60) for m in (s, 2 * s + 3, 3 * s - 1, 5)]
    inst.append((rng.integers(1, 5001, size=s + 2).astype(np.int32), np.array([5000, 3000, 900], dtype=np.int32)))
    b = I.from_instances(inst)
    for crit in H1_CRITERIA:
        ref = run_oracle(b, 2, crit, s, seed=4)
        assert_same(b, run_batch(b, 2, crit, s, seed=4), ref, f"s={s} c{crit}")
        assert_same(b, run_batch(b, 2, crit, s, seed=4, plain=True), ref, f"s={s} plain c{crit}")


def test_exhaustive_ten_items():
    """One 10-item list: all 3,628,800 permutations (the largest case Section
    7 reports for its exhaustive implementations)."""
    rng = np.random.default_rng(90)
    b = I.from_instances([I.random_instance(rng, 10, 3, 100)])
    for crit in (native.FF, native.BF, native.WF):
        assert_same(b, run_batch(b, 2, crit, 10), run_oracle(b, 2, crit, 10), f"ten c{crit}")
