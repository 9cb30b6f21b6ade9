"""The one-warp first-heuristic kernel (systems of at most 32768 bins, or
65536 in 16-bit slots when B_1 <= 255, one warp each) against the oracle,
element by element: every segment-register count it is built for, the BF
residual index and the full-scan BF it uses when B_1 > 1023, the literal
Rule 2 start, the 16-bit slot form, and the spill-and-rerun paths."""
import numpy as np
import pytest

from gpu_util import assert_same, run_batch, run_oracle
from paper_1602_08735_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1602_08735_gb300 import native  # noqa: E402

CRITS = [native.FF, native.BF, native.WF, native.RANDOM]


@pytest.fixture(scope="module", autouse=True)
def _one_warp():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()
    saved = native.get_config()
    native.set_config(large_warps=1, small_m=0)
    yield
    native.set_config(**saved)


def _uniform(rng, m, B):
    B = np.asarray(B, dtype=np.int32)
    return rng.integers(1, int(B[0]) + 1, size=m).astype(np.int32), B


@pytest.mark.parametrize("m_hi", [1500, 3500, 7000, 15000])
def test_segment_register_counts(m_hi):
    """Largest systems of ~m_hi items: slot counts that need 1, 2, 4 and 8
    segment words per lane, a ragged last segment in each."""
    b = I.config3(N=24, m_lo=max(100, m_hi // 3), m_hi=m_hi, seed=100 + m_hi)
    for c in CRITS:
        for pre in (0, 1):
            assert_same(b, run_batch(b, 1, c, preopen=pre, seed=5), run_oracle(b, 1, c, preopen=pre, seed=5),
                        f"m_hi={m_hi} c{c} pre{pre}")


def test_bf_without_index():
    """B_1 > 1023: BF items take the full scan (pure BF and RANDOM)."""
    rng = np.random.default_rng(31)
    inst = [_uniform(rng, m, B) for m, B in
            ((3000, [5000, 3000, 1024]), (800, [1024, 1000]), (5000, [32767, 20000, 1500, 40]),
             (257, [2000]))]
    b = I.from_instances(inst)
    for c in CRITS:
        for pre in (0, 1):
            assert_same(b, run_batch(b, 1, c, preopen=pre, seed=11), run_oracle(b, 1, c, preopen=pre, seed=11),
                        f"no index c{c} pre{pre}")


def test_index_boundaries():
    """B_1 = 1023 (largest indexed residual), tiny capacities, weights equal
    to a capacity (bins that fill at once), one item, one type."""
    rng = np.random.default_rng(32)
    inst = [_uniform(rng, 4000, [1023, 700, 5]), _uniform(rng, 2000, [1]),
            (np.full(600, 7, dtype=np.int32), np.array([7, 3], dtype=np.int32)),
            (np.array([1023], dtype=np.int32), np.array([1023], dtype=np.int32)),
            (np.array([3, 3, 3, 3, 4, 4, 1], dtype=np.int32), np.array([8, 6, 4], dtype=np.int32)),
            _uniform(rng, 1000, [64, 63, 62, 61, 60, 59, 58, 57, 56, 55, 54, 53, 52, 51, 50, 49,
                                 48, 47, 46, 45, 44, 43, 42, 41, 40, 39, 38, 37, 36, 35, 34, 33])]
    b = I.from_instances(inst)
    for c in CRITS:
        for pre in (0, 1):
            assert_same(b, run_batch(b, 1, c, preopen=pre, seed=12), run_oracle(b, 1, c, preopen=pre, seed=12),
                        f"boundaries c{c} pre{pre}")


@pytest.mark.parametrize("pct", [50, 200])
def test_spill_rerun_one_warp(pct):
    """Systems that outgrow their slots are repacked at full size (up to
    2m + 32 = 32768 slots, the kernel's limit)."""
    saved = native.get_config()
    native.set_config(large_warps=1, small_m=0, slot_pct=pct)
    try:
        rng = np.random.default_rng(33)
        inst = [(rng.integers(51, 101, size=m).astype(np.int32), np.array([100, 60], dtype=np.int32))
                for m in (500, 4000, 16368)]
        inst += [I.config3(N=12, m_hi=6000, seed=34).instance(i) for i in range(12)]
        b = I.from_instances(inst)
        for c in CRITS:
            assert_same(b, run_batch(b, 1, c, seed=4), run_oracle(b, 1, c, seed=4), f"spill {pct} c{c}")
            assert_same(b, run_batch(b, 1, c, seed=4, plain=True), run_oracle(b, 1, c, seed=4),
                        f"spill plain {pct} c{c}")
    finally:
        native.set_config(**saved)


@pytest.mark.parametrize("wpb", [2, 16])
def test_many_warps_per_block(wpb):
    """Several systems per block, each warp with its own shared memory."""
    saved = native.get_config()
    native.set_config(large_warps=1, small_m=2000, small_warps_per_block=wpb)
    try:
        b = I.config3(N=200, m_hi=6000, seed=35)
        for c in CRITS:
            assert_same(b, run_batch(b, 1, c, seed=6), run_oracle(b, 1, c, seed=6), f"wpb {wpb} c{c}")
    finally:
        native.set_config(**saved)


def test_large_systems_routes():
    """Systems past the worst-case shared-memory size: held by the one-warp
    kernel when the slot estimate suffices (20k items of U[1,150]), spilled
    twice and finished in global memory when it does not (30k items that
    each fill half a bin: two bins per item), and in the one-warp kernel's
    16-bit slots beyond the 32-bit estimate's reach (45k items, B_1 = 150).
    Results equal the oracle's whatever the route."""
    rng = np.random.default_rng(71)
    B = np.array([150, 120, 100, 80, 50], dtype=np.int32)
    inst = [(rng.integers(1, 151, size=20_000).astype(np.int32), B),
            (rng.integers(51, 101, size=30_000).astype(np.int32), np.array([100, 60], dtype=np.int32)),
            (rng.integers(1, 151, size=45_000).astype(np.int32), B),
            (rng.integers(1, 151, size=3_000).astype(np.int32), B)]
    b = I.from_instances(inst)
    for c in CRITS:
        ref = run_oracle(b, 1, c, seed=7)
        assert_same(b, run_batch(b, 1, c, seed=7), ref, f"routes c{c}")
        assert_same(b, run_batch(b, 1, c, seed=7, plain=True), ref, f"routes plain c{c}")


def test_sixteen_bit_slots():
    """Systems with B_1 <= 255 past the 32-bit slots' reach (more than about
    40.8k items) in the one-warp kernel's 16-bit slots (at most 65536 bins):
    config-5-like requests of 60k and 100k items, B_1 = 255 exactly; one
    system that needs a bin per item (every item fills more than half of the
    largest bin) and leaves the 16-bit slots at once, and one that passes
    65536 bins late (small items, then large ones): both finish in global
    memory.  Every criterion; the literal Rule 2 start and the plain path
    for BF.  Results equal the oracle's whatever the route."""
    rng = np.random.default_rng(72)
    B5 = np.array([150, 120, 100, 80, 50], dtype=np.int32)
    late = np.concatenate([rng.integers(1, 21, size=30_000), rng.integers(129, 256, size=70_000)])
    inst = [(rng.integers(1, 151, size=100_000).astype(np.int32), B5),
            (I.mixture_weights(rng, 0.7, (1, 37), (75, 150), 60_000), B5),
            (rng.integers(1, 256, size=50_000).astype(np.int32), np.array([255, 254, 17], dtype=np.int32)),
            (rng.integers(129, 256, size=70_000).astype(np.int32), np.array([255, 200, 130], dtype=np.int32)),
            (late.astype(np.int32), np.array([255, 130], dtype=np.int32)),
            (rng.integers(1, 151, size=2_000).astype(np.int32), B5)]
    b = I.from_instances(inst)
    for c in CRITS:
        ref = run_oracle(b, 1, c, seed=8)
        assert_same(b, run_batch(b, 1, c, seed=8), ref, f"16-bit c{c}")
        if c == native.BF:
            assert_same(b, run_batch(b, 1, c, seed=8, plain=True), ref, f"16-bit plain c{c}")
            assert_same(b, run_batch(b, 1, c, preopen=1, seed=8), run_oracle(b, 1, c, preopen=1, seed=8),
                        f"16-bit preopen c{c}")
