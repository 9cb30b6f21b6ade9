"""Membrane systems larger than shared memory (global-memory kernel with tile
summaries) against the oracle, and config 4 (64 x 10^6 items) at full size:
the oracle on each instance's first items (a prefix packs the same way, as
items are taken in list order) plus properties that hold at any size."""
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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()


def _cfg4_like(N, m, seed):
    rng = np.random.default_rng(seed)
    return I.from_instances([(I.mixture_weights(rng, 0.8, (1, 100), (400, 1000), m), I.CFG4_B)
                             for _ in range(N)])


@pytest.mark.parametrize("crit", [native.FF, native.BF, native.WF, native.RANDOM])
def test_global_memory_kernel_vs_oracle(crit):
    b = _cfg4_like(3, 60_000, 40 + crit)
    assert_same(b, run_batch(b, 1, crit, seed=2), run_oracle(b, 1, crit, seed=2), f"kc c{crit}")


@pytest.mark.parametrize("preopen", [0, 1])
def test_global_memory_kernel_many_bins(preopen):
    """Items heavier than half of every capacity: ~2 bins per item, many tiles."""
    rng = np.random.default_rng(3 + preopen)
    w = rng.integers(51, 101, size=70_000).astype(np.int32)
    b = I.from_instances([(w, np.array([100, 90, 80], dtype=np.int32)), (w[:40000][::-1].copy(), np.array([100], dtype=np.int32))])
    for crit in (native.BF, native.FF, native.WF):
        assert_same(b, run_batch(b, 1, crit, 0, preopen), run_oracle(b, 1, crit, 0, preopen),
                    f"kc many bins c{crit}")


def test_mixed_batch_all_classes():
    """One batch with single-warp, block, wide-slot and global-memory systems."""
    rng = np.random.default_rng(12)
    inst = []
    for m in (50, 900, 5000, 15000, 30000, 45000):
        inst.append(I.random_instance(rng, m, 5, 1000))
    inst.append(I.random_instance(rng, 3000, 4, 100_000))          # B_1 > 32767
    inst.append(I.random_instance(rng, 0, 3, 100))
    b = I.from_instances(inst)
    for crit in (native.FF, native.BF, native.WF, native.RANDOM):
        assert_same(b, run_batch(b, 1, crit, seed=4), run_oracle(b, 1, crit, seed=4), f"mixed c{crit}")
        assert_same(b, run_batch(b, 1, crit, seed=4, plain=True), run_oracle(b, 1, crit, seed=4),
                    f"mixed plain c{crit}")


def _check_prefix(full_boi, full_types, pre):
    """The prefix packing equals the full packing restricted to the prefix, up
    to an increasing relabelling of bins."""
    k = pre.bin_of_item.shape[0]
    f = {}
    for d, g in zip(pre.bin_of_item.tolist(), full_boi[:k].tolist()):
        assert f.setdefault(d, g) == g
    keys = sorted(f)
    vals = [f[d] for d in keys]
    assert keys == list(range(pre.num_bins))
    assert all(a < b for a, b in zip(vals, vals[1:]))
    assert [int(full_types[v]) for v in vals] == pre.bin_type.tolist()


@pytest.mark.parametrize("crit", [native.BF, native.FF, native.WF])
def test_config4_full_size(crit):
    b = I.config4()
    got = run_batch(b, 1, crit)
    assert np.all(got.status == 0)
    for i in range(b.N):
        w, B = b.instance(i)
        a = int(b.w_off[i])
        nb = int(got.num_bins[i])
        res = oracle.PackResult(0, got.bin_of_item[a:a + len(w)], got.bin_type[a:a + nb], nb,
                                int(got.total[i]))
        P.check_packing(w, B, res)                  # every item once, no overflow, total
        if i % 16 == 0:
            k = 20_000
            pre = oracle.pack(w[:k], B, 1, crit)
            _check_prefix(res.bin_of_item, res.bin_type, pre)


@pytest.mark.parametrize("crit", [native.BF, native.RANDOM])
def test_cluster_kernel_remote_and_overflow(crit):
    """A system of ~1.8*10^5 bins: past CTA 0's shared memory into CTA 1's
    (distributed shared memory) and into the global-memory overflow of the
    two-CTA cluster kernel (BF items: 165 k bins on chip), against the
    oracle; RANDOM keeps every summary (segment maxima and presence rows)."""
    rng = np.random.default_rng(122)
    w = I.mixture_weights(rng, 0.9, (501, 1000), (1, 300), 200_000)
    b = I.from_instances([(w, np.array([1000, 700], dtype=np.int32))])
    assert_same(b, run_batch(b, 1, crit, seed=8), run_oracle(b, 1, crit, seed=8), f"kd overflow c{crit}")


@pytest.mark.parametrize("crit", [native.FF, native.BF, native.WF])
def test_cluster_kernel_closed_form(crit):
    """Items heavier than half of the one capacity: each opens its own bin
    and divides off the empty bin the next item takes (Rule 5), so item j is
    in bin j and the total is m * B_1 for every criterion.  2.5*10^5 items
    reach the global-memory overflow for every criterion; 6*10^5 pass the
    cluster kernel's 2^19 bins, and the global-memory kernel packs them."""
    rng = np.random.default_rng(130 + crit)
    ms = (250_000, 600_000)
    b = I.from_instances([(rng.integers(501, 1001, size=m).astype(np.int32), np.array([1000], dtype=np.int32))
                          for m in ms])
    got = run_batch(b, 1, crit)
    assert np.all(got.status == 0)
    for i, mi in enumerate(ms):
        a = int(b.w_off[i])
        assert got.num_bins[i] == mi and got.total[i] == 1000 * mi
        assert np.array_equal(got.bin_of_item[a:a + mi], np.arange(mi, dtype=np.int32))
        assert np.all(got.bin_type[a:a + mi] == 0)


def test_cluster_kernel_wide_residuals_hand_on():
    """B_1 past the presence rows of BF (1023): the global-memory kernel."""
    rng = np.random.default_rng(140)
    b = I.from_instances([(I.mixture_weights(rng, 0.8, (1, 100), (400, 1500), 60_000),
                           np.array([1500, 1000, 640, 300], dtype=np.int32))])
    for crit in (native.BF, native.RANDOM, native.WF):
        assert_same(b, run_batch(b, 1, crit, seed=3), run_oracle(b, 1, crit, seed=3), f"wide B1 c{crit}")


def test_many_tiny_instances():
    """100,000 instances of 0..12 items (empty ones included) in one batch:
    the size-class machinery, the work queue and the composition pass at a
    scale where per-instance overheads dominate; both heuristics."""
    rng = np.random.default_rng(101)
    ms = rng.integers(0, 13, size=100_000)
    inst = []
    for m in ms:
        n = int(rng.integers(1, 5))
        B = np.sort(rng.choice(np.arange(1, 200), size=n, replace=False))[::-1].astype(np.int32)
        inst.append((rng.integers(1, int(B[0]) + 1, size=int(m)).astype(np.int32), B))
    b = I.from_instances(inst)
    for (h, c, s, plain) in ((1, 1, 0, False), (1, 3, 0, True), (2, 1, 5, False), (2, 0, 3, True),
                             (1, 2, 4, False)):
        got = run_batch(b, h, c, s, seed=6, plain=plain)
        assert_same(b, got, run_oracle(b, h, c, s, seed=6), f"tiny h{h} c{c} s{s} plain={plain}")
