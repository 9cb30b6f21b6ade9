"""vsbpp_pack_batch_noalloc: the batched pack for callers that cannot
allocate device memory (code confined to a fixed memory reservation or
another allocator's arena, allocation-free latency paths).  Its scratch is
one static device array shared by every call, so two calls in a row must not
see each other's leftovers.  Checked through the C ABI against
vsbpp_pack_batch and against the CPU oracle.

This file is collected last on purpose: it must pass both on its own in a
fresh process and after every other test."""
import numpy as np
import pytest

import oracle
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


def _run(fn, db, crit, seed=0, preopen=0):
    out = native.DeviceResult.empty(db.N, db.total_items)
    out.status.fill_(77)
    out.bin_of_item.fill_(-9)
    out.bin_type.fill_(-9)
    rc = fn(db, out, native.H1, crit, 0, preopen, seed)
    assert rc == 0, native.strerror(rc)
    torch.cuda.synchronize()
    return out.to_host(db.N, db.total_items)


def _same(a, b, db, batch):
    st_a, boi_a, bt_a, nb_a, tot_a = a
    st_b, boi_b, bt_b, nb_b, tot_b = b
    assert np.array_equal(st_a, st_b)
    assert np.array_equal(nb_a, nb_b) and np.array_equal(tot_a, tot_b)
    assert np.array_equal(boi_a, boi_b)
    for i in range(db.N):
        a0 = int(batch.w_off[i])
        assert np.array_equal(bt_a[a0:a0 + nb_a[i]], bt_b[a0:a0 + nb_b[i]])


def test_noalloc_equals_batch_on_two_calls_in_a_row():
    first = I.config3(N=300, m_hi=6000, seed=61)
    second = I.config3(N=57, m_hi=2500, seed=62)       # smaller: leftovers would show
    cases = [(first, native.BF, 0, 0), (second, native.RANDOM, 5, 0), (second, native.FF, 0, 1),
             (first, native.WF, 0, 0)]
    for batch, crit, seed, preopen in cases:
        db = native.DeviceBatch.from_host(batch)
        ref = _run(native.pack_batch, db, crit, seed, preopen)
        got = _run(native.pack_batch_noalloc, db, crit, seed, preopen)
        assert np.all(ref[0] == 0)
        _same(got, ref, db, batch)
        orc = oracle.pack_many(batch.w_all, batch.w_off, batch.B_all, batch.B_off, 1, crit, 0,
                               preopen, seed)
        _same(got, (orc.status, orc.bin_of_item, orc.bin_type, orc.num_bins, orc.total), db, batch)


def test_noalloc_rejects_what_it_cannot_hold():
    b = I.config3(N=4, m_hi=500, seed=63)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    assert native.pack_batch_noalloc(db, out, native.H1, native.BF, max_m=20_000) == native.ECAPACITY
    assert native.pack_batch_noalloc(db, out, native.H2, native.BF, 5) == native.EINVAL
    assert native.pack_batch_noalloc(db, out, native.H1, native.BF, 10) == native.ECAPACITY
    big = I.from_instances([(np.array([40_000, 3], dtype=np.int32), np.array([50_000], dtype=np.int32))])
    dbb = native.DeviceBatch.from_host(big)
    outb = native.DeviceResult.empty(dbb.N, dbb.total_items)
    assert native.pack_batch_noalloc(dbb, outb) == 0
    torch.cuda.synchronize()
    assert int(outb.status[0].item()) == native.ECAPACITY          # B_1 > 32767
