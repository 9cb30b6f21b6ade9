"""CUDA-graph plans, the autotuner, work counters and the serving loop
(GPU).  Every result is compared with the CPU oracle bit for bit."""
import os
import threading
import time

import numpy as np
import pytest

import oracle
from gpu_util import assert_same, run_oracle
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
    cfg = native.get_config()
    yield
    native.set_config(**cfg)


def _result(out, db):
    st, boi, bt, nb, tot = out.to_host(db.N, db.total_items)
    return oracle.BatchResult(st, boi, bt, nb, tot)


@pytest.mark.parametrize("h,c,s", [(1, 1, 0), (1, 0, 0), (1, 3, 0), (2, 1, 5), (1, 1, 10)])
def test_plan_replay_matches_oracle(h, c, s):
    b = I.config3(N=200, m_hi=3000, seed=21)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    plan = native.Plan(db.N, db.total_items, db.max_m, h, c, s, 0, 77)
    ref = run_oracle(b, h, c, s, 0, 77)
    for rep in range(3):                       # first run records, then replays
        out.status.fill_(123)
        out.bin_of_item.fill_(-5)
        plan.run(db, out)
        torch.cuda.synchronize()
        assert_same(b, _result(out, db), ref, f"plan rep {rep}")
    out2 = native.DeviceResult.empty(db.N, db.total_items)   # new pointers -> re-record
    plan.run(db, out2)
    torch.cuda.synchronize()
    assert_same(b, _result(out2, db), ref, "plan new pointers")
    plan.close()


def test_plan_captured_inside_user_graph():
    """plan_run allocates nothing, so it can itself sit inside a user capture."""
    b = I.config3(N=64, m_hi=2000, seed=5)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    plan = native.Plan(db.N, db.total_items, db.max_m, 1, 1)
    plan.run(db, out)                          # record the plan's own graph first
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        plan.run(db, out, s)
    out.status.fill_(9)
    g.replay()
    torch.cuda.synchronize()
    assert_same(b, _result(out, db), run_oracle(b, 1, 1), "user graph")
    plan.close()


def test_autotune_keeps_results_exact(tmp_path):
    b = I.config3(N=128, m_hi=4000, seed=31)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    before = native.get_config()
    cfg, ms = native.autotune(db, out, 1, 1)
    assert ms > 0 and cfg == native.get_config()
    path = str(tmp_path / "tune.json")
    native.tune_save(path)
    native.set_config(**before)
    native.tune_load(path)
    assert native.get_config() == cfg
    rc = native.pack_batch(db, out, 1, 1)
    assert rc == 0
    torch.cuda.synchronize()
    assert_same(b, _result(out, db), run_oracle(b, 1, 1), "after autotune")
    native.set_config(**before)


def test_counters_count_items_and_fit_tests():
    b = I.config3(N=50, m_hi=1500, seed=4)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    native.counters_enable(True)
    native.counters_read(reset=True)
    assert native.pack_batch(db, out, 1, 1) == 0
    c1 = native.counters_read(reset=True)
    assert native.pack_plain(db, out, 1, 1) == 0
    c2 = native.counters_read(reset=True)
    native.counters_enable(False)
    assert c1["items"] == b.total_items == c2["items"]
    assert c1["fit_tests"] == c2["fit_tests"] > 0


def test_server_results_alone_and_in_the_mix():
    rng = np.random.default_rng(55)
    reqs = [I.config5_request(rng, r, 100, 20_000) for r in range(40)]
    with native.Server(device_mem_budget=64 << 20, max_slots=16, lanes=4) as srv:
        # each request alone
        alone = []
        for (w, B) in reqs:
            t = srv.submit(w, B, 1, 1)
            rc, res = srv.poll(t)
            assert rc == 0
            alone.append(res)
        # all of them in flight together, criteria mixed in
        tickets = [srv.submit(w, B, 1, 1) for (w, B) in reqs]
        mixed = [srv.poll(t)[1] for t in tickets]
        st = srv.stats()
    assert st["completed"] == 2 * len(reqs)
    assert st["p99_us"] >= st["p50_us"] > 0
    for (w, B), a, m in zip(reqs, alone, mixed):
        ref = oracle.pack(w, B, 1, 1)
        assert a.status == m.status == 0
        assert a.bin_of_item.tobytes() == m.bin_of_item.tobytes() == ref.bin_of_item.tobytes()
        assert a.bin_type.tobytes() == m.bin_type.tobytes() == ref.bin_type.tobytes()
        assert a.total == m.total == ref.total


def test_server_large_requests_in_the_mix():
    """Requests across config 5's whole range: the largest (6*10^4 and 10^5
    items, B_1 = 150) are packed in the one-warp kernel's 16-bit slots (or in
    global memory if they outgrow them); all are submitted at once in
    increasing size, so lanes grow their scratch while other requests are in
    flight.  Each result equals the oracle's."""
    rng = np.random.default_rng(56)
    reqs = [I.config5_request(rng, r, 100, 20_000) for r in range(24)]
    reqs += [I.config5_request(rng, 0, 60_000, 60_000), I.config5_request(rng, 1, 100_000, 100_000)]
    reqs.sort(key=lambda x: len(x[0]))
    with native.Server(device_mem_budget=256 << 20, max_slots=16, lanes=4) as srv:
        tickets = [srv.submit(w, B, 1, 1) for (w, B) in reqs]
        got = [srv.poll(t) for t in tickets]
    for (w, B), (rc, res) in zip(reqs, got):
        ref = oracle.pack(w, B, 1, 1)
        assert rc == 0 and res.total == ref.total, len(w)
        assert res.bin_of_item.tobytes() == ref.bin_of_item.tobytes(), len(w)
        assert res.bin_type.tobytes() == ref.bin_type.tobytes(), len(w)


def test_server_concurrent_submitters_and_errors():
    rng = np.random.default_rng(9)
    with native.Server(device_mem_budget=8 << 20, max_slots=4, lanes=2) as srv:
        with pytest.raises(native.VsbppError) as e:
            srv.submit(np.ones(2_000_000, dtype=np.int32), [5])      # > budget alone
        assert e.value.code == native.ECAPACITY
        rc, _ = srv.poll(987654321, 0)
        assert rc == native.ENOTFOUND
        results = {}

        def client(k):
            r2 = np.random.default_rng(100 + k)
            for r in range(10):
                w, B = I.config5_request(r2, r, 100, 5000)
                crit = r % 3
                t = srv.submit(w, B, 1, crit)
                results[(k, r)] = (w, B, crit, t)

        th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        for (k, r), (w, B, crit, t) in results.items():
            rc, res = srv.poll(t, 10_000_000)
            ref = oracle.pack(w, B, 1, crit)
            assert rc == 0 and res.total == ref.total
            assert res.bin_of_item.tolist() == ref.bin_of_item.tolist()
        # invalid request: status comes back through poll
        t = srv.submit([0, 1], [5])
        rc, _ = srv.poll(t)
        assert rc == native.EINVAL


@pytest.mark.parametrize("h,s", [(1, 0), (1, 7), (2, 5), (2, 4), (2, 6), (2, 7)])
def test_counters_match_the_method_fit_tests(h, s):
    """The kernels' fit-test counters equal the oracle's count of Rule 4 fit
    tests (every bin alive when an item arrives; every permutation for the
    second heuristic), instance by instance summed."""
    b = I.config3(N=12, m_hi=700, seed=21)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    native.counters_enable(True)
    try:
        for crit in (native.FF, native.BF, native.WF, native.RANDOM):
            native.counters_read(reset=True)
            assert native.pack_batch(db, out, h, crit, s, seed=9) == 0
            got = native.counters_read(reset=True)
            want = sum(oracle.fit_tests(*b.instance(i), h, crit, s, 0, 9) for i in range(b.N))
            assert got["fit_tests"] == want, (h, s, crit)
            assert got["items"] == b.total_items
    finally:
        native.counters_enable(False)


def test_counters_second_heuristic_wide_capacities():
    """Capacities above 4095 take the second heuristic's wide-slot path; its
    counters follow the same definition."""
    rng = np.random.default_rng(22)
    inst = [(rng.integers(1, 9001, size=int(m)).astype(np.int32), np.array([9000, 5000, 4100], dtype=np.int32))
            for m in rng.integers(20, 200, size=6)]
    b = I.from_instances(inst)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    native.counters_enable(True)
    try:
        for crit in (native.FF, native.BF, native.WF, native.RANDOM):
            native.counters_read(reset=True)
            assert native.pack_batch(db, out, 2, crit, 5, seed=3) == 0
            got = native.counters_read(reset=True)
            want = sum(oracle.fit_tests(*b.instance(i), 2, crit, 5, 0, 3) for i in range(b.N))
            assert got["fit_tests"] == want, crit
    finally:
        native.counters_enable(False)


def test_kernel_timing_hook():
    """One event-timed duration per uncaptured batched call, none for plan
    replays (captured launches) and none while disabled."""
    b = I.config3(N=30, m_hi=2000, seed=23)
    db = native.DeviceBatch.from_host(b)
    out = native.DeviceResult.empty(db.N, db.total_items)
    native.kernel_timing_enable(True)
    try:
        for (h, c, s) in ((1, native.BF, 0), (2, native.BF, 5), (1, native.FF, 0)):
            assert native.pack_batch(db, out, h, c, s) == 0
        t = native.kernel_timing_read()
        assert len(t) == 3 and all(x > 0 for x in t)
        assert native.kernel_timing_read() == []
        pl = native.Plan(db.N, db.total_items, db.max_m, 1, native.BF, 0)
        try:
            pl.run(db, out)
            pl.run(db, out)
        finally:
            pl.close()
        assert len(native.kernel_timing_read()) <= 1     # at most the call made while recording
    finally:
        native.kernel_timing_enable(False)
    assert native.pack_batch(db, out, 1, native.BF, 0) == 0
    assert native.kernel_timing_read() == []


def test_two_host_threads_on_two_streams():
    """Calls on different streams run at once (each stream's scratch has its
    own lock); every result still equals the oracle's."""
    import threading
    b = I.config3(N=160, m_hi=4000, seed=77)
    ref = run_oracle(b, 1, native.BF)
    res, errs = {}, []

    def work(k):
        try:
            st = torch.cuda.Stream()
            db = native.DeviceBatch.from_host(b)
            out = native.DeviceResult.empty(db.N, db.total_items)
            for _ in range(3):
                rc = native.pack_batch(db, out, 1, native.BF, stream=st)
                assert rc == 0
            st.synchronize()
            res[k] = out.to_host(db.N, db.total_items)
        except Exception as e:          # reported below
            errs.append(e)

    th = [threading.Thread(target=work, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for k in range(2):
        st_, boi, bt, nb, tot = res[k]
        assert_same(b, oracle.BatchResult(st_, boi, bt, nb, tot), ref, f"thread {k}")
