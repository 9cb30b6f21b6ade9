"""The paper-faithful and next-step variants against the oracle, element by
element (bit-exact integers):

  * Remark 3 of Section 6.3 as a condition on Rule 5 (VSBPP_REMARK3) in every
    kernel that packs with it: the group kernel (one membrane system per
    instance, sublists), the global-memory kernel, the second heuristic's
    generic kernel and the exhaustive search (7..12 items);
  * the offline pre-sort (VSBPP_PRESORT, reading G16) on both heuristics,
    the plain and batched paths, including which error code a batch with
    several offending items reports;
  * the bounded-space variant (max_open, reading G15) for every criterion,
    bound and start, on the batched and plain paths;
  * the host-memory batch call (pinned and pageable buffers) against the
    device-memory one."""
import numpy as np
import pytest

import oracle
from gpu_util import assert_same, run_batch, run_oracle
from paper_1602_08735_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1602_08735_gb300 import native  # noqa: E402

CRITS = [native.FF, native.BF, native.WF, native.RANDOM]
R3, PS = native.REMARK3, native.PRESORT


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()


def _fuzz(seed, N, m_hi, cap_hi=200, n_hi=6):
    rng = np.random.default_rng(seed)
    inst = []
    for _ in range(N):
        m = int(rng.integers(0, m_hi + 1))
        inst.append(I.random_instance(rng, m, int(rng.integers(1, n_hi + 1)), cap_hi))
    return I.from_instances(inst)


# ------------------------------------------------------------------ Remark 3
@pytest.mark.parametrize("crit", CRITS)
def test_remark3_configs_1_to_3(crit):
    for name, b in (("cfg1", I.config1()), ("cfg2u", I.config2("u")), ("cfg2m", I.config2("m")),
                    ("cfg3", I.config3())):
        assert_same(b, run_batch(b, 1, crit, seed=9, flags=R3), run_oracle(b, 1, crit, seed=9, flags=R3),
                    f"{name} H1 remark3 c{crit}")
    b = I.config3()
    assert_same(b, run_batch(b, 2, crit, 5, seed=9, flags=R3), run_oracle(b, 2, crit, 5, seed=9, flags=R3),
                f"cfg3 H2 remark3 c{crit}")


@pytest.mark.parametrize("preopen", [0, 1])
def test_remark3_every_path(preopen):
    """Sublists (group kernel in compose mode), the plain path, the second
    heuristic's sublist sizes 1..6, and a system beyond shared memory."""
    b = _fuzz(30 + preopen, 60, 400)
    for crit in CRITS:
        ref = run_oracle(b, 1, crit, 0, preopen, 4, R3)
        assert_same(b, run_batch(b, 1, crit, 0, preopen, 4, flags=R3), ref, f"r3 h1 c{crit}")
        assert_same(b, run_batch(b, 1, crit, 0, preopen, 4, plain=True, flags=R3), ref, f"r3 plain c{crit}")
        assert_same(b, run_batch(b, 1, crit, 10, preopen, 4, flags=R3),
                    run_oracle(b, 1, crit, 10, preopen, 4, R3), f"r3 s10 c{crit}")
        for s in (1, 3, 5, 6):
            assert_same(b, run_batch(b, 2, crit, s, preopen, 4, flags=R3),
                        run_oracle(b, 2, crit, s, preopen, 4, R3), f"r3 h2 s{s} c{crit}")
    rng = np.random.default_rng(40 + preopen)
    big = I.from_instances([(I.mixture_weights(rng, 0.8, (1, 100), (400, 1000), 60_000), I.CFG4_B)])
    for crit in CRITS:
        assert_same(big, run_batch(big, 1, crit, 0, preopen, 2, flags=R3),
                    run_oracle(big, 1, crit, 0, preopen, 2, R3), f"r3 global memory c{crit}")


def test_remark3_exhaustive_search():
    b = _fuzz(50, 6, 16, cap_hi=60)
    for s in (7, 8):
        for crit in CRITS:
            assert_same(b, run_batch(b, 2, crit, s, 0, 6, flags=R3), run_oracle(b, 2, crit, s, 0, 6, R3),
                        f"r3 h2x s{s} c{crit}")


def test_remark3_changes_results():
    """The option is not a no-op on these workloads (else the tests above
    would prove nothing about it)."""
    b = I.config2("m")
    a = run_oracle(b, 1, native.FF, flags=R3)
    z = run_oracle(b, 1, native.FF)
    assert int(a.total[0]) != int(z.total[0])


# ----------------------------------------------------------------- pre-sort
@pytest.mark.parametrize("crit", CRITS)
def test_presort_configs_1_to_3(crit):
    for name, b in (("cfg1", I.config1()), ("cfg2u", I.config2("u")), ("cfg3", I.config3())):
        for h, s in ((1, 0), (2, 5)):
            assert_same(b, run_batch(b, h, crit, s, seed=11, flags=PS), run_oracle(b, h, crit, s, seed=11, flags=PS),
                        f"{name} presort h{h} c{crit}")


@pytest.mark.parametrize("preopen", [0, 1])
def test_presort_paths(preopen):
    """Plain path, sublists, Remark 3 together with the pre-sort, wide
    capacities (several radix passes) and the global-memory kernel."""
    b = _fuzz(60 + preopen, 80, 500, cap_hi=70_000)
    for crit in CRITS:
        ref = run_oracle(b, 1, crit, 0, preopen, 3, PS)
        assert_same(b, run_batch(b, 1, crit, 0, preopen, 3, flags=PS), ref, f"ps c{crit}")
        assert_same(b, run_batch(b, 1, crit, 0, preopen, 3, plain=True, flags=PS), ref, f"ps plain c{crit}")
        assert_same(b, run_batch(b, 1, crit, 10, preopen, 3, flags=PS),
                    run_oracle(b, 1, crit, 10, preopen, 3, PS), f"ps s10 c{crit}")
        assert_same(b, run_batch(b, 1, crit, 0, preopen, 3, flags=PS | R3),
                    run_oracle(b, 1, crit, 0, preopen, 3, PS | R3), f"ps+r3 c{crit}")
    rng = np.random.default_rng(70 + preopen)
    big = I.from_instances([(I.mixture_weights(rng, 0.8, (1, 100), (400, 1000), 50_000), I.CFG4_B)])
    for crit in (native.BF, native.WF):
        assert_same(big, run_batch(big, 1, crit, 0, preopen, flags=PS), run_oracle(big, 1, crit, 0, preopen, flags=PS),
                    f"ps global memory c{crit}")


def test_presort_exhaustive_search():
    """The pre-sort ahead of the exhaustive 7..8-item permutation search
    (Remark 3 alongside), element by element against the oracle."""
    b = _fuzz(55, 6, 16, cap_hi=60)
    for s in (7, 8):
        for crit in CRITS:
            for flags in (PS, PS | R3):
                assert_same(b, run_batch(b, 2, crit, s, 0, 6, flags=flags), run_oracle(b, 2, crit, s, 0, 6, flags),
                            f"ps h2x s{s} c{crit} flags{flags}")


def test_presort_reports_the_callers_first_offender():
    """Validation runs in the caller's order: a zero weight before a too-heavy
    one is EINVAL, the other way round ETOOBIG (sorting would swap them)."""
    B = np.array([100, 50], dtype=np.int32)
    b = I.from_instances([(np.array([5, 0, 101, 7], dtype=np.int32), B),
                          (np.array([5, 101, 0, 7], dtype=np.int32), B),
                          (np.array([9, 60, 3], dtype=np.int32), B)])
    got = run_batch(b, 1, native.BF, flags=PS)
    assert got.status.tolist() == [native.EINVAL, native.ETOOBIG, 0]
    assert_same(b, got, run_oracle(b, 1, native.BF, flags=PS), "ps errors")
    assert native.pack([5, 0, 101], B, flags=PS).status == native.EINVAL


# ------------------------------------------------------------- bounded space
@pytest.mark.parametrize("K", [1, 2, 3, 7, 32])
def test_bounded_space_vs_oracle(K):
    b = _fuzz(80 + K, 120, 800, cap_hi=300)
    for crit in CRITS:
        for preopen in (0, 1):
            ref = run_oracle(b, 1, crit, 0, preopen, 5, max_open=K)
            assert_same(b, run_batch(b, 1, crit, 0, preopen, 5, max_open=K), ref, f"K{K} c{crit} p{preopen}")
    assert_same(b, run_batch(b, 1, native.BF, 0, 0, 5, plain=True, max_open=K),
                run_oracle(b, 1, native.BF, 0, 0, 5, max_open=K), f"K{K} plain")


def test_bounded_space_large_and_presorted():
    """Config 3 in full and a 10^5-item system, with and without pre-sort."""
    b = I.config3()
    for crit in (native.FF, native.BF, native.WF):
        assert_same(b, run_batch(b, 1, crit, max_open=8), run_oracle(b, 1, crit, max_open=8), f"cfg3 K8 c{crit}")
    rng = np.random.default_rng(91)
    big = I.from_instances([(I.uniform_weights(rng, 1, 150, 100_000), I.CFG2_B)])
    for crit in CRITS:
        for flags in (0, PS):
            assert_same(big, run_batch(big, 1, crit, seed=2, flags=flags, max_open=32),
                        run_oracle(big, 1, crit, seed=2, flags=flags, max_open=32), f"big K32 c{crit} f{flags}")


def test_bounded_space_counters_match_oracle():
    """Fit tests of the bounded kernel = the oracle's (one per open bin)."""
    b = _fuzz(95, 40, 300)
    native.counters_enable(True)
    native.counters_read(reset=True)
    run_batch(b, 1, native.BF, max_open=4)
    got = native.counters_read(reset=True)
    native.counters_enable(False)
    want = sum(oracle.fit_tests(*b.instance(i), 1, native.BF, max_open=4) for i in range(b.N))
    assert got["fit_tests"] == want and got["items"] == b.total_items


# --------------------------------------------------------- host-memory batch
@pytest.mark.parametrize("pinned", [False, True])
def test_host_batch_equals_device_batch(pinned):
    b = I.config3(N=300, m_hi=5000, seed=97)
    for (h, c, s, flags, K) in ((1, native.BF, 0, 0, 0), (1, native.WF, 0, PS, 0), (2, native.BF, 5, 0, 0),
                                (1, native.FF, 0, 0, 4)):
        ref = run_batch(b, h, c, s, flags=flags, max_open=K)
        arrs = [b.w_all, b.w_off, b.B_all, b.B_off]
        out = native.HostResult.empty(b.N, b.total_items)
        if pinned:
            arrs = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in arrs]
            out = native.HostResult(*(torch.from_numpy(x).pin_memory() for x in
                                      (out.status, out.bin_of_item, out.bin_type, out.num_bins, out.total)))
        rc = native.pack_batch_host(*arrs, out, h, c, s, flags=flags, max_open=K)
        assert rc == 0, native.strerror(rc)
        got = oracle.BatchResult(*(np.asarray(x)[:n] for x, n in
                                   ((out.status, b.N), (out.bin_of_item, b.total_items),
                                    (out.bin_type, b.total_items), (out.num_bins, b.N), (out.total, b.N))))
        assert_same(b, got, ref, f"host batch h{h} c{c} pinned={pinned}")


def test_host_batch_calls_from_several_threads():
    """Four host threads call vsbpp_pack_batch_host at once (each call holds
    a stream and staging the library lends it alone); every result equals the
    oracle, on two rounds in a row."""
    from concurrent.futures import ThreadPoolExecutor
    b = I.config3(N=256, m_hi=4000, seed=98)
    jobs = [(1, native.FF, 0), (1, native.BF, 0), (1, native.WF, 0), (2, native.BF, 5)]
    refs = [run_oracle(b, h, c, s) for (h, c, s) in jobs]
    arrs = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (b.w_all, b.w_off, b.B_all, b.B_off)]
    dev = torch.cuda.current_device()

    def one(k):
        torch.cuda.set_device(dev)
        h, c, s = jobs[k]
        out = native.HostResult.empty(b.N, b.total_items)
        return native.pack_batch_host(*arrs, out, h, c, s), out

    with ThreadPoolExecutor(len(jobs)) as ex:
        for rnd in range(2):
            for k, (rc, out) in enumerate(ex.map(one, range(len(jobs)))):
                assert rc == 0, native.strerror(rc)
                got = oracle.BatchResult(*(np.asarray(x)[:n] for x, n in
                                           ((out.status, b.N), (out.bin_of_item, b.total_items),
                                            (out.bin_type, b.total_items), (out.num_bins, b.N), (out.total, b.N))))
                assert_same(b, got, refs[k], f"threaded host batch {jobs[k]} round {rnd}")


def test_server_with_options():
    """Requests with the pre-sort, Remark 3 and a bound, served in the mix."""
    rng = np.random.default_rng(99)
    reqs = [I.config5_request(rng, r, 100, 3000) for r in range(24)]
    opts = [dict(flags=PS), dict(flags=R3), dict(max_open=5), dict()]
    with native.Server(device_mem_budget=1 << 30, max_slots=16, lanes=4) as srv:
        tickets = [srv.submit(w, B, 1, native.BF, **opts[k % 4]) for k, (w, B) in enumerate(reqs)]
        for k, (t, (w, B)) in enumerate(zip(tickets, reqs)):
            rc, got = srv.poll(t)
            o = opts[k % 4]
            ref = oracle.pack(w, B, 1, native.BF, flags=o.get("flags", 0), max_open=o.get("max_open", 0))
            assert rc == 0
            assert got.bin_of_item.tolist() == ref.bin_of_item.tolist() and got.total == ref.total
