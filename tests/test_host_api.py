"""Host-side behaviour of the C ABI that needs no GPU: argument and parameter
validation (rejected before any device work), the launch-configuration table
and its file format, and the status strings.  Every call here returns before
the library touches CUDA, so the suite runs on machines without a GPU."""
import ctypes
import json

import numpy as np
import pytest

from paper_1602_08735_gb300 import native

EINVAL, ECAPACITY = native.EINVAL, native.ECAPACITY


@pytest.fixture(scope="module")
def lib():
    from paper_1602_08735_gb300 import build
    build.build()
    return native.load()


@pytest.fixture
def saved_config(lib):
    cfg = native.get_config()
    yield cfg
    native.set_config(**cfg)


def _p(**kw):
    base = dict(heuristic=native.H1, criterion=native.BF, sublist_size=0, preopen=0, flags=0, seed=0,
                max_open=0)
    base.update(kw)
    return native.Params(**base)


def _pack(lib, w, B, params, m=None, n=None):
    w = np.ascontiguousarray(w, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    m = len(w) if m is None else m
    n = len(B) if n is None else n
    boi = np.zeros(max(len(w), 1), dtype=np.int32)
    bt = np.zeros(max(len(w), 1), dtype=np.int32)
    nb, tot = ctypes.c_int64(0), ctypes.c_int64(0)
    wp = w.ctypes.data if len(w) else None
    Bp = B.ctypes.data if len(B) else None
    return lib.vsbpp_pack(wp, m, Bp, n, ctypes.byref(params), boi.ctypes.data, bt.ctypes.data,
                          ctypes.byref(nb), ctypes.byref(tot))


BAD_PARAMS = [dict(heuristic=0), dict(heuristic=3), dict(criterion=-1), dict(criterion=4),
              dict(preopen=2), dict(preopen=-1), dict(flags=4), dict(flags=-1), dict(sublist_size=-1),
              dict(heuristic=native.H2, sublist_size=13), dict(max_open=-1),
              dict(heuristic=native.H2, sublist_size=5, max_open=3),
              dict(flags=native.REMARK3, max_open=2)]


@pytest.mark.parametrize("bad", BAD_PARAMS)
def test_bad_parameters_rejected(lib, bad):
    """vsbpp_params outside the documented ranges: EINVAL from every entry
    point that takes them, before any device work."""
    w, B = [3, 4], [5]
    assert _pack(lib, w, B, _p(**bad)) == EINVAL
    one = np.zeros(2, dtype=np.int64)
    buf = np.zeros(4, dtype=np.int64)
    args = (1, buf.ctypes.data, one.ctypes.data, buf.ctypes.data, buf.ctypes.data, 2, ctypes.byref(_p(**bad)),
            buf.ctypes.data, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data, buf.ctypes.data, None)
    assert lib.vsbpp_pack_batch(*args) == EINVAL
    assert lib.vsbpp_pack_plain(*args) == EINVAL
    plan = ctypes.c_void_p()
    assert lib.vsbpp_plan_create(1, 2, 2, ctypes.byref(_p(**bad)), ctypes.byref(plan)) == EINVAL
    assert not plan.value


def test_bound_above_the_limit(lib):
    """A bounded-space bound above VSBPP_MAX_OPEN: ECAPACITY from every entry
    point, before any device work."""
    p = _p(max_open=native.MAX_OPEN + 1)
    assert _pack(lib, [3, 4], [5], p) == ECAPACITY
    one = np.zeros(2, dtype=np.int64)
    buf = np.zeros(4, dtype=np.int64)
    assert lib.vsbpp_pack_batch(1, buf.ctypes.data, one.ctypes.data, buf.ctypes.data, buf.ctypes.data, 2,
                                ctypes.byref(p), buf.ctypes.data, buf.ctypes.data, buf.ctypes.data,
                                buf.ctypes.data, buf.ctypes.data, None) == ECAPACITY


@pytest.mark.parametrize("case", ["n_neg", "off0", "w_off_down", "B_off_down", "max_m_small", "params"])
def test_host_batch_arguments(lib, case):
    """vsbpp_pack_batch_host checks its host CSR offsets and parameters
    before any device work: EINVAL."""
    w = np.array([1, 2, 3], dtype=np.int32)
    w_off = np.array([0, 2, 3], dtype=np.int64)
    B = np.array([5, 4], dtype=np.int32)
    B_off = np.array([0, 1, 2], dtype=np.int32)
    N, max_m, p = 2, 0, _p()
    if case == "n_neg":
        N = -1
    elif case == "off0":
        w_off = np.array([1, 2, 3], dtype=np.int64)
    elif case == "w_off_down":
        w_off = np.array([0, 3, 2], dtype=np.int64)
    elif case == "B_off_down":
        B_off = np.array([0, 2, 1], dtype=np.int32)
    elif case == "max_m_small":
        max_m = 1
    else:
        p = _p(criterion=7)
    out = native.HostResult.empty(2, 3)
    rc = lib.vsbpp_pack_batch_host(N, w.ctypes.data, w_off.ctypes.data, B.ctypes.data, B_off.ctypes.data,
                                   max_m, ctypes.byref(p), out.bin_of_item.ctypes.data,
                                   out.bin_type.ctypes.data, out.num_bins.ctypes.data, out.total.ctypes.data,
                                   out.status.ctypes.data)
    assert rc == EINVAL


@pytest.mark.parametrize("case", ["n0", "n33", "m_neg", "w_null", "B_null"])
def test_bad_instance_rejected(lib, case):
    """An instance outside the documented shape (n in 1..32, m >= 0, non-null
    arrays): EINVAL before any device work."""
    p = _p()
    if case == "n0":
        assert _pack(lib, [1, 2], [5], p, n=0) == EINVAL
    elif case == "n33":
        assert _pack(lib, [1, 2], list(range(99, 66, -1)), p) == EINVAL
    elif case == "m_neg":
        assert _pack(lib, [1, 2], [5], p, m=-1) == EINVAL
    elif case == "w_null":
        assert _pack(lib, [], [5], p, m=3) == EINVAL
    else:
        assert _pack(lib, [1, 2], [], p, n=1) == EINVAL


def test_empty_batch_is_a_no_op(lib):
    """N = 0 needs no arrays and does nothing."""
    z = [None] * 4
    assert lib.vsbpp_pack_batch(0, *z, 0, ctypes.byref(_p()), None, None, None, None, None, None) == 0
    bad_n = lib.vsbpp_pack_batch(-1, *z, 0, ctypes.byref(_p()), None, None, None, None, None, None)
    assert bad_n == EINVAL


def test_server_arguments(lib):
    """vsbpp_server_create: budget, slots and lanes (1..64) are checked first."""
    h = ctypes.c_void_p()
    for budget, slots, lanes, queued in ((0, 4, 2, 8), (1 << 20, 0, 2, 8), (1 << 20, 4, 0, 8),
                                         (1 << 20, 4, 65, 8), (1 << 20, 4, 2, 0)):
        assert lib.vsbpp_server_create(budget, slots, lanes, queued, ctypes.byref(h)) == EINVAL
        assert not h.value
    assert lib.vsbpp_server_create(1, 1, 1, 1, None) == EINVAL
    t = ctypes.c_uint64(0)
    w = np.array([1], dtype=np.int32)
    assert lib.vsbpp_server_submit(None, w.ctypes.data, 1, w.ctypes.data, 1, None, ctypes.byref(t)) == EINVAL
    assert lib.vsbpp_server_poll(None, 1, None, None, None, None, 0) == EINVAL
    assert lib.vsbpp_server_destroy(None) == 0


CONFIG_LIMITS = [dict(large_warps=3), dict(large_warps=64), dict(small_warps_per_block=0),
                 dict(small_warps_per_block=17), dict(small_m=-1), dict(chunk=16), dict(chunk=48),
                 dict(chunk=16384), dict(slot_pct=49), dict(slot_pct=201), dict(h2_blocks_per_sm=-1),
                 dict(h2_blocks_per_sm=33)]


@pytest.mark.parametrize("bad", CONFIG_LIMITS)
def test_config_limits(saved_config, bad):
    """vsbpp_set_config rejects each out-of-range field and leaves the table
    as it was."""
    with pytest.raises(native.VsbppError) as e:
        native.set_config(**bad)
    assert e.value.code == EINVAL
    assert native.get_config() == saved_config


def test_config_round_trip_and_file(saved_config, tmp_path):
    """set / get, then vsbpp_tune_save writes the table as JSON that
    vsbpp_tune_load reads back; a file from before h2_blocks_per_sm existed
    loads with that field unchanged; a file missing another field, or with
    an out-of-range value, is rejected and changes nothing."""
    want = dict(large_warps=4, small_m=512, small_warps_per_block=8, chunk=1024, slot_pct=130,
                h2_blocks_per_sm=3)
    native.set_config(**want)
    assert native.get_config() == want
    path = tmp_path / "tune.json"
    native.tune_save(str(path))
    assert json.loads(path.read_text()) == want
    native.set_config(**saved_config)
    native.tune_load(str(path))
    assert native.get_config() == want

    old = dict(want, large_warps=2)
    del old["h2_blocks_per_sm"]
    path.write_text(json.dumps(old))
    native.tune_load(str(path))
    assert native.get_config() == dict(old, h2_blocks_per_sm=3)

    before = native.get_config()
    for broken in ({k: v for k, v in want.items() if k != "chunk"}, dict(want, slot_pct=10)):
        path.write_text(json.dumps(broken))
        with pytest.raises(native.VsbppError):
            native.tune_load(str(path))
        assert native.get_config() == before
    with pytest.raises(native.VsbppError):
        native.tune_load(str(tmp_path / "missing.json"))


def test_status_strings(lib):
    """Every documented status has its own message; unknown codes say so."""
    codes = [0, native.EINVAL, native.ETOOBIG, native.ENOMEM, native.ECUDA, native.ETIMEDOUT,
             native.EBUSY, native.ENOTFOUND, ECAPACITY]
    msgs = [native.strerror(c) for c in codes]
    assert len(set(msgs)) == len(codes)
    assert native.strerror(12345) == "unknown status code"
