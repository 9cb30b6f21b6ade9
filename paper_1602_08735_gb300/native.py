"""Thin ctypes binding over ``libvsbpp.so`` (include/vsbpp.h).

Argument marshalling only: every step of the packing runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  When the library
has not been built, loading fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvsbpp.so")

FF, BF, WF, RANDOM = 0, 1, 2, 3
H1, H2 = 1, 2
OK, EINVAL, ETOOBIG, ENOMEM, ECUDA, ETIMEDOUT, EBUSY, ENOTFOUND, ECAPACITY = 0, -1, -2, -3, -4, -5, -6, -7, -8
MAX_TYPES = 32
MAX_OPEN = 32                 # largest bound of the bounded-space variant
REMARK3, PRESORT = 1, 2       # option flags (vsbpp_params.flags)

# Every entry point declared in include/vsbpp.h.
EXPORTS = (
    "vsbpp_strerror", "vsbpp_version", "vsbpp_last_cuda_error",
    "vsbpp_pack", "vsbpp_pack_device", "vsbpp_pack_batch", "vsbpp_pack_plain",
    "vsbpp_pack_batch_host", "vsbpp_pack_batch_noalloc", "vsbpp_shard",
    "vsbpp_counters_enable", "vsbpp_counters_read",
    "vsbpp_kernel_timing_enable", "vsbpp_kernel_timing_read",
    "vsbpp_plan_create", "vsbpp_plan_run", "vsbpp_plan_destroy",
    "vsbpp_get_config", "vsbpp_set_config", "vsbpp_autotune", "vsbpp_tune_save", "vsbpp_tune_load",
    "vsbpp_server_create", "vsbpp_server_submit", "vsbpp_server_poll", "vsbpp_server_stats",
    "vsbpp_server_destroy",
)


class VsbppError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class Params(ctypes.Structure):
    _fields_ = [("heuristic", ctypes.c_int32), ("criterion", ctypes.c_int32),
                ("sublist_size", ctypes.c_int64), ("preopen", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("seed", ctypes.c_uint64), ("max_open", ctypes.c_int64)]


class Config(ctypes.Structure):
    _fields_ = [("large_warps", ctypes.c_int32), ("small_m", ctypes.c_int32),
                ("small_warps_per_block", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("slot_pct", ctypes.c_int32), ("h2_blocks_per_sm", ctypes.c_int32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Counters(ctypes.Structure):
    _fields_ = [("items", ctypes.c_uint64), ("fit_tests", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("items_packed", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("busy_s", ctypes.c_double),
                ("wait_p50_us", ctypes.c_double), ("wait_p99_us", ctypes.c_double),
                ("service_p50_us", ctypes.c_double), ("service_p99_us", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Open the CUDA library (build it first with ``paper_1602_08735_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run paper_1602_08735_gb300.build.build() first "
                              "(the library has no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, i32p, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        pp = ctypes.POINTER(Params)
        lib.vsbpp_strerror.restype = ctypes.c_char_p
        lib.vsbpp_strerror.argtypes = [ctypes.c_int]
        lib.vsbpp_version.restype = ctypes.c_int
        lib.vsbpp_last_cuda_error.restype = ctypes.c_int
        lib.vsbpp_pack.restype = ctypes.c_int
        lib.vsbpp_pack.argtypes = [vp, i64, vp, i32, pp, vp, vp, i64p, i64p]
        lib.vsbpp_pack_device.restype = ctypes.c_int
        lib.vsbpp_pack_device.argtypes = [vp, i64, vp, i32, pp, vp, vp, vp, vp, vp, vp]
        for name in ("vsbpp_pack_batch", "vsbpp_pack_plain", "vsbpp_pack_batch_noalloc"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int
            f.argtypes = [i64, vp, vp, vp, vp, i64, pp, vp, vp, vp, vp, vp, vp]
        lib.vsbpp_shard.restype = ctypes.c_int
        lib.vsbpp_shard.argtypes = [i64, vp, i32, vp, vp]
        lib.vsbpp_pack_batch_host.restype = ctypes.c_int
        lib.vsbpp_pack_batch_host.argtypes = [i64, vp, vp, vp, vp, i64, pp, vp, vp, vp, vp, vp]
        if hasattr(lib, "vsbpp_plan_create"):
            lib.vsbpp_plan_create.restype = ctypes.c_int
            lib.vsbpp_plan_create.argtypes = [i64, i64, i64, pp, ctypes.POINTER(vp)]
            lib.vsbpp_plan_run.restype = ctypes.c_int
            lib.vsbpp_plan_run.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            lib.vsbpp_plan_destroy.restype = ctypes.c_int
            lib.vsbpp_plan_destroy.argtypes = [vp]
        lib.vsbpp_counters_enable.restype = ctypes.c_int
        lib.vsbpp_counters_enable.argtypes = [ctypes.c_int]
        lib.vsbpp_counters_read.restype = ctypes.c_int
        lib.vsbpp_counters_read.argtypes = [ctypes.POINTER(Counters), ctypes.c_int]
        lib.vsbpp_kernel_timing_enable.restype = ctypes.c_int
        lib.vsbpp_kernel_timing_enable.argtypes = [ctypes.c_int]
        lib.vsbpp_kernel_timing_read.restype = ctypes.c_int
        lib.vsbpp_kernel_timing_read.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_int32)]
        lib.vsbpp_get_config.restype = ctypes.c_int
        lib.vsbpp_get_config.argtypes = [ctypes.POINTER(Config)]
        lib.vsbpp_set_config.restype = ctypes.c_int
        lib.vsbpp_set_config.argtypes = [ctypes.POINTER(Config)]
        if hasattr(lib, "vsbpp_autotune"):
            lib.vsbpp_autotune.restype = ctypes.c_int
            lib.vsbpp_autotune.argtypes = [i64, vp, vp, vp, vp, i64, pp, vp, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_double)]
            lib.vsbpp_tune_save.restype = ctypes.c_int
            lib.vsbpp_tune_save.argtypes = [ctypes.c_char_p]
            lib.vsbpp_tune_load.restype = ctypes.c_int
            lib.vsbpp_tune_load.argtypes = [ctypes.c_char_p]
        if hasattr(lib, "vsbpp_server_create"):
            lib.vsbpp_server_create.restype = ctypes.c_int
            lib.vsbpp_server_create.argtypes = [ctypes.c_size_t, i32, i32, i32, ctypes.POINTER(vp)]
            lib.vsbpp_server_submit.restype = ctypes.c_int
            lib.vsbpp_server_submit.argtypes = [vp, vp, i64, vp, i32, pp, ctypes.POINTER(ctypes.c_uint64)]
            lib.vsbpp_server_poll.restype = ctypes.c_int
            lib.vsbpp_server_poll.argtypes = [vp, ctypes.c_uint64, vp, vp, i64p, i64p, i64]
            lib.vsbpp_server_stats.restype = ctypes.c_int
            lib.vsbpp_server_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
            lib.vsbpp_server_destroy.restype = ctypes.c_int
            lib.vsbpp_server_destroy.argtypes = [vp]
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().vsbpp_strerror(int(code)).decode()
    except ImportError:
        return f"status {code}"


def make_params(heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
                preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> Params:
    return Params(heuristic, criterion, sublist_size, preopen, flags, seed & (2**64 - 1), max_open)


def _ptr(x) -> int | None:
    """Address of a numpy array or torch tensor (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


@dataclass
class Packing:
    status: int
    bin_of_item: np.ndarray
    bin_type: np.ndarray
    num_bins: int
    total: int


def pack(w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0, preopen: int = 0,
         seed: int = 0, flags: int = 0, max_open: int = 0) -> Packing:
    """Host-memory call (vsbpp_pack): numpy in, numpy out, synchronous."""
    lib = load()
    w = np.ascontiguousarray(w, dtype=np.int32)
    B = np.ascontiguousarray(B, dtype=np.int32)
    m = int(w.shape[0])
    boi = np.full(max(m, 1), -1, dtype=np.int32)
    bt = np.full(max(m, 1), -1, dtype=np.int32)
    nb = ctypes.c_int64(0)
    tot = ctypes.c_int64(0)
    p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
    wb = w if m > 0 else np.zeros(1, dtype=np.int32)
    Bb = B if B.shape[0] > 0 else np.zeros(1, dtype=np.int32)
    rc = lib.vsbpp_pack(_ptr(wb), m, _ptr(Bb), int(B.shape[0]), ctypes.byref(p), _ptr(boi), _ptr(bt),
                        ctypes.byref(nb), ctypes.byref(tot))
    k = int(nb.value)
    return Packing(int(rc), boi[:m].copy(), bt[:k].copy(), k, int(tot.value))


def pack_device(w, B, bin_of_item, bin_type, num_bins, total, status, heuristic: int = H1,
                criterion: int = BF, sublist_size: int = 0, preopen: int = 0, seed: int = 0,
                stream=None, flags: int = 0, max_open: int = 0) -> int:
    """Device-memory call (vsbpp_pack_device) on torch CUDA tensors; async."""
    lib = load()
    p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
    return int(lib.vsbpp_pack_device(_ptr(w), int(w.numel()), _ptr(B), int(B.numel()), ctypes.byref(p),
                                     _ptr(bin_of_item), _ptr(bin_type), _ptr(num_bins), _ptr(total),
                                     _ptr(status), _stream_handle(stream)))


@dataclass
class DeviceBatch:
    """A CSR batch resident on the GPU (torch tensors)."""
    w_all: object
    w_off: object
    B_all: object
    B_off: object
    N: int
    total_items: int
    max_m: int

    @classmethod
    def from_host(cls, batch, device="cuda"):
        import torch
        w_off = np.asarray(batch.w_off, dtype=np.int64)
        ms = np.diff(w_off)
        return cls(torch.from_numpy(np.ascontiguousarray(batch.w_all, dtype=np.int32)).to(device),
                   torch.from_numpy(w_off).to(device),
                   torch.from_numpy(np.ascontiguousarray(batch.B_all, dtype=np.int32)).to(device),
                   torch.from_numpy(np.ascontiguousarray(batch.B_off, dtype=np.int32)).to(device),
                   int(w_off.shape[0]) - 1, int(w_off[-1]), int(ms.max()) if ms.size else 0)


@dataclass
class DeviceResult:
    bin_of_item: object
    bin_type: object
    num_bins: object
    total: object
    status: object

    @classmethod
    def empty(cls, N: int, total_items: int, device="cuda"):
        import torch
        return cls(torch.empty(max(total_items, 1), dtype=torch.int32, device=device),
                   torch.empty(max(total_items, 1), dtype=torch.int32, device=device),
                   torch.empty(max(N, 1), dtype=torch.int64, device=device),
                   torch.empty(max(N, 1), dtype=torch.int64, device=device),
                   torch.empty(max(N, 1), dtype=torch.int32, device=device))

    def to_host(self, N: int, total_items: int):
        return (self.status[:N].cpu().numpy(), self.bin_of_item[:total_items].cpu().numpy(),
                self.bin_type[:total_items].cpu().numpy(), self.num_bins[:N].cpu().numpy(),
                self.total[:N].cpu().numpy())


def _batch_call(fn_name, db: DeviceBatch, out: DeviceResult, params: Params, stream, max_m=None) -> int:
    lib = load()
    fn = getattr(lib, fn_name)
    return int(fn(db.N, _ptr(db.w_all), _ptr(db.w_off), _ptr(db.B_all), _ptr(db.B_off),
                  int(db.max_m if max_m is None else max_m), ctypes.byref(params),
                  _ptr(out.bin_of_item), _ptr(out.bin_type), _ptr(out.num_bins), _ptr(out.total),
                  _ptr(out.status), _stream_handle(stream)))


def pack_batch(db: DeviceBatch, out: DeviceResult, heuristic: int = H1, criterion: int = BF,
               sublist_size: int = 0, preopen: int = 0, seed: int = 0, stream=None, max_m=None,
               flags: int = 0, max_open: int = 0) -> int:
    """Batched persistent launch (vsbpp_pack_batch); async on ``stream``."""
    return _batch_call("vsbpp_pack_batch", db, out,
                       make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open),
                       stream, max_m)


def pack_plain(db: DeviceBatch, out: DeviceResult, heuristic: int = H1, criterion: int = BF,
               sublist_size: int = 0, preopen: int = 0, seed: int = 0, stream=None, max_m=None,
               flags: int = 0, max_open: int = 0) -> int:
    """One launch per instance (vsbpp_pack_plain); async on ``stream``."""
    return _batch_call("vsbpp_pack_plain", db, out,
                       make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open),
                       stream, max_m)


def pack_batch_noalloc(db: DeviceBatch, out: DeviceResult, heuristic: int = H1, criterion: int = BF,
                       sublist_size: int = 0, preopen: int = 0, seed: int = 0, stream=None,
                       max_m=None, flags: int = 0, max_open: int = 0) -> int:
    """vsbpp_pack_batch_noalloc: the batched pack with the library's static
    device scratch (for callers that cannot allocate); async on ``stream``."""
    return _batch_call("vsbpp_pack_batch_noalloc", db, out,
                       make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open),
                       stream, max_m)


def shard(w_off, world: int):
    """vsbpp_shard: (rank_of[N] int32, items_of_rank[world] int64) for a
    batch's host CSR offsets split over `world` processes."""
    w_off = np.ascontiguousarray(w_off, dtype=np.int64)
    N = int(w_off.shape[0]) - 1
    rank_of = np.zeros(max(N, 1), dtype=np.int32)
    items = np.zeros(max(world, 1), dtype=np.int64)
    rc = load().vsbpp_shard(N, _ptr(w_off), int(world), _ptr(rank_of), _ptr(items))
    if rc != 0:
        raise VsbppError(rc, "vsbpp_shard")
    return rank_of[:N].copy(), items[:world].copy()


@dataclass
class HostResult:
    """Outputs of a host-memory batch call (numpy, or pinned torch tensors)."""
    status: object
    bin_of_item: object
    bin_type: object
    num_bins: object
    total: object

    @classmethod
    def empty(cls, N: int, total_items: int):
        return cls(np.zeros(max(N, 1), dtype=np.int32), np.full(max(total_items, 1), -1, dtype=np.int32),
                   np.full(max(total_items, 1), -1, dtype=np.int32), np.zeros(max(N, 1), dtype=np.int64),
                   np.zeros(max(N, 1), dtype=np.int64))


def pack_batch_host(w_all, w_off, B_all, B_off, out: HostResult, heuristic: int = H1,
                    criterion: int = BF, sublist_size: int = 0, preopen: int = 0, seed: int = 0,
                    max_m: int = 0, flags: int = 0, max_open: int = 0) -> int:
    """vsbpp_pack_batch_host: a CSR batch in host memory (numpy arrays or
    pinned torch CPU tensors) packed in one synchronous call; the library
    copies in and out.  Returns the host-side status."""
    lib = load()
    N = int((w_off.shape[0] if hasattr(w_off, "shape") else len(w_off))) - 1
    p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
    return int(lib.vsbpp_pack_batch_host(N, _ptr(w_all), _ptr(w_off), _ptr(B_all), _ptr(B_off), int(max_m),
                                         ctypes.byref(p), _ptr(out.bin_of_item), _ptr(out.bin_type),
                                         _ptr(out.num_bins), _ptr(out.total), _ptr(out.status)))


def get_config() -> dict:
    c = Config()
    rc = load().vsbpp_get_config(ctypes.byref(c))
    if rc != 0:
        raise VsbppError(rc, "vsbpp_get_config")
    return c.as_dict()


def set_config(**kw) -> None:
    cur = get_config()
    cur.update(kw)
    c = Config(**cur)
    rc = load().vsbpp_set_config(ctypes.byref(c))
    if rc != 0:
        raise VsbppError(rc, "vsbpp_set_config")


def counters_enable(on: bool = True) -> None:
    rc = load().vsbpp_counters_enable(1 if on else 0)
    if rc != 0:
        raise VsbppError(rc, "vsbpp_counters_enable")


def kernel_timing_enable(on: bool = True) -> None:
    rc = load().vsbpp_kernel_timing_enable(1 if on else 0)
    if rc != 0:
        raise VsbppError(rc, "vsbpp_kernel_timing_enable")


def kernel_timing_read(max_n: int = 256) -> list:
    """Durations (ms) of the main packing kernel of each timed call, oldest first."""
    buf = (ctypes.c_float * max_n)()
    n = ctypes.c_int32(0)
    rc = load().vsbpp_kernel_timing_read(buf, max_n, ctypes.byref(n))
    if rc != 0:
        raise VsbppError(rc, "vsbpp_kernel_timing_read")
    return [float(buf[i]) for i in range(n.value)]


def counters_read(reset: bool = True) -> dict:
    c = Counters()
    rc = load().vsbpp_counters_read(ctypes.byref(c), 1 if reset else 0)
    if rc != 0:
        raise VsbppError(rc, "vsbpp_counters_read")
    return {"items": int(c.items), "fit_tests": int(c.fit_tests)}


class Plan:
    """A batch shape recorded into a CUDA graph (vsbpp_plan_*)."""

    def __init__(self, N: int, total_m: int, max_m: int, heuristic: int = H1, criterion: int = BF,
                 sublist_size: int = 0, preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0):
        self._lib = load()
        self._p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
        h = ctypes.c_void_p()
        rc = self._lib.vsbpp_plan_create(N, total_m, max_m, ctypes.byref(self._p), ctypes.byref(h))
        if rc != 0:
            raise VsbppError(rc, "vsbpp_plan_create")
        self._h = h

    def run(self, db: "DeviceBatch", out: "DeviceResult", stream=None) -> None:
        rc = self._lib.vsbpp_plan_run(self._h, _ptr(db.w_all), _ptr(db.w_off), _ptr(db.B_all),
                                      _ptr(db.B_off), _ptr(out.bin_of_item), _ptr(out.bin_type),
                                      _ptr(out.num_bins), _ptr(out.total), _ptr(out.status),
                                      _stream_handle(stream))
        if rc != 0:
            raise VsbppError(rc, "vsbpp_plan_run")

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vsbpp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(db: "DeviceBatch", out: "DeviceResult", heuristic: int = H1, criterion: int = BF,
             sublist_size: int = 0, preopen: int = 0, seed: int = 0, stream=None, flags: int = 0,
             max_open: int = 0):
    """Time candidate launch configurations on this batch and install the
    fastest; returns (config dict, best milliseconds)."""
    lib = load()
    p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
    best = Config()
    ms = ctypes.c_double(0)
    rc = lib.vsbpp_autotune(db.N, _ptr(db.w_all), _ptr(db.w_off), _ptr(db.B_all), _ptr(db.B_off),
                            db.max_m, ctypes.byref(p), _ptr(out.bin_of_item), _ptr(out.bin_type),
                            _ptr(out.num_bins), _ptr(out.total), _ptr(out.status),
                            _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms))
    if rc != 0:
        raise VsbppError(rc, "vsbpp_autotune")
    return best.as_dict(), float(ms.value)


def tune_save(path: str) -> None:
    rc = load().vsbpp_tune_save(path.encode())
    if rc != 0:
        raise VsbppError(rc, "vsbpp_tune_save")


def tune_load(path: str) -> None:
    rc = load().vsbpp_tune_load(path.encode())
    if rc != 0:
        raise VsbppError(rc, "vsbpp_tune_load")


class Server:
    """Continuous-batching packing server (vsbpp_server_*)."""

    def __init__(self, device_mem_budget: int, max_slots: int = 64, lanes: int = 32,
                 max_queued: int = 1 << 20):
        self._lib = load()
        h = ctypes.c_void_p()
        self._m = {}
        rc = self._lib.vsbpp_server_create(device_mem_budget, max_slots, lanes, max_queued, ctypes.byref(h))
        if rc != 0:
            raise VsbppError(rc, "vsbpp_server_create")
        self._h = h

    def submit(self, w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
               preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> int:
        """Returns a ticket (>0), or raises VsbppError (e.g. EBUSY)."""
        w = np.ascontiguousarray(w, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.int32)
        p = make_params(heuristic, criterion, sublist_size, preopen, seed, flags, max_open)
        t = ctypes.c_uint64(0)
        wb = w if w.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        rc = self._lib.vsbpp_server_submit(self._h, _ptr(wb), int(w.shape[0]), _ptr(B), int(B.shape[0]),
                                           ctypes.byref(p), ctypes.byref(t))
        if rc != 0:
            raise VsbppError(rc, "vsbpp_server_submit")
        self._m[int(t.value)] = int(w.shape[0])
        return int(t.value)

    def poll(self, ticket: int, timeout_us: int = -1):
        """Returns (status, Packing or None); status ETIMEDOUT keeps the ticket."""
        m = self._m.get(ticket, 0)
        boi = np.full(max(m, 1), -1, dtype=np.int32)
        bt = np.full(max(m, 1), -1, dtype=np.int32)
        nb = ctypes.c_int64(0)
        tot = ctypes.c_int64(0)
        rc = self._lib.vsbpp_server_poll(self._h, ticket, _ptr(boi), _ptr(bt), ctypes.byref(nb),
                                         ctypes.byref(tot), int(timeout_us))
        if rc == ETIMEDOUT:
            return rc, None
        self._m.pop(ticket, None)
        k = int(nb.value)
        return int(rc), Packing(int(rc), boi[:m].copy(), bt[:k].copy(), k, int(tot.value))

    def stats(self) -> dict:
        st = ServerStats()
        rc = self._lib.vsbpp_server_stats(self._h, ctypes.byref(st))
        if rc != 0:
            raise VsbppError(rc, "vsbpp_server_stats")
        return {k: (float(getattr(st, k)) if "us" in k or k == "busy_s" else int(getattr(st, k)))
                for k, _ in st._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.vsbpp_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
