"""CPU oracle for the hybrid-P-system VSBPP heuristics (arXiv:1602.08735).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1602_08735_gb300``) never imports, links or calls it, and it never
imports the product library: the two share no code.

The arithmetic lives in plain C (``vsbpp_oracle.c``): a flat, single-threaded
simulation of Rules 2-6 of Section 6.3 and of the permutation sweep of
Section 6.4, plus an exact subset-DP optimum for tiny instances (Section 1's
definition of the problem).  This module only compiles that file with gcc and
marshals numpy arrays through ctypes.

Status codes: 0 ok, -1 invalid input, -2 an item heavier than B_1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("vsbpp_oracle.c", "oracle_threads.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FF, BF, WF, RANDOM = 0, 1, 2, 3
H1, H2 = 1, 2
OK, EINVAL, ETOOBIG = 0, -1, -2
REMARK3 = 1        # flag: Rule 5 with Remark 3's per-type condition (reading in vsbpp_oracle.c, G7)
PRESORT = 2        # flag: items packed in non-increasing weight order, ties in list order (G16)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` with gcc (portable C11,
    no architecture flags, so the same source builds on x86-64 and aarch64)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_mtime = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_mtime for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
           *srcs, "-lpthread", "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_splitmix64.restype = ctypes.c_uint64
    lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_pack.restype = ctypes.c_int
    lib.oracle_pack.argtypes = [i32p, ctypes.c_int64, i32p, ctypes.c_int32,
                                ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                ctypes.c_int32, ctypes.c_uint64,
                                i32p, i32p, i64p, i64p]
    lib.oracle_pack_flags.restype = ctypes.c_int
    lib.oracle_pack_flags.argtypes = [i32p, ctypes.c_int64, i32p, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32,
                                      i32p, i32p, i64p, i64p]
    lib.oracle_pack_ext.restype = ctypes.c_int
    lib.oracle_pack_ext.argtypes = [i32p, ctypes.c_int64, i32p, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                    ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                    i32p, i32p, i64p, i64p]
    lib.oracle_fit_tests_ext.restype = ctypes.c_uint64
    lib.oracle_fit_tests_ext.argtypes = [i32p, ctypes.c_int64, i32p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                         ctypes.c_int32, ctypes.c_int64]
    lib.oracle_opt_bruteforce.restype = ctypes.c_int64
    lib.oracle_opt_bruteforce.argtypes = [i32p, ctypes.c_int32, i32p, ctypes.c_int32]
    lib.oracle_fit_tests.restype = ctypes.c_uint64
    lib.oracle_fit_tests.argtypes = [i32p, ctypes.c_int64, i32p, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64]
    lib.oracle_pack_many.restype = ctypes.c_int
    lib.oracle_pack_many.argtypes = [ctypes.c_int64, i32p, i64p, i32p, i32p,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                     ctypes.c_int32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                     i32p, i32p, i64p, i64p, i32p, ctypes.c_int32]
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


@dataclass
class PackResult:
    status: int
    bin_of_item: np.ndarray   # int32[m], dense bin id per item
    bin_type: np.ndarray      # int32[num_bins], 0-based type (0 = largest)
    num_bins: int
    total: int                # total capacity of used bins


@dataclass
class BatchResult:
    status: np.ndarray        # int32[N]
    bin_of_item: np.ndarray   # int32[sum m], CSR-aligned with w_off
    bin_type: np.ndarray      # int32[sum m], instance i's types at w_off[i]..+num_bins[i]
    num_bins: np.ndarray      # int64[N]
    total: np.ndarray         # int64[N]


class OracleLib:
    """ctypes front-end over one compiled copy of the oracle.  The default
    copy is ``oracle/liboracle.so``; tests that plant a mistake compile a
    modified copy of the C source elsewhere and open it through this class."""

    def __init__(self, path: str):
        self.path = path
        self._lib = _bind(ctypes.CDLL(path))

    def splitmix64(self, seed: int, key: int) -> int:
        """key-th output of SplitMix64 seeded with ``seed`` (Steele et al. 2014)."""
        return int(self._lib.oracle_splitmix64(seed & (2**64 - 1), key & (2**64 - 1)))

    def pack(self, w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
             preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> PackResult:
        """Pack one instance with the hybrid P system (Sections 6.3 / 6.4).
        flags: REMARK3 (Rule 5 divides only when every bin of the type then
        holds at least half its capacity, Remark 3 of Section 6.3) and/or
        PRESORT (non-increasing weight order first, reading G16).  max_open:
        0, or K >= 1 for the bounded-space variant (reading G15)."""
        w = np.ascontiguousarray(w, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.int32)
        m = int(w.shape[0])
        bin_of_item = np.full(max(m, 1), -1, dtype=np.int32)
        bin_type = np.full(max(m, 1), -1, dtype=np.int32)
        nb = np.zeros(1, dtype=np.int64)
        tot = np.zeros(1, dtype=np.int64)
        wbuf = w if m > 0 else np.zeros(1, dtype=np.int32)
        Bbuf = B if B.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        rc = self._lib.oracle_pack_ext(_ptr(wbuf, ctypes.c_int32), m, _ptr(Bbuf, ctypes.c_int32),
                                       int(B.shape[0]), heuristic, criterion, sublist_size, preopen,
                                       seed & (2**64 - 1), flags, max_open,
                                       _ptr(bin_of_item, ctypes.c_int32), _ptr(bin_type, ctypes.c_int32),
                                       _ptr(nb, ctypes.c_int64), _ptr(tot, ctypes.c_int64))
        k = int(nb[0])
        return PackResult(int(rc), bin_of_item[:m].copy(), bin_type[:k].copy(), k, int(tot[0]))

    def fit_tests(self, w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
                  preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> int:
        """Rule 4 fit tests the oracle performs on this instance (one per
        bin membrane that is open when an item arrives)."""
        w = np.ascontiguousarray(w, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.int32)
        wbuf = w if w.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        return int(self._lib.oracle_fit_tests_ext(_ptr(wbuf, ctypes.c_int32), int(w.shape[0]),
                                                  _ptr(B, ctypes.c_int32), int(B.shape[0]), heuristic,
                                                  criterion, sublist_size, preopen, seed & (2**64 - 1),
                                                  flags, max_open))

    def opt_bruteforce(self, w, B) -> int:
        """Exact VSBPP optimum by subset DP (m <= 20); -1 if infeasible/invalid."""
        w = np.ascontiguousarray(w, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.int32)
        wbuf = w if w.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        return int(self._lib.oracle_opt_bruteforce(_ptr(wbuf, ctypes.c_int32), int(w.shape[0]),
                                                   _ptr(B, ctypes.c_int32), int(B.shape[0])))

    def pack_many(self, w_all, w_off, B_all, B_off, heuristic: int = H1, criterion: int = BF,
                  sublist_size: int = 0, preopen: int = 0, seed: int = 0, flags: int = 0,
                  nthreads: int | None = None, max_open: int = 0) -> BatchResult:
        """Pack N independent instances given in CSR form; one oracle call per
        instance, spread over ``nthreads`` host threads (default: all cores).
        flags as in ``pack``."""
        w_all = np.ascontiguousarray(w_all, dtype=np.int32)
        w_off = np.ascontiguousarray(w_off, dtype=np.int64)
        B_all = np.ascontiguousarray(B_all, dtype=np.int32)
        B_off = np.ascontiguousarray(B_off, dtype=np.int32)
        N = int(w_off.shape[0]) - 1
        tot_m = int(w_off[-1]) if N > 0 else 0
        if nthreads is None:
            nthreads = host_cores()
        boi = np.full(max(tot_m, 1), -1, dtype=np.int32)
        bty = np.full(max(tot_m, 1), -1, dtype=np.int32)
        nb = np.zeros(max(N, 1), dtype=np.int64)
        tot = np.zeros(max(N, 1), dtype=np.int64)
        st = np.zeros(max(N, 1), dtype=np.int32)
        wbuf = w_all if w_all.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        Bbuf = B_all if B_all.shape[0] > 0 else np.zeros(1, dtype=np.int32)
        rc = self._lib.oracle_pack_many(N, _ptr(wbuf, ctypes.c_int32), _ptr(w_off, ctypes.c_int64),
                                        _ptr(Bbuf, ctypes.c_int32), _ptr(B_off, ctypes.c_int32),
                                        heuristic, criterion, sublist_size, preopen,
                                        seed & (2**64 - 1), flags, max_open,
                                        _ptr(boi, ctypes.c_int32), _ptr(bty, ctypes.c_int32),
                                        _ptr(nb, ctypes.c_int64), _ptr(tot, ctypes.c_int64),
                                        _ptr(st, ctypes.c_int32), int(nthreads))
        if rc != 0:
            raise RuntimeError(f"oracle_pack_many failed: {rc}")
        return BatchResult(st[:N].copy(), boi[:tot_m].copy(), bty[:tot_m].copy(),
                           nb[:N].copy(), tot[:N].copy())


def host_cores() -> int:
    """Host cores this process may run on (its CPU affinity set)."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a (possibly modified) copy of the oracle C source together with
    the unmodified thread driver into ``out_path``."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                    src, os.path.join(_HERE, "oracle_threads.c"), "-lpthread", "-o", out_path],
                   check=True)
    return out_path


def source_text() -> str:
    with open(os.path.join(_HERE, "vsbpp_oracle.c")) as f:
        return f.read()


def default() -> OracleLib:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = OracleLib(_LIB_PATH)
        return _lib


def splitmix64(seed: int, key: int) -> int:
    return default().splitmix64(seed, key)


def pack(w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
         preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> PackResult:
    return default().pack(w, B, heuristic, criterion, sublist_size, preopen, seed, flags, max_open)


def fit_tests(w, B, heuristic: int = H1, criterion: int = BF, sublist_size: int = 0,
              preopen: int = 0, seed: int = 0, flags: int = 0, max_open: int = 0) -> int:
    return default().fit_tests(w, B, heuristic, criterion, sublist_size, preopen, seed, flags, max_open)


def opt_bruteforce(w, B) -> int:
    return default().opt_bruteforce(w, B)


def pack_many(w_all, w_off, B_all, B_off, heuristic: int = H1, criterion: int = BF,
              sublist_size: int = 0, preopen: int = 0, seed: int = 0, flags: int = 0,
              nthreads: int | None = None, max_open: int = 0) -> BatchResult:
    return default().pack_many(w_all, w_off, B_all, B_off, heuristic, criterion,
                               sublist_size, preopen, seed, flags, nthreads, max_open)
