"""Seeded synthetic VSBPP instances (inputs only; no packing arithmetic here).

Both the CUDA path and the CPU oracle are fed from this module, which holds
none of the method's arithmetic: it only draws item weights and bin
capacities with numpy's PCG64 generator and lays them out as a CSR batch.

Shapes follow the paper's workloads where it states them (Section 7: item
weights drawn uniformly from {1..20}, bin types {100, 200, 300}, m up to
10^5) and the five benchmark configurations of this library:

  config1      m=100, B={100,70,40}, w ~ U[1,100], seed 0
  config2u     m=10^4, B={150,120,100,80,50}, w ~ U[1,150], seed 1
  config2m     same B, w ~ 0.7*U[1,37] + 0.3*U[75,150] (mixture), seed 2
  config3      4096 instances, m log-uniform in [100, 10^4], n in {3,5,7},
               B distinct ints in [20,1000] sorted descending, w ~ U[1,B_1]
  config4      64 instances, m=10^6, B={1000,800,640,500,400,300,200},
               w ~ 0.8*U[1,100] + 0.2*U[400,1000]
  config5      Poisson request stream, m log-uniform in [100, 10^5],
               n in {3..7}, B and w drawn as in config 2 (see ``config5``)
  configP      paper-like: m=10^5, B={300,200,100}, w ~ U{1..20}

The Correia et al. benchmark files the paper uses for its Groups 1, 3 and 4
are not available; these synthetic instances stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Batch:
    """N instances in CSR form (the layout the batched entry point takes)."""
    w_all: np.ndarray   # int32[sum m]
    w_off: np.ndarray   # int64[N+1]
    B_all: np.ndarray   # int32[sum n]
    B_off: np.ndarray   # int32[N+1]

    @property
    def N(self) -> int:
        return int(self.w_off.shape[0]) - 1

    @property
    def total_items(self) -> int:
        return int(self.w_off[-1])

    def m(self, i: int) -> int:
        return int(self.w_off[i + 1] - self.w_off[i])

    def instance(self, i: int):
        a, b = int(self.w_off[i]), int(self.w_off[i + 1])
        c, d = int(self.B_off[i]), int(self.B_off[i + 1])
        return self.w_all[a:b], self.B_all[c:d]

    def subset(self, idx) -> "Batch":
        return from_instances([self.instance(int(i)) for i in idx])

    def prefix_items(self, k: int) -> "Batch":
        """Each instance cut to its first k items (a valid batch again)."""
        return from_instances([(w[:k], B) for (w, B) in
                               (self.instance(i) for i in range(self.N))])


def from_instances(instances) -> Batch:
    ws = [np.ascontiguousarray(w, dtype=np.int32) for (w, _) in instances]
    Bs = [np.ascontiguousarray(B, dtype=np.int32) for (_, B) in instances]
    w_off = np.zeros(len(ws) + 1, dtype=np.int64)
    B_off = np.zeros(len(Bs) + 1, dtype=np.int32)
    if ws:
        w_off[1:] = np.cumsum([w.shape[0] for w in ws])
        B_off[1:] = np.cumsum([B.shape[0] for B in Bs])
    w_all = np.concatenate(ws) if ws else np.zeros(0, dtype=np.int32)
    B_all = np.concatenate(Bs) if Bs else np.zeros(0, dtype=np.int32)
    return Batch(w_all.astype(np.int32), w_off, B_all.astype(np.int32), B_off)


def log_uniform_int(rng: np.random.Generator, lo: int, hi: int, size) -> np.ndarray:
    """floor(exp(U[ln lo, ln(hi+1)))), clipped to hi."""
    x = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size)))
    return np.minimum(x, hi).astype(np.int64)


def uniform_weights(rng, lo: int, hi: int, m: int) -> np.ndarray:
    return rng.integers(lo, hi + 1, size=m, dtype=np.int64).astype(np.int32)


def mixture_weights(rng, p_first: float, first: tuple, second: tuple, m: int) -> np.ndarray:
    """Per item, a Bernoulli(p_first) draw picks U[first] else U[second]."""
    pick = rng.random(m) < p_first
    a = rng.integers(first[0], first[1] + 1, size=m, dtype=np.int64)
    b = rng.integers(second[0], second[1] + 1, size=m, dtype=np.int64)
    return np.where(pick, a, b).astype(np.int32)


def distinct_capacities(rng, n: int, lo: int, hi: int) -> np.ndarray:
    """n distinct integers in [lo, hi], sorted descending."""
    if hi - lo + 1 <= 1_000_000:
        return np.sort(rng.choice(np.arange(lo, hi + 1), size=n, replace=False))[::-1].astype(np.int32)
    picked = set()
    while len(picked) < n:           # wide range: draw until n distinct values
        picked.add(int(rng.integers(lo, hi + 1)))
    return np.array(sorted(picked, reverse=True), dtype=np.int32)


CFG1_B = np.array([100, 70, 40], dtype=np.int32)
CFG2_B = np.array([150, 120, 100, 80, 50], dtype=np.int32)
CFG4_B = np.array([1000, 800, 640, 500, 400, 300, 200], dtype=np.int32)
CFGP_B = np.array([300, 200, 100], dtype=np.int32)


def config1(seed: int = 0) -> Batch:
    rng = np.random.default_rng(seed)
    return from_instances([(uniform_weights(rng, 1, 100, 100), CFG1_B)])


def config2(variant: str = "u", seed: int | None = None, m: int = 10_000) -> Batch:
    if variant == "u":
        rng = np.random.default_rng(1 if seed is None else seed)
        w = uniform_weights(rng, 1, 150, m)
    elif variant == "m":
        rng = np.random.default_rng(2 if seed is None else seed)
        w = mixture_weights(rng, 0.7, (1, 37), (75, 150), m)
    else:
        raise ValueError(variant)
    return from_instances([(w, CFG2_B)])


def config3(seed: int = 3, N: int = 4096, m_lo: int = 100, m_hi: int = 10_000) -> Batch:
    rng = np.random.default_rng(seed)
    ms = log_uniform_int(rng, m_lo, m_hi, N)
    ns = rng.choice(np.array([3, 5, 7]), size=N)
    inst = []
    for i in range(N):
        B = distinct_capacities(rng, int(ns[i]), 20, 1000)
        inst.append((uniform_weights(rng, 1, int(B[0]), int(ms[i])), B))
    return from_instances(inst)


def config4(seed: int = 4, N: int = 64, m: int = 1_000_000) -> Batch:
    rng = np.random.default_rng(seed)
    inst = [(mixture_weights(rng, 0.8, (1, 100), (400, 1000), m), CFG4_B) for _ in range(N)]
    return from_instances(inst)


def config5_request(rng: np.random.Generator, request_id: int, m_lo: int = 100,
                    m_hi: int = 100_000):
    """One serving request: m log-uniform in [m_lo, m_hi], n uniform in {3..7}.
    n = 5 uses config 2's capacities; other n use B_1 = 150 plus n-1 distinct
    ints in [50, 149] sorted descending.  Even request ids draw w ~ U[1,150],
    odd ids the config-2 mixture."""
    m = int(log_uniform_int(rng, m_lo, m_hi, 1)[0])
    n = int(rng.integers(3, 8))
    if n == 5:
        B = CFG2_B.copy()
    else:
        rest = distinct_capacities(rng, n - 1, 50, 149)
        B = np.concatenate([np.array([150], dtype=np.int32), rest]).astype(np.int32)
    if request_id % 2 == 0:
        w = uniform_weights(rng, 1, 150, m)
    else:
        w = mixture_weights(rng, 0.7, (1, 37), (75, 150), m)
    return w, B


def config5(seed: int = 5, num_requests: int = 256, rate_per_s: float = 1000.0,
            m_lo: int = 100, m_hi: int = 100_000):
    """A Poisson request stream: (arrival_time_s, w, B) per request."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=num_requests)
    t = np.cumsum(gaps)
    out = []
    for r in range(num_requests):
        w, B = config5_request(rng, r, m_lo, m_hi)
        out.append((float(t[r]), w, B))
    return out


def configP(seed: int = 6, m: int = 100_000) -> Batch:
    rng = np.random.default_rng(seed)
    return from_instances([(uniform_weights(rng, 1, 20, m), CFGP_B)])


def random_instance(rng: np.random.Generator, m: int, n: int, cap_hi: int,
                    w_hi: int | None = None, cap_lo: int = 1):
    """Small fuzz instance: n distinct capacities in [cap_lo, cap_hi], items
    uniform in [1, min(w_hi, B_1)]."""
    n = min(n, cap_hi - cap_lo + 1)
    B = distinct_capacities(rng, n, cap_lo, cap_hi)
    top = int(B[0]) if w_hi is None else min(int(w_hi), int(B[0]))
    return uniform_weights(rng, 1, top, m), B
