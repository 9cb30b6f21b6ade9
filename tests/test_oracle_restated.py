"""The oracle against a second, independent restatement of the method in
plain Python (CPU): Rules 2-6 on a membrane system (fit test residual >= w,
FF / BF / WF with the lowest creation index on ties, a bin of the smallest
type holding the item when nothing fits, the Rule 5 division when a bin's
load first reaches half its capacity, reading G7), the first heuristic's
sublists (reading G1), the second heuristic's lexicographic permutations with
the cheapest winning at the lowest rank (readings G9-G11), the literal Rule 2
start (reading G3), the RANDOM criterion's keys (reading G12), Remark 3
(reading G7), the bounded-space variant (reading G15) and the pre-sort
(reading G16), on small random instances of every shape the library takes
(instances shorter than the sublist size included).  This is a restatement of the same readings, not
a pin: the pins in oracle_pins.py tie the oracle to values fixed outside it.
"""
import itertools

import numpy as np

import oracle
from oracle_pins import splitmix64_py

F12 = 479001600


def run_system(items, crits, B, preopen, remark3=False, K=0):
    """Rules 2-6 on one membrane system: the bin each item goes to and the
    bins [residual, capacity, type] in creation order.  remark3: a division
    also needs every bin of the type at half its capacity or more (reading
    G7).  K > 0: only the K or fewer open bins take part, a bin closes when
    full, and before a bin is created while K are open the oldest open bin
    closes (reading G15)."""
    bins = []
    active = []                                       # open bins in creation order

    def new_bin(t):
        if K and len(active) >= K:
            active.pop(0)
        bins.append([B[t], B[t], t])
        active.append(len(bins) - 1)
        return len(bins) - 1

    if preopen:
        for t in range(len(B)):
            new_bin(t)
    raw = []
    for x, c in zip(items, crits):
        fit = [b for b in (active if K else range(len(bins))) if bins[b][0] >= x]
        if not fit:
            b = new_bin(max(i for i in range(len(B)) if B[i] >= x))   # smallest type holding x
        elif c == 0:
            b = fit[0]
        elif c == 1:
            b = min(fit, key=lambda y: (bins[y][0] - x, y))
        else:
            b = min(fit, key=lambda y: (-bins[y][0], y))
        old, cap, t = bins[b]
        new = old - x
        bins[b][0] = new
        if K and new == 0:
            active.remove(b)                          # a full bin closes first
        if cap < 2 * old and 2 * new <= cap:          # load first reaches half: Rule 5
            if not remark3 or all(2 * (y[1] - y[0]) >= y[1] for y in bins if y[2] == t):
                new_bin(t)
        raw.append(b)
    return raw, bins


def dense_of(bins):
    """Dense ids of the used bins (load > 0) in creation order (reading G8)."""
    d = {}
    for b in range(len(bins)):
        if bins[b][0] < bins[b][1]:
            d[b] = len(d)
    return d


def brute(w, B, h, crit, s, preopen, seed, remark3=False, K=0, presort=False):
    """Every sublist packed as the readings state: (bin of each item, bin
    types, bins, total).  presort: the list in non-increasing weight order,
    equal weights in list order, each bin id reported at the item's original
    position (reading G16)."""
    m = len(w)
    if m == 0:
        return [], [], 0, 0
    if presort:
        order = sorted(range(m), key=lambda j: (-w[j], j))
        boi_s, types, nb, tot = brute([w[j] for j in order], B, h, crit, s, preopen, seed, remark3, K)
        boi = [0] * m
        for jj, j in enumerate(order):
            boi[j] = boi_s[jj]
        return boi, types, nb, tot
    s_ = (m if s == 0 else s) if h == 1 else (5 if s == 0 else s)
    boi, types, total, off = [0] * m, [], 0, 0

    def draw(key, c):
        return splitmix64_py(seed, key) % 3 if c == 3 else c

    for g, a in enumerate(range(0, m, s_)):
        sub = w[a:a + s_]
        k = len(sub)
        if h == 1:
            raw, bins = run_system(sub, [draw(a + q, crit) for q in range(k)], B, preopen, remark3, K)
            d = dense_of(bins)
            for q in range(k):
                boi[a + q] = off + d[raw[q]]
            total += sum(bins[b][1] for b in d)
            types += [bins[b][2] for b in sorted(d, key=d.get)]
            off += len(d)
            continue
        best = None
        for rank, perm in enumerate(itertools.permutations(range(k))):
            keys = [((g * 720 + rank) * 8 + q) if s_ <= 6 else ((g * F12 + rank) * 16 + q) for q in range(k)]
            raw, bins = run_system([sub[x] for x in perm], [draw(kq, crit) for kq in keys], B, preopen, remark3)
            d = dense_of(bins)
            tot = sum(bins[b][1] for b in d)
            if best is None or tot < best[0]:
                ib = [0] * k
                for q, x in enumerate(perm):
                    ib[x] = d[raw[q]]
                best = (tot, ib, [bins[b][2] for b in sorted(d, key=d.get)])
        for q in range(k):
            boi[a + q] = off + best[1][q]
        total += best[0]
        types += best[2]
        off += len(best[2])
    return boi, types, off, total


def test_oracle_equals_restatement():
    rng = np.random.default_rng(2024)
    bad = []
    for t in range(600):
        n = int(rng.integers(1, 5))
        cap_hi = int(rng.choice([12, 40, 120]))
        B = sorted(rng.choice(np.arange(1, cap_hi + 1), size=min(n, cap_hi), replace=False).tolist(), reverse=True)
        h = int(rng.integers(1, 3))
        crit = int(rng.integers(0, 4))
        preopen = int(rng.integers(0, 2))
        s = int(rng.choice([0, 1, 2, 3, 5, 6, 7, 8])) if h == 2 else int(rng.choice([0, 0, 1, 3, 4]))
        if h == 2 and s >= 7:
            preopen = 0            # the exhaustive search starts without pre-opened bins
        remark3 = bool(rng.integers(0, 2))
        presort = bool(rng.integers(0, 2))
        K = int(rng.choice([0, 0, 1, 2, 3, 5])) if (h == 1 and not remark3) else 0
        m = int(rng.integers(0, 9 if (h == 2 and s >= 7) else 13))
        w = rng.integers(1, B[0] + 1, size=m).tolist()
        seed = int(rng.integers(0, 2**40))
        flags = (oracle.REMARK3 if remark3 else 0) | (oracle.PRESORT if presort else 0)
        r = oracle.pack(np.array(w, dtype=np.int32), np.array(B, dtype=np.int32), h, crit, s, preopen, seed,
                        flags, K)
        boi, types, nb, tot = brute(w, B, h, crit, s, preopen, seed, remark3, K, presort)
        if not (r.status == 0 and r.bin_of_item.tolist() == boi and r.bin_type.tolist() == types
                and r.num_bins == nb and r.total == tot):
            bad.append(dict(w=w, B=B, h=h, crit=crit, s=s, preopen=preopen, seed=seed, flags=flags, K=K))
    assert not bad, bad[:3]
