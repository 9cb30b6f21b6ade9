"""Pins that tie the CPU oracle to something other than itself.

Each ``pin_*`` function takes an ``oracle.OracleLib`` and raises
AssertionError when the oracle disagrees with what the paper or the
mathematics fixes:

  * hand-worked packings (tests/golden/hand_examples.json, traced by hand from
    Section 6.3 Rules 2-6, Section 6.4 and the FF/BF/WF definitions of
    Section 1);
  * the published SplitMix64 test vectors (RANDOM criterion, Rule 3), both
    as raw outputs and through the criterion each one gives an item;
  * with one bin type (n = 1, classical bin packing, Section 1), FF and BF
    reduce to the textbook First-Fit and Best-Fit written out below in a
    different form (no empty bins, no division rule);
  * the exact optimum from an independent set-partition enumeration, and
    heuristic >= optimum;
  * closed forms: a single item costs min{B_i >= w} (also when w equals a
    capacity); m items of weight B_1 cost m*B_1;
  * the second heuristic equals the cheapest permutation, enumerated here with
    itertools (Section 6.4); with the RANDOM criterion, each permutation's
    criteria follow from the SplitMix64 stream property (output K of the
    stream seeded s is output 0 of the stream seeded s + K*gamma), which pins
    the second heuristic's key layout (reading G12) to the first heuristic's
    RANDOM packing;
  * invariants of any packing (each item once, no bin over capacity, total =
    sum of used capacities >= sum of weights);
  * the bounded-space variant (reading G15): a bound no packing can reach
    gives the unbounded packing, one open bin makes FF, BF and WF identical,
    and no step ever meets more open bins than the bound;
  * the offline pre-sort (reading G16): with one bin type FF and BF in
    decreasing order are the textbook FFD and BFD, and a list already in
    non-increasing order is packed as it stands.

The same functions run against copies of the oracle with planted mistakes
(tests/test_oracle_mutants.py) to show that each plausible slip is caught.
"""
from __future__ import annotations

import itertools
import json
import os

import math

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------- textbook
def textbook_first_fit(w, C):
    """Classical First-Fit: put each item in the first opened bin with room,
    else open a new bin.  Returns (bin index per item, number of bins)."""
    loads = []
    out = []
    for x in w:
        for i, ld in enumerate(loads):
            if ld + x <= C:
                loads[i] += x
                out.append(i)
                break
        else:
            loads.append(x)
            out.append(len(loads) - 1)
    return out, len(loads)


def textbook_best_fit(w, C):
    """Classical Best-Fit: the opened bin with the least room that still holds
    the item (lowest index on ties), else a new bin."""
    loads = []
    out = []
    for x in w:
        best, room = -1, None
        for i, ld in enumerate(loads):
            r = C - ld
            if r >= x and (room is None or r < room):
                best, room = i, r
        if best < 0:
            loads.append(x)
            out.append(len(loads) - 1)
        else:
            loads[best] += x
            out.append(best)
    return out, len(loads)


def set_partition_optimum(w, B):
    """Exact VSBPP optimum by enumerating every set partition of the items
    (restricted growth strings); cost of a block = smallest B_i >= its sum."""
    m = len(w)
    if m == 0:
        return 0
    caps = sorted(B)
    best = None
    labels = [0] * m

    def cost(lbl):
        sums = {}
        for x, l in zip(w, lbl):
            sums[l] = sums.get(l, 0) + x
        tot = 0
        for s in sums.values():
            c = next((c for c in caps if c >= s), None)
            if c is None:
                return None
            tot += c
        return tot

    def rec(i, k):
        nonlocal best
        if i == m:
            c = cost(labels)
            if c is not None and (best is None or c < best):
                best = c
            return
        for l in range(k + 1):
            labels[i] = l
            rec(i + 1, max(k, l + 1))

    rec(0, 0)
    return best


def check_packing(w, B, res, m_expected=None):
    """Invariants every packing must satisfy."""
    w = np.asarray(w, dtype=np.int64)
    B = np.asarray(B, dtype=np.int64)
    assert res.status == 0
    m = w.shape[0]
    boi = np.asarray(res.bin_of_item, dtype=np.int64)
    bty = np.asarray(res.bin_type, dtype=np.int64)
    assert boi.shape[0] == m
    assert bty.shape[0] == res.num_bins
    if m == 0:
        assert res.num_bins == 0 and res.total == 0
        return
    assert boi.min() >= 0 and boi.max() < res.num_bins
    loads = np.bincount(boi, weights=w, minlength=res.num_bins)
    assert np.all(loads > 0), "every reported bin holds an item"
    assert np.all(bty >= 0) and np.all(bty < B.shape[0])
    assert np.all(loads <= B[bty]), "no bin over capacity"
    assert res.total == int(B[bty].sum())
    assert res.total >= int(w.sum())
    assert res.num_bins <= m
    # dense ids in creation order: first appearance of each id is increasing
    # within one membrane system; ids are a permutation-free labelling.
    assert np.unique(boi).shape[0] == res.num_bins


# ---------------------------------------------------------------- SplitMix64
# Steele, Lea & Flood (OOPSLA 2014): the state advances by the odd constant
# gamma (the golden-ratio increment of the published generator), and each
# output is the state passed through the variant-13 mixer.  Written here
# independently of the oracle's C copy and checked against the published
# vectors by pin_h2_random_key.
SM_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64_py(seed: int, key: int) -> int:
    """Output number `key` (0-based) of the SplitMix64 stream seeded `seed`."""
    z = (seed + (key + 1) * SM_GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


FACT12 = math.factorial(12)


def h2_random_key_base(g: int, rank: int, s: int) -> int:
    """Reading G12: the RANDOM key of step q of permutation `rank` of sublist
    g is base + q, base = (g*720 + rank)*8 for s <= 6 and (g*12! + rank)*16
    for the exhaustive search (s = 7..12)."""
    return (g * 720 + rank) * 8 if s <= 6 else (g * FACT12 + rank) * 16


# --------------------------------------------------------------------- pins
def pin_hand_examples(lib):
    d = load_golden("hand_examples.json")
    for ex in d["examples"]:
        r = lib.pack(ex["w"], ex["B"], ex["heuristic"], ex["criterion"], ex["sublist_size"],
                     ex["preopen"], ex["seed"], ex.get("flags", 0), ex.get("max_open", 0))
        assert r.status == 0, ex["name"]
        assert r.bin_of_item.tolist() == ex["bin_of_item"], ex["name"]
        assert r.bin_type.tolist() == ex["bin_type"], ex["name"]
        assert r.total == ex["total"], ex["name"]
        if "opt" in ex:
            assert lib.opt_bruteforce(ex["w"], ex["B"]) == ex["opt"], ex["name"]


def pin_splitmix64(lib):
    d = load_golden("splitmix64_vectors.json")
    for k, v in enumerate(d["outputs"]):
        assert lib.splitmix64(d["seed"], k) == int(v)


def pin_random_criterion_vectors(lib):
    """RANDOM (Rule 3 with the criterion drawn per item, reading G12: item j
    of the instance takes criterion SplitMix64(seed, j) mod 3, 0 = FF, 1 = BF,
    2 = WF) against the published SplitMix64 outputs for seed 1234567, read
    off the packing itself.  With one type of capacity 100, the items
    [100] * (p - 2) + [60, 80] are placed the same way under every criterion
    (each fits only the empty bin the previous one divided off) and leave
    bins with room 40 (dense id p - 2), 20 (p - 1) and an empty one (p);
    item p = 15 then goes to p - 2 under FF, p - 1 under BF and p under WF.
    After [60] alone (room 40, and an empty bin) an item of 30 separates WF
    from FF / BF."""
    d = load_golden("splitmix64_vectors.json")
    seed = int(d["seed"])
    crit = [int(x) % 3 for x in d["outputs"]]
    for p in (2, 3, 4):
        r = lib.pack([100] * (p - 2) + [60, 80, 15], [100], 1, 3, 0, 0, seed)
        assert r.status == 0
        assert int(r.bin_of_item[p]) == p - 2 + crit[p], (p, crit[p], r.bin_of_item.tolist())
    r = lib.pack([60, 30], [100], 1, 3, 0, 0, seed)
    assert int(r.bin_of_item[1]) == (1 if crit[1] == 2 else 0), (crit[1], r.bin_of_item.tolist())


def pin_textbook_n1(lib, trials=150, seed=11):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        C = int(rng.integers(1, 60))
        m = int(rng.integers(0, 40))
        w = rng.integers(1, C + 1, size=m).tolist()
        for crit, ref in ((0, textbook_first_fit), (1, textbook_best_fit)):
            r = lib.pack(w, [C], 1, crit)
            idx, nbins = ref(w, C)
            assert r.status == 0
            assert r.bin_of_item.tolist() == idx, (crit, C, w)
            assert r.num_bins == nbins
            assert r.total == nbins * C


def pin_optimum(lib, trials=60, seed=12):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        m = int(rng.integers(0, 8))
        n = int(rng.integers(1, 4))
        B = sorted(rng.choice(np.arange(3, 40), size=n, replace=False).tolist(), reverse=True)
        w = rng.integers(1, B[0] + 1, size=m).tolist()
        opt = lib.opt_bruteforce(w, B)
        assert opt == set_partition_optimum(w, B), (w, B)
        for h, s in ((1, 0), (2, 0)):
            for crit in (0, 1, 2):
                r = lib.pack(w, B, h, crit, s)
                assert r.total >= opt, (w, B, h, crit)


def pin_closed_forms(lib, seed=13):
    rng = np.random.default_rng(seed)
    for t in range(40):
        n = int(rng.integers(1, 6))
        B = sorted(rng.choice(np.arange(1, 500), size=n, replace=False).tolist(), reverse=True)
        x = int(rng.integers(1, B[0] + 1))
        want = min(b for b in B if b >= x)
        for h in (1, 2):
            for crit in (0, 1, 2, 3):
                r = lib.pack([x], B, h, crit, 0, 0, t)
                assert r.total == want and r.num_bins == 1
                assert r.bin_type.tolist() == [B.index(want)]
        # an item exactly as heavy as a capacity takes a bin of that type
        i = int(rng.integers(0, n))
        r = lib.pack([B[i]], B, 1, int(rng.integers(0, 3)))
        assert r.total == B[i] and r.bin_type.tolist() == [i]
        m = int(rng.integers(1, 30))
        r = lib.pack([B[0]] * m, B, 1, int(rng.integers(0, 3)))
        assert r.total == m * B[0] and r.num_bins == m
        assert r.bin_of_item.tolist() == list(range(m))
        assert r.bin_type.tolist() == [0] * m


def pin_h2_is_best_permutation(lib, trials=60, seed=14):
    """The second heuristic (Section 6.4) and the exhaustive search of
    Section 7 (sublists of 7..12 items) equal the best permutation by
    itertools, each packed by the first heuristic: least total, earliest in
    lexicographic order on ties."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        k = int(rng.integers(1, 6)) if t < trials - 3 else 7 + (t % 2)
        n = int(rng.integers(1, 4))
        B = sorted(rng.choice(np.arange(2, 30), size=n, replace=False).tolist(), reverse=True)
        w = rng.integers(1, B[0] + 1, size=k).tolist()
        crit = int(rng.integers(0, 3))
        pre = int(rng.integers(0, 2))
        best = None
        for perm in itertools.permutations(range(k)):       # lexicographic
            seq = [w[p] for p in perm]
            r = lib.pack(seq, B, 1, crit, 0, pre)
            if best is None or r.total < best[0]:
                item_bin = [0] * k
                for q, p in enumerate(perm):
                    item_bin[p] = int(r.bin_of_item[q])
                best = (r.total, item_bin, r.bin_type.tolist())
        r2 = lib.pack(w, B, 2, crit, k, pre)
        assert r2.total == best[0], (w, B, crit)
        assert r2.bin_of_item.tolist() == best[1], (w, B, crit)
        assert r2.bin_type.tolist() == best[2]


def pin_h2_random_key(lib, seed=17):
    """The second heuristic with the RANDOM criterion (Rule 3's draw "with
    equal probabilities", Section 6.4's permutations, reading G12).  Step q of
    permutation `rank` of sublist g takes criterion SplitMix64(seed, base + q)
    mod 3, with base as in h2_random_key_base.  SplitMix64 output K of the
    stream seeded `seed` is output 0 of the stream seeded seed + K*gamma
    (the state only ever advances by gamma), so that permutation packs
    exactly as the first heuristic with RANDOM packs the permuted items with
    seed + base*gamma: the first heuristic's RANDOM is pinned to the published
    vectors by pin_random_criterion_vectors.  Several sublists (g > 0), the
    two key layouts (s <= 6 and s = 7) and the switch between them (s = 6 vs
    7) are all exercised; the cheapest permutation wins, lowest rank on
    ties, ids offset by the earlier sublists' bins (reading G11)."""
    d = load_golden("splitmix64_vectors.json")
    for k, v in enumerate(d["outputs"]):
        assert splitmix64_py(int(d["seed"]), k) == int(v)
    # the stream property used below, on the published seed
    for K in (0, 1, 7, 5765, 2**40 + 3):
        assert splitmix64_py(int(d["seed"]), K) == splitmix64_py((int(d["seed"]) + K * SM_GAMMA) & _M64, 0)
    rng = np.random.default_rng(seed)

    def check(s, m, w=None, B=None, run_seed=None):
        if w is None:
            n = int(rng.integers(2, 4))
            B = sorted(rng.choice(np.arange(6, 40), size=n, replace=False).tolist(), reverse=True)
            w = rng.integers(1, B[0] + 1, size=m).tolist()
            run_seed = int(rng.integers(0, 2**63))
        want_boi, want_bt, total, off = [], [], 0, 0
        for g, a in enumerate(range(0, m, s)):
            sub = w[a:a + s]
            k = len(sub)
            best = None
            for rank, perm in enumerate(itertools.permutations(range(k))):
                # the layout is the run's (sublist size s), whatever k is
                seed_p = (run_seed + h2_random_key_base(g, rank, s) * SM_GAMMA) & _M64
                r = lib.pack([sub[x] for x in perm], B, 1, 3, 0, 0, seed_p)
                if best is None or r.total < best[0]:
                    item_bin = [0] * k
                    for q, x in enumerate(perm):
                        item_bin[x] = int(r.bin_of_item[q])
                    best = (r.total, item_bin, r.bin_type.tolist(), r.num_bins)
            want_boi += [off + b for b in best[1]]
            want_bt += best[2]
            total += best[0]
            off += best[3]
        r2 = lib.pack(w, B, 2, 3, s, 0, run_seed)
        assert r2.status == 0
        assert r2.bin_of_item.tolist() == want_boi, (s, w, B, run_seed)
        assert r2.bin_type.tolist() == want_bt, (s, w, B)
        assert r2.total == total

    for s, trials in ((3, 6), (5, 3), (6, 2), (7, 1)):
        for t in range(trials):
            check(s, 2 * s + int(rng.integers(1, 3)))       # two full sublists and a partial one
    # an instance shorter than the run's sublist size is one sublist that
    # still takes the run's layout (7..12: the exhaustive search's keys)
    for s, m in ((7, 5), (7, 6), (8, 4)):
        check(s, m)
    # five items over five capacities, where the two layouts' criteria lead
    # to different cheapest packings
    check(7, 5, [38, 22, 33, 26, 32], [58, 57, 36, 28, 5], 6)


def pin_invariants(lib, trials=200, seed=15):
    rng = np.random.default_rng(seed)
    for t in range(trials):
        m = int(rng.integers(0, 60))
        n = int(rng.integers(1, 8))
        cap_hi = int(rng.choice([20, 100, 1000, 40000]))
        B = sorted(rng.choice(np.arange(1, cap_hi + 1), size=min(n, cap_hi), replace=False).tolist(),
                   reverse=True)
        w = rng.integers(1, B[0] + 1, size=m).tolist()
        h = int(rng.integers(1, 3))
        s = int(rng.integers(0, 7)) if h == 2 else int(rng.choice([0, 0, 1, 3, 10]))
        crit = int(rng.integers(0, 4))
        pre = int(rng.integers(0, 2))
        r = lib.pack(w, B, h, crit, s, pre, t)
        check_packing(w, B, r)


def pin_errors(lib):
    B = [100, 50]
    assert lib.pack([1, 2], [], 1, 0).status == -1          # n = 0
    assert lib.pack([1, 2], [50, 100], 1, 0).status == -1   # not decreasing
    assert lib.pack([1, 2], [50, 50], 1, 0).status == -1    # not strictly
    assert lib.pack([1, 2], [50, 0], 1, 0).status == -1     # B_n must be > 0
    assert lib.pack([0, 2], B, 1, 0).status == -1           # w >= 1
    assert lib.pack([101], B, 1, 0).status == -2            # w <= B_1
    assert lib.pack([0, 101], B, 1, 0).status == -1         # first offender decides
    assert lib.pack([101, 0], B, 1, 0).status == -2
    assert lib.pack([1], B, 3, 0).status == -1              # heuristic id
    assert lib.pack([1], B, 1, 4).status == -1              # criterion id
    assert lib.pack([1], B, 1, 0, 0, 0, 0, 4).status == -1  # unknown flag
    assert lib.pack([1], B, 1, 0, max_open=-1).status == -1            # bound >= 0
    assert lib.pack([1], B, 2, 0, 5, max_open=3).status == -1          # bounded: first heuristic only
    assert lib.pack([1], B, 1, 0, 0, 0, 0, 1, max_open=3).status == -1  # not with Remark 3
    assert lib.pack([0, 2], B, 1, 0, 0, 0, 0, 2).status == -1           # pre-sort: list order decides
    assert lib.pack([101, 0], B, 1, 0, 0, 0, 0, 2).status == -2
    assert lib.pack([1], B, 1, 0, -1).status == -1          # sublist size
    assert lib.pack([1], B, 2, 0, 13).status == -1          # H2 sublist <= 12
    assert lib.pack([1], B, 1, 0, 0, 2).status == -1        # preopen flag
    r = lib.pack([], B, 1, 0)
    assert r.status == 0 and r.num_bins == 0 and r.total == 0


def pin_fit_tests(lib, seed=16):
    """The fit-test count (Rule 4: every bin membrane alive when an item
    arrives tests it).  Closed form: with every weight equal to B_1 the first
    item finds no bin, opens one, fills it and Rule 5 divides off an empty
    bin; item j >= 1 then meets j + 1 bins, takes the empty one and divides
    off another, so m items make 2 + 3 + ... + m = (m - 1)(m + 2) / 2 tests,
    for every criterion and with one type or several.  The second heuristic
    repeats that for each of the s! permutations of every sublist.  Hand
    example (BF, B = {8, 6, 4}, w = 3,3,3,3,4,4,1): the 3s and 4s each fill a
    fresh 4-bin that divides, so the items meet 0, 2, 3, 4, 5, 6, 7 bins: 27."""
    assert lib.fit_tests([3, 3, 3, 3, 4, 4, 1], [8, 6, 4], 1, 1) == 27
    rng = np.random.default_rng(seed)
    for t in range(20):
        n = int(rng.integers(1, 6))
        B = sorted(rng.choice(np.arange(1, 500), size=n, replace=False).tolist(), reverse=True)
        m = int(rng.integers(1, 60))
        for crit in (0, 1, 2, 3):
            assert lib.fit_tests([B[0]] * m, B, 1, crit, 0, 0, t) == (m - 1) * (m + 2) // 2
        s = int(rng.integers(1, 7))
        full, rest = divmod(m, s)
        per = lambda k: (k - 1) * (k + 2) // 2 * math.factorial(k)
        assert lib.fit_tests([B[0]] * m, B, 2, int(rng.integers(0, 3)), s) == full * per(s) + (per(rest) if rest else 0)
    # with the literal Rule 2 start every item also meets the n pre-opened bins
    assert lib.fit_tests([5], [5, 3], 1, 1, 0, 1) == 2


def pin_bounded_space(lib, seed=18):
    """Reading G15 (Section 1's bounded-space FF / BF / WF).  (a) A bound of
    2m + n open bins is never reached, and closing a full bin never changes a
    later choice (a full bin holds no further item), so the packing is the
    unbounded one.  (b) With one open bin at a time there is nothing to
    choose: FF, BF and WF pack alike.  (c) The fit tests per item are the open
    bins, so a run never makes more than K per item; when every weight is B_1
    each bin fills and closes at once and only the empty bin it divided off
    is open for the next item: m - 1 fit tests (unbounded: (m-1)(m+2)/2).
    Plus the invariants of any packing."""
    rng = np.random.default_rng(seed)
    for t in range(60):
        m = int(rng.integers(0, 50))
        n = int(rng.integers(1, 5))
        B = sorted(rng.choice(np.arange(2, 60), size=n, replace=False).tolist(), reverse=True)
        w = rng.integers(1, B[0] + 1, size=m).tolist()
        pre = int(rng.integers(0, 2))
        for crit in (0, 1, 2, 3):
            ref = lib.pack(w, B, 1, crit, 0, pre, t)
            big = lib.pack(w, B, 1, crit, 0, pre, t, max_open=2 * m + n)
            assert big.bin_of_item.tolist() == ref.bin_of_item.tolist(), (w, B, crit, pre)
            assert big.bin_type.tolist() == ref.bin_type.tolist() and big.total == ref.total
        one = [lib.pack(w, B, 1, crit, 0, pre, max_open=1) for crit in (0, 1, 2)]
        assert one[0].bin_of_item.tolist() == one[1].bin_of_item.tolist() == one[2].bin_of_item.tolist(), (w, B)
        for K in (1, 2, 3, 7):
            crit = int(rng.integers(0, 4))
            r = lib.pack(w, B, 1, crit, 0, pre, t, max_open=K)
            check_packing(w, B, r)
            ft = lib.fit_tests(w, B, 1, crit, 0, pre, t, max_open=K)
            assert ft <= K * m, (w, B, K)
            if m > 0:
                assert lib.fit_tests([B[0]] * m, B, 1, crit, 0, 0, t, max_open=K) == m - 1


def textbook_decreasing(w, C, fit):
    """FFD / BFD: sort by non-increasing weight (stable), then the textbook
    first-fit or best-fit; bins reported per original item."""
    order = sorted(range(len(w)), key=lambda j: -w[j])
    idx, nb = fit([w[j] for j in order], C)
    out = [0] * len(w)
    for pos, j in enumerate(order):
        out[j] = idx[pos]
    return out, nb


def pin_presort(lib, trials=120, seed=19):
    """Reading G16.  With one bin type, FF and BF on the list sorted by
    non-increasing weight are the textbook First-Fit-Decreasing and
    Best-Fit-Decreasing (the n = 1 reduction of pin_textbook_n1 applied to
    the sorted list); a list that is already non-increasing packs exactly as
    without the flag; any pre-sorted packing satisfies the invariants."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        C = int(rng.integers(1, 60))
        m = int(rng.integers(0, 40))
        w = rng.integers(1, C + 1, size=m).tolist()
        for crit, ref in ((0, textbook_first_fit), (1, textbook_best_fit)):
            r = lib.pack(w, [C], 1, crit, 0, 0, 0, 2)
            idx, nbins = textbook_decreasing(w, C, ref)
            assert r.status == 0
            assert r.bin_of_item.tolist() == idx, (crit, C, w)
            assert r.num_bins == nbins and r.total == nbins * C
        n = int(rng.integers(1, 5))
        B = sorted(rng.choice(np.arange(2, 80), size=n, replace=False).tolist(), reverse=True)
        w = sorted(rng.integers(1, B[0] + 1, size=m).tolist(), reverse=True)
        h = int(rng.integers(1, 3))
        s = int(rng.integers(0, 6)) if h == 2 else 0
        crit = int(rng.integers(0, 4))
        a = lib.pack(w, B, h, crit, s, 0, t)
        b = lib.pack(w, B, h, crit, s, 0, t, 2)
        assert a.bin_of_item.tolist() == b.bin_of_item.tolist() and a.total == b.total, (w, B, h, crit)
        rng.shuffle(w)
        check_packing(w, B, lib.pack(w, B, h, crit, s, int(rng.integers(0, 2)), t, 2))


ALL_PINS = [pin_hand_examples, pin_splitmix64, pin_random_criterion_vectors, pin_textbook_n1, pin_optimum,
            pin_closed_forms, pin_h2_is_best_permutation, pin_h2_random_key, pin_invariants, pin_errors,
            pin_fit_tests, pin_bounded_space, pin_presort]


def failing_pins(lib):
    """Names of the pins this oracle copy fails (used by the mutant tests)."""
    bad = []
    for p in ALL_PINS:
        try:
            p(lib)
        except AssertionError:
            bad.append(p.__name__)
        except Exception as e:     # a crash counts as a detected mistake too
            bad.append(f"{p.__name__}:{type(e).__name__}")
    return bad
