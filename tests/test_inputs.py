"""The seeded synthetic inputs follow their stated recipes (CPU only): sizes,
capacity sets, weight ranges, mixture proportions and the log-uniform size
law of configs 1-5 and the paper-like config P."""
import numpy as np

from paper_1602_08735_gb300 import instances as I


def _frac_in(w, lo, hi):
    return float(np.mean((w >= lo) & (w <= hi)))


def test_config2_variants():
    w, B = I.config2("u").instance(0)
    assert len(w) == 10_000 and B.tolist() == [150, 120, 100, 80, 50]
    assert w.min() >= 1 and w.max() <= 150 and abs(w.mean() - 75.5) < 2.0
    w, B = I.config2("m").instance(0)
    assert len(w) == 10_000 and B.tolist() == [150, 120, 100, 80, 50]
    # 70 % from U[1,37], 30 % from U[75,150], nothing between
    assert _frac_in(w, 38, 74) == 0.0
    assert abs(_frac_in(w, 1, 37) - 0.7) < 0.02 and abs(_frac_in(w, 75, 150) - 0.3) < 0.02


def test_config3_size_law():
    """m log-uniform in [100, 10^4]: log m is uniform, so each decade holds
    half of the instances and the mean is (10^4 - 100) / ln(100) ~ 2150."""
    b = I.config3(N=4096)
    m = np.diff(b.w_off)
    assert m.min() >= 100 and m.max() <= 10_000
    assert abs(float(np.mean(m < 1000)) - 0.5) < 0.03
    assert abs(float(m.mean()) - (10_000 - 100) / np.log(100)) < 120
    ns = np.diff(b.B_off)
    assert set(np.unique(ns).tolist()) == {3, 5, 7}
    for i in range(0, b.N, 97):
        w, B = b.instance(i)
        assert len(set(B.tolist())) == len(B) and np.all(np.diff(B) < 0)
        assert 20 <= B[-1] and B[0] <= 1000 and w.max() <= B[0]


def test_config4_shape():
    b = I.config4(N=2, m=200_000)
    for i in range(b.N):
        w, B = b.instance(i)
        assert len(w) == 200_000 and B.tolist() == [1000, 800, 640, 500, 400, 300, 200]
        assert _frac_in(w, 101, 399) == 0.0
        assert abs(_frac_in(w, 1, 100) - 0.8) < 0.01 and abs(_frac_in(w, 400, 1000) - 0.2) < 0.01


def test_config5_requests():
    """Requests: m log-uniform in [100, 10^5], n in {3..7}; n = 5 takes
    config 2's capacities, other n B_1 = 150 and n - 1 distinct capacities in
    [50, 149]; even request ids draw U[1,150], odd ones config 2's mixture;
    arrivals are a Poisson stream at the stated rate."""
    reqs = I.config5(seed=5, num_requests=600, rate_per_s=200.0)
    t = np.array([r[0] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(float(gaps.mean()) - 1 / 200) < 0.0012
    ms = np.array([len(r[1]) for r in reqs])
    assert ms.min() >= 100 and ms.max() <= 100_000
    assert abs(float(np.mean(ms < 10_000)) - 2 / 3) < 0.06        # two of three decades
    for rid, (_, w, B) in enumerate(reqs):
        assert 3 <= len(B) <= 7 and np.all(np.diff(B) < 0) and w.max() <= B[0]
        if len(B) == 5:
            assert B.tolist() == [150, 120, 100, 80, 50]
        else:
            assert B[0] == 150 and B[1] <= 149 and B[-1] >= 50
        if rid % 2 == 1 and len(w) >= 2000:
            assert _frac_in(w, 38, 74) == 0.0


def test_paper_like_config():
    w, B = I.configP().instance(0)
    assert len(w) == 100_000 and B.tolist() == [300, 200, 100]
    assert w.min() >= 1 and w.max() <= 20
