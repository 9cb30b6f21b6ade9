"""Random option combinations through the C interface against the oracle,
element by element: heuristic, criterion (RANDOM included), sublist size
(the paper's 5- and 10-item sublists, the exhaustive 7..8-item search),
the literal Rule 2 start, Remark 3, the pre-sort and a bound on open bins,
on small random batches (instances shorter than the sublist size, empty
instances and one-type instances included), batched and plain."""
import numpy as np
import pytest

from gpu_util import assert_same, run_batch, run_oracle
from paper_1602_08735_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_1602_08735_gb300 import native  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1602_08735_gb300 import build
    build.build()
    native.load()


def _combos(rng, count):
    out = []
    while len(out) < count:
        h = int(rng.integers(1, 3))
        crit = int(rng.integers(0, 4))
        s = int(rng.choice([0, 1, 3, 5, 6, 7, 8])) if h == 2 else int(rng.choice([0, 0, 1, 3, 10]))
        preopen = int(rng.integers(0, 2))
        flags = int(rng.integers(0, 4))            # REMARK3 = 1, PRESORT = 2
        K = int(rng.choice([0, 0, 1, 2, 5, 32])) if h == 1 else 0
        if h == 2 and s >= 7:
            preopen = 0                             # the exhaustive search: no pre-opened bins
        if K and (flags & native.REMARK3):
            K = 0                                   # the bound is not combined with Remark 3
        if K:
            s = 0                                   # bounded space: one membrane system per instance
        out.append((h, crit, s, preopen, flags, K))
    return out


def _batch(rng, N, m_hi):
    inst = []
    for _ in range(N):
        m = int(rng.integers(0, m_hi + 1))
        inst.append(I.random_instance(rng, m, int(rng.integers(1, 6)), int(rng.choice([20, 150, 1000]))))
    return I.from_instances(inst)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_option_combinations(seed):
    rng = np.random.default_rng(900 + seed)
    for (h, crit, s, preopen, flags, K) in _combos(rng, 14):
        m_hi = 9 if (h == 2 and s >= 7) else 60
        b = _batch(rng, 24, m_hi)
        rs = int(rng.integers(0, 2**40))
        ref = run_oracle(b, h, crit, s, preopen, rs, flags, max_open=K)
        what = f"h{h} c{crit} s{s} pre{preopen} flags{flags} K{K}"
        assert_same(b, run_batch(b, h, crit, s, preopen, rs, flags=flags, max_open=K), ref, what)
        if rng.integers(0, 3) == 0:
            assert_same(b, run_batch(b, h, crit, s, preopen, rs, plain=True, flags=flags, max_open=K), ref,
                        what + " plain")
