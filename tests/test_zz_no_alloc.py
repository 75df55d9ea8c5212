"""The static-scratch best-shift entry point (no per-handle scratch) against
chap_bs_best_shift.  Collected last: the library-wide scratch is shared by
every handle, so this file runs after the other GPU tests have used the
library and must find the scratch cleared."""
import numpy as np
import pytest

from paper_2605_05086_gb300 import instances as inst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chap():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap as c
    c.load()
    return c


def _same(a, b):
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    assert (a[3].var, a[3].score_half, a[3].dnviol) == (b[3].var, b[3].score_half, b[3].dnviol)


def test_static_scratch_matches_handle_scratch(chap):
    prob = inst.gen_skewed(seed=3, n=200_000, m=100_000, n_dense=4, dense_len=20_000)
    bs = chap.BestShift(prob, tenure=10)
    assert bs.info.n_hist_cols == 4
    for _ in range(3):
        ref = chap.chap_bs_best_shift(bs.h, prob.n)
        # two calls in a row: the first must leave the scratch cleared for the second
        a = chap.chap_bs_best_shift_static_scratch(bs.h, prob.n)
        b = chap.chap_bs_best_shift_static_scratch(bs.h, prob.n)
        _same(ref, a)
        _same(ref, b)
        bs.run(max_iters=50, stop_at_feasible=0)
    bs.close()


def test_static_scratch_rejects_oversized(chap):
    # 17 integer columns with 4096-value domains and 130 rows each take the
    # counting sort: 17 * 4096 bins > 65536
    rng = np.random.default_rng(0)
    rows, cols, vals, rhs = [], [], [], []
    i = 0
    for j in range(17):
        for _ in range(130):
            rows.append(i); cols.append(j); vals.append(1.0); rhs.append(float(rng.integers(0, 4096)))
            i += 1
    n, m = 17, i
    prob = inst.from_triplets("wide_domains", n, m, rows, cols, vals, np.zeros(n), np.full(n, 4095.0), np.ones(n),
                              np.array(rhs), np.full(n, inst.VAR_INT), np.zeros(m, np.uint8), x0=np.zeros(n))
    bs = chap.BestShift(prob, tenure=10)
    assert bs.info.n_hist_cols == 17
    with pytest.raises(chap.ChapError) as ei:
        chap.chap_bs_best_shift_static_scratch(bs.h, prob.n)
    assert "static scratch" in str(ei.value)
    # the handle stays usable through the regular entry point
    chap.chap_bs_best_shift(bs.h, prob.n)
    bs.close()
