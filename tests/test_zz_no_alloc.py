"""The fixed-scratch best-shift entry point against chap_bs_best_shift.

Some callers cannot give a handle device memory of its own for the counting
sort's scratch (many handles under a fixed device-memory budget, or a pool that
owns the device); chap_bs_best_shift_static_scratch runs the pass on a scratch
compiled into the library instead, and a handle created with
static_scratch_only holds none.  Collected last: the library-wide scratch is
shared by every handle, so this file runs after the other GPU tests have used
the library and must find the scratch cleared."""
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


def _hist_columns(n_cols, dom, rows_per_col, seed):
    """Integer columns with `rows_per_col` single-variable rows each (more than
    a warp sorts) and domain [0, dom - 1]: every column takes the counting sort."""
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs = [], [], [], []
    i = 0
    for j in range(n_cols):
        for _ in range(rows_per_col):
            a = float(rng.choice([1, 2, -1]))
            rows.append(i); cols.append(j); vals.append(a); rhs.append(a * float(rng.integers(0, dom)))
            i += 1
    sense = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=i, p=[0.45, 0.45, 0.1])
    return inst.from_triplets(f"hist_{n_cols}_{dom}", n_cols, i, rows, cols, vals, np.zeros(n_cols),
                              np.full(n_cols, float(dom - 1)), np.ones(n_cols), np.array(rhs),
                              np.full(n_cols, inst.VAR_INT), sense, x0=np.zeros(n_cols))


def test_static_scratch_two_layouts_alternating(chap):
    """Two handles whose counting-sort columns lay their bins out differently
    (3 columns of 2,000 values, 9 columns of 300) take turns on the one
    library-wide scratch: each pass must find it cleared by the other's."""
    pa, pb = _hist_columns(3, 2000, 150, 1), _hist_columns(9, 300, 140, 2)
    ha, hb = chap.BestShift(pa, tenure=5), chap.BestShift(pb, tenure=5)
    assert ha.info.n_hist_cols == 3 and hb.info.n_hist_cols == 9
    for _ in range(4):
        for bs, prob in ((ha, pa), (hb, pb)):
            ref = chap.chap_bs_best_shift(bs.h, prob.n)
            _same(ref, chap.chap_bs_best_shift_static_scratch(bs.h, prob.n))
            bs.run(max_iters=3, stop_at_feasible=0)
    ha.close()
    hb.close()


def test_static_scratch_rejects_too_many_columns(chap):
    # 257 counting-sorted columns of 11 values: few bins, one column too many
    prob = _hist_columns(257, 11, 130, 3)
    bs = chap.BestShift(prob, tenure=10)
    assert bs.info.n_hist_cols == 257
    with pytest.raises(chap.ChapError) as ei:
        chap.chap_bs_best_shift_static_scratch(bs.h, prob.n)
    assert ei.value.status == chap.CHAP_E_UNSUPPORTED and "static scratch" in str(ei.value)
    bs.close()


def test_handle_without_own_scratch(chap):
    """static_scratch_only: the handle holds no counting-sort scratch; its
    passes run through the fixed scratch and equal a regular handle's, and the
    calls that would use its own scratch refuse with CHAP_E_STATE."""
    prob = inst.gen_skewed(seed=5, n=50_000, m=25_000, n_dense=3, dense_len=6_000)
    reg = chap.BestShift(prob, tenure=10)
    own = chap.BestShift(prob, tenure=10, static_scratch_only=1)
    assert own.info.n_hist_cols == 3
    for call in (lambda: chap.chap_bs_best_shift(own.h, prob.n), lambda: chap.chap_bs_step(own.h),
                 lambda: own.run(max_iters=2)):
        with pytest.raises(chap.ChapError) as ei:
            call()
        assert ei.value.status == chap.CHAP_E_STATE
    for _ in range(3):
        ref = chap.chap_bs_best_shift(reg.h, prob.n)
        _same(ref, chap.chap_bs_best_shift_static_scratch(own.h, prob.n))
        mv = ref[3]
        for bs in (reg, own):
            bs.apply(mv.var, mv.new_value)
    own.close()
    reg.close()
