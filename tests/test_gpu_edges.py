"""Edge cases of the CUDA best-shift path against the oracle: empty columns,
fixed variables, infinite bounds, an instance without rows, breakpoints on the
bounds and at x, ties across variables, and columns exactly at the boundaries
between the evaluation kernels (128 / 129 breakpoint entries)."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst

pytestmark = pytest.mark.gpu

B, I, C = inst.VAR_BIN, inst.VAR_INT, inst.VAR_CONT
LE, GE, EQ = inst.ROW_LE, inst.ROW_GE, inst.ROW_EQ


@pytest.fixture(scope="module")
def chap():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap as c
    c.load()
    return c


def check(chap, prob, tenure=3, steps=5, feas_tol=0.0):
    orc = Oracle(prob, feas_tol=feas_tol)
    bs = chap.BestShift(prob, tenure=tenure, feas_tol=feas_tol)
    for _ in range(steps):
        st = bs.state()
        _, _, nv = orc.residuals(st["x"])
        assert nv == st["nviol"]
        g = bs.best_shift()[:3]
        o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"])
        bad = np.nonzero((g[0] != o[0]) | (g[1] != o[1]) | (g[2] != o[2]))[0]
        assert len(bad) == 0, [(int(k), g[0][k], o[0][k], int(g[1][k]), int(o[1][k])) for k in bad[:8]]
        bs.step()
    bs.close()


def test_empty_columns_and_fixed_variables(chap):
    # vars 0..5 in rows, 6..8 in no row (one of each type), 9..11 fixed (one of each type)
    rows = [0, 0, 1, 1, 1, 2, 2, 3, 3]
    cols = [0, 9, 1, 2, 10, 3, 4, 5, 11]
    vals = [2.0, 1.0, -1.0, 3.0, 1.0, 1.0, 1.0, 2.0, -0.5]
    vt = [B, I, I, C, B, I, B, I, C, B, I, C]
    lb = [0, 0, -2, 0, 0, 0, 0, 0, 0, 1, 3, 0.5]
    ub = [1, 6, 4, 2.5, 1, 9, 1, 5, 3, 1, 3, 0.5]
    prob = inst.from_triplets("empty_fixed", 12, 4, rows, cols, vals, lb, ub, np.ones(12), [1.0, 0.0, 1.0, 2.0],
                              vt, [GE, LE, EQ, GE])
    check(chap, prob)


def test_infinite_bounds(chap):
    rows = [0, 0, 1, 1, 2, 2, 3]
    cols = [0, 1, 1, 2, 0, 2, 3]
    vals = [1.0, -2.0, 0.5, 1.0, -1.0, 4.0, 1.0]
    vt = [C, C, I, C]
    inf = np.inf
    lb = [-inf, 0.0, -inf, -5.0]
    ub = [inf, inf, 10.0, inf]
    prob = inst.from_triplets("infinite", 4, 4, rows, cols, vals, lb, ub, np.ones(4), [3.0, 1.0, -2.0, 7.5],
                              vt, [LE, GE, EQ, GE], x0=[0.0, 0.0, 0.0, 0.0])
    check(chap, prob)


def test_no_rows(chap):
    prob = inst.from_triplets("norows", 5, 0, [], [], [], np.zeros(5), [1, 4, 2.5, 1, 3], np.ones(5), [],
                              [B, I, C, B, I], [])
    bs = chap.BestShift(prob, tenure=3)
    xh, s, dc, mv = bs.best_shift()
    assert np.all(s == 0) and np.all(dc == 0) and mv.var == -1
    assert bs.step().var == -1
    bs.close()


def test_breakpoints_on_bounds_at_x_and_ties(chap):
    # integer vars in [0, 4]: rows whose breakpoints fall exactly on l, u and x;
    # vars 3 and 4 are identical copies, so their scores tie (the lower index wins)
    rows = [0, 1, 2, 3, 4, 4, 5, 5]
    cols = [0, 0, 1, 2, 3, 4, 3, 4]
    vals = [1.0, 1.0, -1.0, 2.0, 1.0, 1.0, 1.0, 1.0]
    rhs = [4.0, 0.0, -4.0, 2.0, 1.0, 1.0]
    prob = inst.from_triplets("onbounds", 5, 6, rows, cols, vals, np.zeros(5), np.full(5, 4.0), np.ones(5), rhs,
                              np.full(5, I), [LE, GE, LE, EQ, GE, GE], x0=[2.0, 1.0, 1.0, 0.0, 0.0])
    check(chap, prob, steps=8)


def _single_column(n_rows, vtype, dom, seed):
    """One column with n_rows single-variable rows (plus a partner column so that
    rows have two nonzeros), all breakpoints inside the domain."""
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs, sense = [], [], [], [], []
    for i in range(n_rows):
        a = float(rng.choice([1, 2, -1, -2]))
        t = float(rng.integers(0, dom))
        rows += [i, i]; cols += [0, 1]; vals += [a, 1.0]
        rhs.append(a * t + 0.5 if vtype == C else a * t)
        sense.append(int(rng.choice([LE, GE])))
    vt = [vtype, B]
    return inst.from_triplets(f"col{n_rows}", 2, n_rows, rows, cols, vals, [0.0, 0.0], [float(dom), 1.0], [1.0, 1.0],
                              rhs, vt, sense, x0=[0.0, 0.0])


@pytest.mark.parametrize("n_rows", [126, 127, 128])
@pytest.mark.parametrize("vtype", [I, C])
def test_kernel_boundary_columns(chap, n_rows, vtype):
    # entries = rows + 2 bounds: 128 stays on the short-column kernel, 129 and
    # 130 move to the counting sort (integer) or the CTA sort (continuous)
    prob = _single_column(n_rows, vtype, 64, seed=n_rows)
    bs = chap.BestShift(prob, tenure=3)
    expect_long = n_rows + 2 > 128
    if vtype == I:
        assert (bs.info.n_hist_cols == 1) == expect_long
    bs.close()
    check(chap, prob, steps=4)


def test_create_releases_everything_on_allocation_failure(chap, monkeypatch):
    """An injected device-allocation failure at several points of chap_bs_create
    returns CHAP_E_OOM and leaves no device memory behind; without it the same
    problem builds and runs."""
    import torch
    prob = inst.gen_general(seed=2, n=3000, m=1500, len_cap=200)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n_ok in (0, 1, 7, 20, 33):
        monkeypatch.setenv("CHAP_FAIL_ALLOC_AFTER", str(n_ok))
        with pytest.raises(chap.ChapError) as e:
            chap.BestShift(prob, tenure=5)
        assert e.value.status == chap.CHAP_E_OOM
    monkeypatch.delenv("CHAP_FAIL_ALLOC_AFTER")
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    bs = chap.BestShift(prob, tenure=5)
    bs.run(max_iters=20, stop_at_feasible=0)
    assert bs.state()["iter"] == 20
    bs.close()
