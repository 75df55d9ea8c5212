"""Randomised parity of the CUDA path with the oracle over instance shapes that
reach every evaluation kernel: binary, integer and continuous variables, short
columns (4 or 8 lanes), hub columns long enough for the CTA sort (continuous)
or the counting sort (integer), "=" rows, infinite and fixed bounds, random
weights, tabu stamps and best counts, with and without kept binary scores.

Coefficients, bounds and values are small dyadic rationals and the tolerance is
0, so double arithmetic is exact on both sides and every result is compared
bit for bit; a few dozen tabu steps are compared move by move as well.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst

pytestmark = pytest.mark.gpu

B, I, C = inst.VAR_BIN, inst.VAR_INT, inst.VAR_CONT


@pytest.fixture(scope="module")
def chap():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap as c
    c.load()
    return c


def random_instance(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 60))
    m = int(rng.integers(6, 70))
    vt = rng.choice(np.array([B, I, C], dtype=np.uint8), size=n, p=rng.dirichlet([2, 2, 1]))
    lb = np.where(vt == B, 0.0, rng.integers(-4, 3, size=n).astype(np.float64))
    ub = np.where(vt == B, 1.0, lb + rng.integers(0, 12, size=n))          # width 0: fixed
    inf_lo = (vt != B) & (rng.random(n) < 0.08)
    inf_hi = (vt != B) & (rng.random(n) < 0.08)
    lb[inf_lo] = -np.inf
    ub[inf_hi] = np.inf
    x0 = np.where(np.isfinite(lb), lb, np.where(np.isfinite(ub), ub, 0.0)).astype(np.float64)
    for j in range(n):
        lo = lb[j] if np.isfinite(lb[j]) else x0[j] - 5
        hi = ub[j] if np.isfinite(ub[j]) else x0[j] + 5
        if vt[j] == C:
            x0[j] = lo + np.floor(rng.random() * 4 * (hi - lo)) / 4
        else:
            x0[j] = float(rng.integers(int(lo), int(hi) + 1))
    # hub columns: a few variables in many rows (long lists: CTA or counting sort)
    hubs = rng.choice(n, size=int(rng.integers(0, 3)), replace=False) if rng.random() < 0.5 else []
    extra_rows = int(rng.integers(130, 260)) if len(hubs) else 0
    rows, cols, vals = [], [], []
    choices = np.array([-4, -2, -1, -0.5, 0.5, 1, 2, 4])
    for i in range(m + extra_rows):
        k = int(rng.integers(1, 6))
        js = set(rng.choice(n, size=min(k, n), replace=False).tolist())
        if i >= m:
            js.add(int(hubs[i % len(hubs)]))
        for j in sorted(js):
            rows.append(i); cols.append(j); vals.append(float(rng.choice(choices)))
    mm = m + extra_rows
    ax = np.zeros(mm)
    for r, c, v in zip(rows, cols, vals):
        ax[r] += v * x0[c]
    sense = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=mm, p=[0.4, 0.4, 0.2])
    rhs = ax + rng.integers(-3, 4, size=mm) * 0.5
    return inst.from_triplets(f"fuzz_{seed}", n, mm, rows, cols, vals, lb, ub, rng.integers(1, 5, size=n),
                              rhs, vt, sense, x0=x0)


def random_state(prob, orc, rng):
    x = prob.x0.copy()
    for j in range(prob.n):
        lo, hi = prob.lb[j], prob.ub[j]
        lo = lo if np.isfinite(lo) else x[j] - 4
        hi = hi if np.isfinite(hi) else x[j] + 4
        if rng.random() < 0.7:
            if prob.vtype[j] == C:
                x[j] = lo + np.floor(rng.random() * 4 * (hi - lo)) / 4
            else:
                x[j] = float(rng.integers(int(lo), int(hi) + 1))
    w = rng.integers(1, 6, size=orc.mn).astype(np.int32)
    it = int(rng.integers(0, 8))
    ti = rng.integers(0, it + 5, size=prob.n)
    td = rng.integers(0, it + 5, size=prob.n)
    _, _, nv = orc.residuals(x)
    return dict(x=x, w=w, tabu_inc=ti, tabu_dec=td, iter=it, best_nviol=max(0, nv - int(rng.integers(0, 3))))


def compare(bs, orc):
    st = bs.state()
    _, _, nv = orc.residuals(st["x"])
    assert nv == st["nviol"]
    g = bs.best_shift()
    o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"])
    bad = np.nonzero((g[0] != o[0]) | (g[1] != o[1]) | (g[2] != o[2]))[0]
    assert len(bad) == 0, [(int(k), g[0][k], o[0][k], int(g[1][k]), int(o[1][k]), int(g[2][k]), int(o[2][k]))
                           for k in bad[:6]]
    # the selected move: largest score, lowest variable
    best = int(np.argmax(o[1])) if o[1].max() > 0 else -1
    assert g[3].var == best
    assert np.array_equal(bs.residuals(), orc.residuals(st["x"])[0])


@pytest.mark.parametrize("seed", range(200))
def test_fuzz_states_and_steps(chap, seed):
    prob = random_instance(seed)
    orc = Oracle(prob, feas_tol=0.0)
    lazy = seed % 2
    bs = chap.BestShift(prob, tenure=3, feas_tol=0.0, lazy_binary=lazy)
    rng = np.random.default_rng(1000 + seed)
    for _ in range(3):
        bs.set_checkpoint(random_state(prob, orc, rng))
        compare(bs, orc)
    # a short trajectory from the last state, move by move
    st = bs.state()
    ost = dict(x=st["x"].copy(), w=st["w"].copy(), tabu_inc=st["tabu_inc"].copy(), tabu_dec=st["tabu_dec"].copy(),
               iter=st["iter"], best_nviol=st["best_nviol"])
    dyadic = True
    for k in range(30):
        mv = bs.step()
        tr = orc.run(ost, tenure=3, n_iters=1, stop_at_feasible=False)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
        if mv.var >= 0:
            assert mv.new_value == tr["val"][0]
        if not np.array_equal(ost["x"] * 1024.0, np.round(ost["x"] * 1024.0)):
            dyadic = False   # a non-dyadic continuous value: incremental and recomputed residuals may round apart
            break
    if dyadic:
        compare(bs, orc)
    bs.close()


def random_fp_instance(seed):
    """General coefficients (N(0,1) rows mixed with integer rows), tolerance 1e-9."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(10, 50))
    m = int(rng.integers(8, 50))
    vt = rng.choice(np.array([B, I, C], dtype=np.uint8), size=n, p=[0.4, 0.35, 0.25])
    lb = np.where(vt == B, 0.0, rng.integers(-3, 2, size=n).astype(np.float64))
    ub = np.where(vt == B, 1.0, lb + rng.integers(1, 30, size=n))
    xs = np.where(vt == C, lb + rng.random(n) * (ub - lb), np.floor(lb + rng.random(n) * (ub - lb + 1)))
    xs = np.minimum(xs, ub)
    rows, cols, vals = [], [], []
    for i in range(m):
        js = rng.choice(n, size=int(rng.integers(1, min(7, n) + 1)), replace=False)
        integral = rng.random() < 0.5
        for j in sorted(js.tolist()):
            rows.append(i); cols.append(j)
            vals.append(float(rng.integers(-9, 10) or 1) if integral else float(rng.normal()))
    ax = np.zeros(m)
    for r, c, v in zip(rows, cols, vals):
        ax[r] += v * xs[c]
    sense = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=m, p=[0.4, 0.4, 0.2])
    slack = rng.random(m) * 2.0
    rhs = np.where(sense == 0, ax + slack, np.where(sense == 1, ax - slack, ax))
    x0 = np.clip(np.zeros(n), lb, ub)
    return inst.from_triplets(f"fuzzfp_{seed}", n, m, rows, cols, vals, lb, ub, rng.integers(1, 5, size=n),
                              rhs, vt, sense, x0=x0)


@pytest.mark.parametrize("seed", range(60))
def test_fuzz_general_coefficients_within_tolerance(chap, seed):
    """Non-dyadic rows at feas_tol 1e-9, state-fed (the device recomputes the
    residuals of the state it reached, as the oracle does): every variable's
    score and violation change equal, its shift within 1e-9 relative."""
    prob = random_fp_instance(seed)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=3)
    for _ in range(4):
        bs.set_checkpoint(bs.state())
        st = bs.state()
        g = bs.best_shift()
        o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"])
        xok = np.abs(g[0] - o[0]) <= 1e-9 * np.maximum(1.0, np.abs(o[0]))
        bad = np.nonzero(~(xok & (g[1] == o[1]) & (g[2] == o[2])))[0]
        assert len(bad) == 0, [(int(k), g[0][k], o[0][k], int(g[1][k]), int(o[1][k])) for k in bad[:6]]
        bs.run(max_iters=5, stop_at_feasible=0)
    bs.close()
