"""Columns whose breakpoint lists are longer than one CTA sorts (over 8192
entries): continuous columns and integer columns with domains wider than the
counting sort takes.  They run on the multi-CTA merge-sort path (runs sorted
per CTA, pairwise merge rounds across the grid, a tiled scan with a carry).
Dyadic coefficients and values with feas_tol = 0 make double arithmetic exact
on both sides, so the CUDA path must equal the oracle bit for bit."""
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


def long_instance(seed, long_types, rows_per_long=10_000, n_other=300, dom_long=1_000_000, eq_frac=0.2):
    """len(long_types) hub variables (continuous in [0, 1024] or integer in
    [0, dom_long]), each in rows_per_long rows together with one or two short
    variables; breakpoints spread over the hub's domain."""
    rng = np.random.default_rng(seed)
    nh = len(long_types)
    n = nh + n_other
    vt = np.concatenate([np.array(long_types, dtype=np.uint8),
                         rng.choice(np.array([B, I, C], dtype=np.uint8), size=n_other)])
    lb = np.zeros(n)
    ub = np.where(vt == B, 1.0, np.where(vt == I, 20.0, 16.0))
    ub[:nh] = np.where(vt[:nh] == C, 1024.0, float(dom_long))
    x0 = np.where(vt == C, np.floor(rng.random(n) * ub * 4) / 4, np.floor(rng.random(n) * (ub + 1)))
    x0 = np.minimum(x0, ub)
    rows, cols, vals, rhs, sense = [], [], [], [], []
    coef = np.array([-4.0, -2.0, -1.0, -0.5, 0.5, 1.0, 2.0, 4.0])
    i = 0
    for h in range(nh):
        for _ in range(rows_per_long):
            js = sorted(set([h] + rng.choice(np.arange(nh, n), size=int(rng.integers(1, 3)), replace=False).tolist()))
            act = 0.0
            for j in js:
                a = float(rng.choice(coef)) if (vt[j] == C or vt[h] == C) else float(rng.choice([-3, -2, -1, 1, 2, 3]))
                rows.append(i); cols.append(j); vals.append(a)
                # breakpoint target of the hub: a value spread over its domain
                act += a * (np.floor(rng.random() * ub[h] * 4) / 4 if (j == h and vt[h] == C)
                            else (float(rng.integers(0, int(ub[h]) + 1)) if j == h else x0[j]))
            s = int(rng.choice([0, 1, 2], p=[(1 - eq_frac) / 2, (1 - eq_frac) / 2, eq_frac]))
            rhs.append(act + float(rng.integers(-2, 3)) * (0.5 if vt[h] == C else 1.0))
            sense.append(s)
            i += 1
    return inst.from_triplets(f"long_{seed}", n, i, rows, cols, vals, lb, ub, np.ones(n), np.array(rhs), vt,
                              np.array(sense, dtype=np.uint8), x0=x0)


def _pass_exact(bs, orc, vars_=None):
    st = bs.state()
    g = bs.best_shift()
    o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"],
                       vars=vars_)
    gx, gs, gd = (a if vars_ is None else a[vars_] for a in g[:3])
    bad = np.nonzero((gx != o[0]) | (gs != o[1]) | (gd != o[2]))[0]
    assert len(bad) == 0, [(int(k), gx[k], o[0][k], int(gs[k]), int(o[1][k]), int(gd[k]), int(o[2][k]))
                           for k in bad[:6]]
    return g


@pytest.mark.parametrize("types", [[C], [I], [C, I], [C, C, I]])
def test_long_lists_exact(chap, types):
    prob = long_instance(len(types) * 7 + int(types[0]), types)
    orc = Oracle(prob, feas_tol=0.0)
    bs = chap.BestShift(prob, tenure=3, feas_tol=0.0)
    assert bs.info.n_long_cols == len(types)
    rng = np.random.default_rng(11)
    vars_ = np.unique(np.concatenate([np.arange(len(types)), rng.choice(prob.n, 60, replace=False)])).astype(np.int32)
    for _ in range(3):
        _pass_exact(bs, orc, vars_)
        bs.run(max_iters=4, stop_at_feasible=0)
    bs.close()


def test_long_list_trajectory_graph(chap):
    """The tabu loop through the CUDA graph (every kernel of the long path
    recorded once per iteration) against the oracle, move by move."""
    prob = long_instance(3, [C, I], rows_per_long=8_000, n_other=120)
    orc = Oracle(prob, feas_tol=0.0)
    bs = chap.BestShift(prob, tenure=4, feas_tol=0.0, graph_iters=4)
    assert bs.info.n_long_cols == 2
    bs.set_state(prob.x0)
    ost = orc.initial_state(prob.x0)
    tr = orc.run(ost, tenure=4, n_iters=12, stop_at_feasible=False)
    bs.run(max_iters=12, stop_at_feasible=0)
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    assert st["iter"] == 12 and len(tr["var"]) == 12
    bs.close()


def test_long_list_scratch_returns_to_zero(chap):
    """Two handles with long lists take turns: each pass must find its column
    accumulators cleared by its own previous pass."""
    pa = long_instance(5, [I], rows_per_long=9_000, n_other=80)
    pb = long_instance(6, [C], rows_per_long=9_000, n_other=80)
    oa, ob = Oracle(pa, feas_tol=0.0), Oracle(pb, feas_tol=0.0)
    ha = chap.BestShift(pa, tenure=3, feas_tol=0.0)
    hb = chap.BestShift(pb, tenure=3, feas_tol=0.0)
    for _ in range(3):
        for bs, orc in ((ha, oa), (hb, ob)):
            _pass_exact(bs, orc, np.array([0], dtype=np.int32))
            _pass_exact(bs, orc, np.array([0], dtype=np.int32))
            bs.step()
    ha.close()
    hb.close()
