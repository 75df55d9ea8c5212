"""Pins of the CPU oracle against facts that do not come from the oracle itself.

- hand-derived worked examples (tests/golden/worked_examples.json);
- exhaustive enumeration of every integer domain value (oracle/definition.py,
  exact rationals) on many tiny instances, with random tabu/aspiration states;
- a dense grid over continuous domains: no admissible point beats the reported
  best (the step-function claim of Sec. 3.1);
- binary variables scored as integers in [0, 1] give the flip result;
- closed form of a single-row problem;
- trajectory invariant: each applied move's score equals the penalty sum
  recomputed from the whole residual vector before and after (scipy.sparse);
- determinism across thread counts.
"""
from fractions import Fraction as F

import numpy as np
import pytest
import scipy.sparse as sp

from conftest import fp_tiny, golden_cases, problem_from_case
from oracle import definition
from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst


def _state(prob, case):
    return (np.array(case["x"], float), np.array(case["w"], np.int32),
            np.array(case["tabu_inc"], np.int64), np.array(case["tabu_dec"], np.int64),
            int(case["iter"]), int(case["best_nviol"]))


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_worked_examples(case):
    prob = problem_from_case(case)
    tol = case.get("feas_tol", 1e-9)
    orc = Oracle(prob, feas_tol=tol)
    x, w, ti, td, it, bn = _state(prob, case)
    _, _, nviol = orc.residuals(x)
    xh, sh, dc = orc.best_shift(x, w, ti, td, it, nviol, bn)
    got = [[float(a), int(b), int(c)] for a, b, c in zip(xh, sh, dc)]
    assert got == [[float(a), int(b), int(c)] for a, b, c in case["expect"]]
    if "expect_best_var" in case:
        assert int(np.argmax(sh)) == case["expect_best_var"]
    # every listed domain score agrees with the exact definition
    rows = definition.normalised_rows(prob, tol)
    xf = [F(float(v)) for v in x]
    for key in ("domain_scores_half", "candidate_scores_half", "domain_scores_half_var0"):
        for v, s in case.get(key, {}).items():
            assert definition.score(rows, xf, w, 0, F(v))[0] == s, (key, v)
    if "candidates_var0" in case:
        assert definition.candidate_values(prob, x, 0, tol) == {F(v) for v in case["candidates_var0"]}
    if all(t != inst.VAR_CONT for t in case["vtype"]):
        _check_against_exhaustive(prob, x, w, ti, td, it, nviol, bn, tol, xh, sh, dc)


def _check_against_exhaustive(prob, x, w, ti, td, it, nviol, bn, tol, xh, sh, dc):
    """The oracle's score is the maximum over the whole domain, its value attains it,
    and it is the closest maximiser among the bounds and breakpoints."""
    ex = definition.exhaustive_max(prob, x, w, ti, td, it, nviol, bn, feas_tol=tol)
    for j, (best, arg) in enumerate(ex):
        if best is None or best <= 0:
            assert (float(xh[j]), int(sh[j]), int(dc[j])) == (float(x[j]), 0, 0), j
            continue
        assert int(sh[j]) == best, j
        v = int(xh[j])
        assert v == xh[j] and v in arg and int(dc[j]) == arg[v], j
        cands = definition.candidate_values(prob, x, j, tol)
        tied = [u for u in arg if F(u) in cands]
        assert v == min(tied, key=lambda u: (abs(u - float(x[j])), u)), j


def _random_tabu(rng, n, it):
    ti = rng.integers(0, it + 3, size=n).astype(np.int64)
    td = rng.integers(0, it + 3, size=n).astype(np.int64)
    return ti, td


@pytest.mark.parametrize("seed", range(60))
@pytest.mark.parametrize("dyadic", [False, True])
def test_exhaustive_integer_domains(seed, dyadic):
    prob = inst.gen_tiny_mixed(seed, n=6, m=5, max_len=4, dom=12, cont_frac=0.0, dyadic=dyadic)
    rng = np.random.default_rng(1000 + seed)
    tol = 0.0 if dyadic else 1e-9
    orc = Oracle(prob, feas_tol=tol)
    x = prob.x0
    w = rng.integers(1, 4, size=orc.mn).astype(np.int32)
    it = 2
    ti, td = _random_tabu(rng, prob.n, it)
    _, _, nviol = orc.residuals(x)
    bn = nviol - int(rng.integers(0, 2))
    xh, sh, dc = orc.best_shift(x, w, ti, td, it, nviol, bn)
    _check_against_exhaustive(prob, x, w, ti, td, it, nviol, bn, tol, xh, sh, dc)


@pytest.mark.parametrize("seed", range(40))
def test_exhaustive_integer_domains_with_tolerance(seed):
    """Non-integral rows (dyadic coefficients) with a tolerance eps = 0.25 max(1,|b|):
    the integer breakpoints are the step points of the tolerance-aware penalty,
    so the maximum over the whole domain is still attained at a candidate."""
    prob = inst.gen_tiny_mixed(500 + seed, n=6, m=5, max_len=4, dom=12, cont_frac=0.0, dyadic=True)
    rng = np.random.default_rng(1500 + seed)
    orc = Oracle(prob, feas_tol=0.25)
    x = prob.x0
    w = rng.integers(1, 4, size=orc.mn).astype(np.int32)
    ti, td = _random_tabu(rng, prob.n, 2)
    _, _, nviol = orc.residuals(x)
    bn = nviol - int(rng.integers(0, 2))
    xh, sh, dc = orc.best_shift(x, w, ti, td, 2, nviol, bn)
    _check_against_exhaustive(prob, x, w, ti, td, 2, nviol, bn, 0.25, xh, sh, dc)


@pytest.mark.parametrize("seed", range(40))
def test_continuous_grid_never_beats_best(seed):
    prob = inst.gen_tiny_mixed(seed, n=5, m=5, max_len=4, dom=6, cont_frac=0.5, dyadic=True)
    rng = np.random.default_rng(2000 + seed)
    orc = Oracle(prob, feas_tol=0.0)
    x = prob.x0
    w = rng.integers(1, 4, size=orc.mn).astype(np.int32)
    it = 1
    ti, td = _random_tabu(rng, prob.n, it)
    _, _, nviol = orc.residuals(x)
    bn = nviol
    xh, sh, dc = orc.best_shift(x, w, ti, td, it, nviol, bn)
    rows = definition.normalised_rows(prob, 0.0)
    xf = [F(float(v)) for v in x]
    for j in range(prob.n):
        if prob.vtype[j] != inst.VAR_CONT:
            continue
        if sh[j] > 0:
            s, d = definition.score(rows, xf, w, j, F(float(xh[j])))
            assert (s, d) == (int(sh[j]), int(dc[j]))
            assert definition.admissible(F(float(xh[j])), xf[j], j, d, ti, td, it, nviol, bn)
        lo, hi = F(float(prob.lb[j])), F(float(prob.ub[j]))
        grid = [lo + (hi - lo) * F(q, 256) for q in range(257)]
        for g in grid:
            if g == xf[j]:
                continue
            s, d = definition.score(rows, xf, w, j, g)
            if definition.admissible(g, xf[j], j, d, ti, td, it, nviol, bn):
                assert s <= max(int(sh[j]), 0), (j, g, s, sh[j])


@pytest.mark.parametrize("seed", range(80))
def test_continuous_grid_with_tolerance_exact_classification(seed):
    """feas_tol = 1e-9 on N(0,1) rows, every classification in exact rationals
    (violated iff r > eps): the oracle's score is the exact score of its value;
    it is the best admissible score over the exact candidate set (finite bounds
    and the tight points of rows not satisfied within eps -- a row with
    |r| <= eps contributes none), its value is that set's tie-break winner (largest
    score, smallest |x - xbar|, smaller x) up to the rounding of the breakpoint;
    and no point of a dense grid of [l, u] or next to a candidate scores
    higher."""
    tol = 1e-9
    prob, x = fp_tiny(seed, tol)
    rng = np.random.default_rng(4000 + seed)
    orc = Oracle(prob, feas_tol=tol)
    w = rng.integers(1, 4, size=orc.mn).astype(np.int32)
    it = 2
    ti, td = _random_tabu(rng, prob.n, it)
    _, _, nviol = orc.residuals(x)
    exact_r, exact_v, exact_nv = definition.residual_state(prob, x, tol)
    assert nviol == exact_nv
    bn = nviol - int(rng.integers(0, 2))
    xh, sh, dc = orc.best_shift(x, w, ti, td, it, nviol, bn)
    rows = definition.normalised_rows(prob, tol)
    xf = [F(float(v)) for v in x]
    for j in range(prob.n):
        if prob.vtype[j] != inst.VAR_CONT:
            continue
        scored = []
        for c in definition.candidate_values(prob, x, j, tol):
            s, d = definition.score(rows, xf, w, j, c)
            if definition.admissible(c, xf[j], j, d, ti, td, it, nviol, bn):
                scored.append((s, c, d))
        best = max([s for s, _, _ in scored], default=None)
        if best is None or best <= 0:
            assert (float(xh[j]), int(sh[j]), int(dc[j])) == (float(x[j]), 0, 0), j
        else:
            win = min((c for s, c, _ in scored if s == best), key=lambda c: (abs(c - xf[j]), c))
            assert int(sh[j]) == best, (j, int(sh[j]), best)
            assert abs(F(float(xh[j])) - win) <= F(1, 10**12) * max(F(1), abs(win)), (j, float(xh[j]), float(win))
            s, d = definition.score(rows, xf, w, j, F(float(xh[j])))
            assert (s, d) == (int(sh[j]), int(dc[j])), j
        lo, hi = F(float(prob.lb[j])), F(float(prob.ub[j]))
        pts = [lo + (hi - lo) * F(q, 400) for q in range(401)]
        for _, c, _ in scored:
            pts += [c - F(1, 10**4), c + F(1, 10**4)]
        for g in pts:
            if g == xf[j] or not lo <= g <= hi:
                continue
            s, d = definition.score(rows, xf, w, j, g)
            if definition.admissible(g, xf[j], j, d, ti, td, it, nviol, bn):
                assert s <= max(int(sh[j]), 0), (j, float(g), s, int(sh[j]))


def test_fp_tiny_states_exercise_the_tolerance():
    """The generator above does produce rows satisfied within eps but not
    exactly tight (0 < |r| <= eps), the case the tight-row rule is about."""
    hits = 0
    for seed in range(80):
        prob, x = fp_tiny(seed, 1e-9)
        r, _, _ = definition.residual_state(prob, x, 1e-9)
        for rk, (_, _, eps) in zip(r, definition.normalised_rows(prob, 1e-9)):
            hits += int(0 < abs(rk) <= eps)
    assert hits >= 20, hits


@pytest.mark.parametrize("seed", range(20))
def test_binary_equals_integer_zero_one(seed):
    prob = inst.gen_tiny_mixed(seed, n=8, m=6, max_len=5, dom=5, cont_frac=0.0, dyadic=False)
    rng = np.random.default_rng(3000 + seed)
    orc = Oracle(prob)
    x = prob.x0
    w = rng.integers(1, 4, size=orc.mn).astype(np.int32)
    ti, td = _random_tabu(rng, prob.n, 1)
    _, _, nviol = orc.residuals(x)
    a = orc.best_shift(x, w, ti, td, 1, nviol, nviol)
    prob2 = inst.from_triplets("as_int", prob.n, prob.m,
                               np.repeat(np.arange(prob.m), np.diff(prob.row_ptr)), prob.col_idx,
                               prob.row_val, prob.lb, prob.ub, prob.obj, prob.rhs,
                               np.where(prob.vtype == inst.VAR_BIN, inst.VAR_INT, prob.vtype), prob.sense,
                               x0=prob.x0)
    b = Oracle(prob2).best_shift(x, w, ti, td, 1, nviol, nviol)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("a,b,xbar,ub", [(3, 10, 9, 12), (2, 7, 8, 8), (5, 4, 3, 6), (1, 0, 5, 5)])
def test_single_row_closed_form(a, b, xbar, ub):
    """One integer var, one row a*x <= b violated at xbar: the best shift is the
    largest feasible value floor(b/a) (score +w, i.e. 2 half units) when it is in
    the domain; values between it and xbar only reduce the violation (+w/2)."""
    prob = inst.from_triplets("single", 1, 1, [0], [0], [float(a)], lb=[0], ub=[ub], obj=[1],
                              rhs=[float(b)], vtype=[inst.VAR_INT], sense=[inst.ROW_LE], x0=[xbar])
    orc = Oracle(prob)
    x = np.array([float(xbar)])
    _, _, nviol = orc.residuals(x)
    assert nviol == 1
    xh, sh, dc = orc.best_shift(x, np.ones(1, np.int32), np.zeros(1, np.int64), np.zeros(1, np.int64), 0, 1, 1)
    assert xh[0] == b // a and sh[0] == 2 and dc[0] == -1


def _normalised_matrix(prob):
    """Independent normalisation with scipy: returns (A_norm csr, b_norm)."""
    A = sp.csr_matrix((prob.row_val, prob.col_idx, prob.row_ptr), shape=(prob.m, prob.n))
    blocks, rhs = [], []
    for i in range(prob.m):
        s = prob.sense[i]
        if s in (inst.ROW_LE, inst.ROW_EQ):
            blocks.append(A[i]); rhs.append(prob.rhs[i])
        if s in (inst.ROW_GE, inst.ROW_EQ):
            blocks.append(-A[i]); rhs.append(-prob.rhs[i])
    return sp.vstack(blocks).tocsr(), np.array(rhs)


@pytest.mark.parametrize("which", ["setcover", "tiny_int"])
def test_move_score_equals_recomputed_penalty(which):
    if which == "setcover":
        prob = inst.gen_setcover(seed=3, n=300, m=150, k=8)
        iters = 300
    else:
        prob = inst.gen_tiny_mixed(7, n=12, m=10, max_len=5, dom=10, dyadic=False)
        iters = 200
    orc = Oracle(prob)
    An, bn = _normalised_matrix(prob)
    st = orc.initial_state()
    for _ in range(iters):
        x0 = st["x"].copy()
        w0 = st["w"].copy()
        tr = orc.run(st, tenure=5, n_iters=1, stop_at_feasible=True)
        if len(tr["var"]) == 0:
            break
        r0 = An @ x0 - bn
        r1 = An @ st["x"] - bn
        v0, v1 = r0 > 0, r1 > 0
        p = np.where(~v0 & v1, -2 * w0, np.where(v0 & ~v1, 2 * w0,
                     np.where(v0 & v1 & (r1 < r0), w0, np.where(v0 & v1 & (r1 > r0), -w0, 0))))
        if tr["var"][0] >= 0:
            assert int(p.sum()) == int(tr["s_half"][0]) > 0
            assert np.count_nonzero(x0 != st["x"]) == 1
        else:
            assert np.array_equal(st["x"], x0)
            assert np.array_equal(st["w"] - w0, v0.astype(np.int32))
        assert int(v1.sum()) == int(tr["nviol_after"][0])
        assert (st["w"] >= w0).all()


def test_thread_count_does_not_change_trajectory():
    prob = inst.gen_setcover(seed=1, n=500, m=250, k=8)
    orc = Oracle(prob)
    a, b = orc.initial_state(), orc.initial_state()
    ta = orc.run(a, tenure=10, n_iters=200, nthreads=1)
    tb = orc.run(b, tenure=10, n_iters=200, nthreads=4)
    for k in ta:
        assert np.array_equal(ta[k], tb[k])
    assert np.array_equal(a["x"], b["x"]) and np.array_equal(a["w"], b["w"])


def test_tabu_trajectory_hand_derived():
    """Tabu stamps (iter + 1 + tenure), aspiration and weight updates over seven
    iterations against a trajectory worked out by hand
    (tests/golden/tabu_example.json): a stamp one iteration short would take
    the move at iteration 5 instead of 6."""
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tabu_example.json")))
    pr = g["problem"]
    rows, cols, vals = [], [], []
    for i, r in enumerate(pr["rows"]):
        for j, a in r["coefs"]:
            rows.append(i); cols.append(j); vals.append(float(a))
    prob = inst.from_triplets("tabu_golden", pr["n"], len(pr["rows"]), rows, cols, vals, np.array(pr["lb"], float),
                              np.array(pr["ub"], float), np.ones(pr["n"]),
                              np.array([r["rhs"] for r in pr["rows"]], float), np.array(pr["vtype"], np.uint8),
                              np.array([r["sense"] for r in pr["rows"]], np.uint8), x0=np.array(pr["x0"], float))
    orc = Oracle(prob)
    st = orc.initial_state()
    tr = orc.run(st, pr["tenure"], len(g["steps"]), stop_at_feasible=False)
    assert tr["var"].tolist() == [s["var"] for s in g["steps"]]
    assert tr["s_half"].tolist() == [s["s_half"] for s in g["steps"]]
    for k, s in enumerate(g["steps"]):
        if s["var"] >= 0:
            assert tr["val"][k] == s["val"], k
    assert tr["nviol_after"].tolist() == g["nviol_after"]
    assert st["x"].tolist() == g["x_after"] and st["w"].tolist() == g["w_after"]
    assert st["tabu_inc"].tolist() == g["tabu_inc_after"] and st["tabu_dec"].tolist() == g["tabu_dec_after"]
    assert st["best_nviol"] == g["best_nviol_after"]
