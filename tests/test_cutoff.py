"""Objective cutoff (Sec. 3.2, "Solution Pool": the best known objective is
imposed as a cutoff constraint so that the search keeps looking for improving
solutions).

CPU part: the oracle's cutoff run pinned by facts that do not come from the
oracle itself -- every recorded solution is feasible for the original rows and
its objective is c^T x (both recomputed here with scipy.sparse), recorded
objectives fall by at least delta, no recorded objective is below the optimum
found by enumerating every point of tiny binary instances, the run is the plain
run until its first feasible iteration, and the tightened rhs is y - delta
(with the tolerance floor on a non-integral row).

GPU part (through the C ABI): the device search under the cutoff against the
oracle, bit-exact on integral instances (every move, every recorded solution,
the best solution copy) and on dyadic mixed instances.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst


def feasible(prob, x, tol=0.0):
    """Every original row satisfied at x (within tol * max(1, |b|))."""
    A = sp.csr_matrix((prob.row_val, prob.col_idx, prob.row_ptr), shape=(prob.m, prob.n))
    y = A @ x
    eps = tol * np.maximum(1.0, np.abs(prob.rhs))
    le = y <= prob.rhs + eps
    ge = y >= prob.rhs - eps
    ok = np.where(prob.sense == inst.ROW_LE, le, np.where(prob.sense == inst.ROW_GE, ge, le & ge))
    return bool(ok.all())


# ------------------------------------------------------------------ oracle pins (CPU)


def test_oracle_cutoff_solutions_feasible_and_improving():
    base = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    prob = inst.with_objective_row(base)
    orc = Oracle(prob)
    st = orc.initial_state()
    cut = dict(row=prob.m - 1, delta=3.0)
    count, prev = 0, None
    for _ in range(30):
        orc.run_cutoff(st, 10, 100, cut)
        if cut["count"] > count:
            xb = cut["x_best"]
            assert feasible(base, xb)
            assert cut["obj"] == float(base.obj @ xb)
            if prev is not None:
                assert cut["obj"] <= prev - 3.0
            assert cut["rhs"] == cut["obj"] - 3.0
            count, prev = cut["count"], cut["obj"]
    assert cut["count"] >= 2


def test_oracle_cutoff_equals_plain_run_until_first_solution():
    prob = inst.with_objective_row(inst.gen_setcover(seed=1, n=800, m=400, k=8))
    orc_a, orc_b = Oracle(prob), Oracle(prob)
    sa, sb = orc_a.initial_state(), orc_b.initial_state()
    plain = orc_a.run(sa, 10, 2000, stop_at_feasible=True)
    cut = dict(row=prob.m - 1, delta=1.0)
    tr = orc_b.run_cutoff(sb, 10, len(plain["var"]), cut)
    assert plain["nviol_after"][-1] == 0
    assert np.array_equal(plain["var"], tr["var"]) and np.array_equal(plain["val"], tr["val"])
    assert np.array_equal(plain["s_half"], tr["s_half"])
    # the last iteration found the first solution: the tightened row is violated
    assert np.array_equal(plain["nviol_after"][:-1], tr["nviol_after"][:-1])
    assert tr["nviol_after"][-1] == 1 and cut["count"] == 1 and cut["best_iter"] == len(plain["var"])
    assert sb["best_nviol"] == 1            # the record of the tightened problem
    assert np.array_equal(cut["x_best"], sa["x"])


@pytest.mark.parametrize("seed", range(6))
def test_oracle_cutoff_never_below_enumerated_optimum(seed):
    base = inst.gen_setcover(seed=10 + seed, n=12, m=6, k=3)
    prob = inst.with_objective_row(base)
    best = None
    for bits in itertools.product((0.0, 1.0), repeat=base.n):
        x = np.array(bits)
        if feasible(base, x):
            v = float(base.obj @ x)
            best = v if best is None else min(best, v)
    orc = Oracle(prob)
    st = orc.initial_state()
    cut = dict(row=prob.m - 1, delta=1.0)
    prev = None
    for _ in range(400):
        before = cut.get("count", 0)
        orc.run_cutoff(st, 2, 1, cut)
        if cut["count"] > before:
            assert feasible(base, cut["x_best"]) and cut["obj"] == float(base.obj @ cut["x_best"])
            assert prev is None or cut["obj"] <= prev - 1.0
            prev = cut["obj"]
    assert best is not None and cut["count"] >= 1
    assert cut["obj"] >= best


def test_oracle_cutoff_fp_row_tolerance_floor():
    # continuous variables make the objective row non-integral: the required
    # improvement is raised to 4 feas_tol max(1, |y|)
    for seed in range(40):
        base = inst.gen_tiny_mixed(seed, n=10, m=6, max_len=4, dom=8, cont_frac=0.3, dyadic=True, eq_frac=0.0)
        if not (base.vtype == inst.VAR_CONT).any():
            continue
        prob = inst.with_objective_row(base)
        tol = 1e-3
        orc = Oracle(prob, feas_tol=tol)
        st = orc.initial_state()
        cut = dict(row=prob.m - 1, delta=1e-12)
        for _ in range(300):
            before = cut.get("count", 0)
            orc.run_cutoff(st, 2, 1, cut)
            if cut["count"] > before:
                y = cut["obj"]
                assert cut["rhs"] == y - 4.0 * tol * max(1.0, abs(y))
                assert feasible(base, cut["x_best"], tol)
                assert abs(y - float(base.obj @ cut["x_best"])) <= 1e-9 * max(1.0, abs(y))
                return
    pytest.fail("no tiny mixed instance reached a solution")


# ------------------------------------------------------------------ device search (GPU)


@pytest.fixture(scope="module")
def chap():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap as c
    c.load()
    return c


def check_cutoff(info, xb, cut):
    assert info.solutions == cut["count"]
    assert info.best_iter == (cut["best_iter"] if cut["count"] else -1)
    if cut["count"]:
        assert info.best_objective == cut["obj"] and info.rhs == cut["rhs"]
        assert np.array_equal(xb, cut["x_best"])


@pytest.mark.gpu
def test_cutoff_setcover_steps_bit_exact(chap):
    prob = inst.with_objective_row(inst.gen_setcover(seed=0, n=2000, m=1000, k=8))
    bs = chap.BestShift(prob, tenure=10)
    bs.set_cutoff(prob.m - 1, 1.0)
    orc = Oracle(prob)
    ost = orc.initial_state()
    cut = dict(row=prob.m - 1, delta=1.0)
    for k in range(3000):
        mv = bs.step()
        tr = orc.run_cutoff(ost, 10, 1, cut)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
        if mv.var >= 0:
            assert mv.new_value == tr["val"][0]
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    assert (st["iter"], st["nviol"], st["best_nviol"]) == (ost["iter"], orc.residuals(ost["x"])[2], ost["best_nviol"])
    assert cut["count"] >= 10
    info, xb = bs.cutoff()
    check_cutoff(info, xb, cut)
    assert np.array_equal(bs.residuals(), orc.residuals(ost["x"])[0])


@pytest.mark.gpu
def test_cutoff_graph_run_matches_oracle(chap):
    prob = inst.with_objective_row(inst.gen_setcover(seed=3, n=3000, m=1500, k=8))
    bs = chap.BestShift(prob, tenure=12, graph_iters=64)
    bs.set_cutoff(prob.m - 1, 2.0)
    res = bs.run(max_iters=2500, stop_at_feasible=1)     # never stops at a solution under the cutoff
    orc = Oracle(prob)
    ost = orc.initial_state()
    cut = dict(row=prob.m - 1, delta=2.0)
    orc.run_cutoff(ost, 12, 2500, cut)
    st = bs.state()
    assert res.iters == 2500 == st["iter"]
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    assert cut["count"] >= 2
    info, xb = bs.cutoff()
    check_cutoff(info, xb, cut)


@pytest.mark.gpu
def test_cutoff_feasible_start_recorded_by_weight_update(chap):
    # a feasible start: the first iteration has no positive move, updates no
    # weight and records the start as a solution (the copy is taken by the
    # weight-update kernel)
    base = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    prob = inst.with_objective_row(base)
    x = np.ones(base.n)
    assert feasible(base, x)
    bs = chap.BestShift(prob, tenure=10)
    bs.set_state(x)
    bs.set_cutoff(prob.m - 1, 5.0)
    mv = bs.step()
    assert mv.var == -1
    orc = Oracle(prob)
    ost = orc.initial_state(x)
    cut = dict(row=prob.m - 1, delta=5.0)
    orc.run_cutoff(ost, 10, 200, cut)
    assert cut["best_iter"] >= 1
    info, xb = bs.cutoff()
    assert info.solutions == 1 and info.best_iter == 1 and info.best_objective == float(base.obj.sum())
    assert np.array_equal(xb, x) and info.rhs == base.obj.sum() - 5.0
    for _ in range(199):
        bs.step()
    info, xb = bs.cutoff()
    check_cutoff(info, xb, cut)
    assert np.array_equal(bs.state()["x"], ost["x"])


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(16))
def test_cutoff_tiny_dyadic_mixed_exact(chap, seed):
    base = inst.gen_tiny_mixed(200 + seed, n=12, m=8, max_len=5, dom=10, cont_frac=0.25, dyadic=True, eq_frac=0.2)
    prob = inst.with_objective_row(base)
    bs = chap.BestShift(prob, tenure=3, feas_tol=0.0)
    bs.set_state(prob.x0)
    bs.set_cutoff(prob.m - 1, 0.5 if (base.vtype == inst.VAR_CONT).any() else 1.0)
    orc = Oracle(prob, feas_tol=0.0)
    ost = orc.initial_state(prob.x0)
    cut = dict(row=prob.m - 1, delta=0.5 if (base.vtype == inst.VAR_CONT).any() else 1.0)
    for k in range(250):
        mv = bs.step()
        tr = orc.run_cutoff(ost, 3, 1, cut)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
        if mv.var >= 0:
            assert mv.new_value == tr["val"][0]
        # exact while every value is dyadic: a continuous breakpoint such as
        # 25/12 makes the incremental residuals (device) and the recomputed
        # ones (oracle) round differently from here on (feas_tol = 0)
        if not np.array_equal(ost["x"] * 1024.0, np.round(ost["x"] * 1024.0)):
            break
        info, xb = bs.cutoff()
        check_cutoff(info, xb, cut)


@pytest.mark.gpu
def test_cutoff_arguments(chap):
    base = inst.gen_tiny_mixed(3, n=8, m=5, max_len=4, dom=6, dyadic=False)
    prob = inst.with_objective_row(base)
    bs = chap.BestShift(prob, tenure=3)
    ge = [i for i in range(base.m) if base.sense[i] != inst.ROW_LE]
    for row, delta in ((prob.m, 1.0), (-2, 1.0), (prob.m - 1, 0.0), (prob.m - 1, 0.5), (prob.m - 1, float("nan"))):
        with pytest.raises(chap.ChapError) as e:
            bs.set_cutoff(row, delta)
        assert e.value.status == chap.CHAP_E_INVALID
    if ge:
        with pytest.raises(chap.ChapError):
            bs.set_cutoff(ge[0], 1.0)
    bs.set_cutoff(prob.m - 1, 2.0)
    info, _ = bs.cutoff()
    assert info.row == prob.m - 1 and info.solutions == 0 and info.best_iter == -1 and np.isnan(info.best_objective)
    bs.set_cutoff(-1)
    info, _ = bs.cutoff()
    assert info.row == -1


def _golden_problem():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cutoff_example.json")))
    pr = g["problem"]
    rows, cols, vals = [], [], []
    for i, r in enumerate(pr["rows"]):
        for j, a in r["coefs"]:
            rows.append(i); cols.append(j); vals.append(float(a))
    prob = inst.from_triplets("cutoff_golden", pr["n"], len(pr["rows"]), rows, cols, vals, np.array(pr["lb"], float),
                              np.array(pr["ub"], float), np.array(pr["obj"], float),
                              np.array([r["rhs"] for r in pr["rows"]], float), np.array(pr["vtype"], np.uint8),
                              np.array([r["sense"] for r in pr["rows"]], np.uint8), x0=np.array(pr["x0"], float))
    return g, pr, prob


def test_oracle_cutoff_hand_derived_example():
    """The oracle's cutoff run against a trajectory worked out by hand
    (tests/golden/cutoff_example.json)."""
    g, pr, prob = _golden_problem()
    orc = Oracle(prob)
    st = orc.initial_state()
    cut = dict(row=pr["cutoff_row"], delta=float(pr["delta"]))
    tr = orc.run_cutoff(st, pr["tenure"], len(g["steps"]), cut)
    assert tr["var"].tolist() == [s["var"] for s in g["steps"]]
    assert tr["s_half"].tolist() == [s["s_half"] for s in g["steps"]]
    assert tr["nviol_after"].tolist() == g["nviol_after"]
    assert (cut["count"], cut["best_iter"], cut["obj"], cut["rhs"]) == \
        (g["solutions"], g["best_iter"], g["best_objective"], g["rhs_after"])
    assert cut["x_best"].tolist() == g["x_best"]
    assert st["w"].tolist() == g["w_after"]


@pytest.mark.gpu
def test_cutoff_hand_derived_example_on_gpu(chap):
    g, pr, prob = _golden_problem()
    bs = chap.BestShift(prob, tenure=pr["tenure"])
    bs.set_cutoff(pr["cutoff_row"], float(pr["delta"]))
    got = [(mv.var, mv.score_half) for mv in (bs.step() for _ in g["steps"])]
    assert got == [(s["var"], s["s_half"]) for s in g["steps"]]
    info, xb = bs.cutoff()
    assert (info.solutions, info.best_iter, info.best_objective, info.rhs) == \
        (g["solutions"], g["best_iter"], g["best_objective"], g["rhs_after"])
    assert xb.tolist() == g["x_best"] and bs.state()["w"].tolist() == g["w_after"]
