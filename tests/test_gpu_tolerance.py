"""The CUDA path at a positive feasibility tolerance (feas_tol = 1e-9 on
non-integral rows), through the C ABI, against values that do not come from it:

- every hand-derived worked example (tests/golden/worked_examples.json), among
  them a row satisfied within eps whose breakpoint is no candidate, the same
  rows without a tolerance, and the continuous tie-break cases;
- two rows whose breakpoints coincide in exact arithmetic but round one ulp
  apart (3x >= 1 and 0.3x >= 0.1), where the row satisfied within eps at the
  other's point must count as satisfied there;
- random tiny N(0,1) instances in states with rows satisfied within eps but
  not exactly tight, against the oracle (scores and violation changes equal,
  shifts within 1e-9 relative).
"""
import numpy as np
import pytest

from conftest import fp_tiny, golden_cases, problem_from_case
from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst

pytestmark = pytest.mark.gpu
REL = 1e-9


@pytest.fixture(scope="module")
def chap():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap as c
    c.load()
    return c


def _close(a, b):
    return np.abs(a - b) <= REL * np.maximum(1.0, np.abs(b))


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_worked_examples_on_device(chap, case):
    prob = problem_from_case(case)
    tol = case.get("feas_tol", 1e-9)
    bs = chap.BestShift(prob, tenure=3, feas_tol=tol)
    st = dict(x=np.array(case["x"], float), w=np.array(case["w"], np.int32),
              tabu_inc=np.array(case["tabu_inc"], np.int64), tabu_dec=np.array(case["tabu_dec"], np.int64),
              iter=int(case["iter"]), best_nviol=int(case["best_nviol"]))
    bs.set_checkpoint(st)
    xh, sh, dc, _ = bs.best_shift()
    exp = np.array(case["expect"], float)
    assert np.all(_close(xh, exp[:, 0])), (xh, exp)
    assert sh.tolist() == exp[:, 1].astype(int).tolist()
    assert dc.tolist() == exp[:, 2].astype(int).tolist()
    bs.close()


def _compare(bs, orc, st):
    g = bs.best_shift()
    o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"])
    bad = np.nonzero(~(_close(g[0], o[0]) & (g[1] == o[1]) & (g[2] == o[2])))[0]
    assert len(bad) == 0, [(int(k), g[0][k], o[0][k], int(g[1][k]), int(o[1][k]), int(g[2][k]), int(o[2][k]))
                           for k in bad[:6]]
    return g


@pytest.mark.parametrize("xbar", [0.0, 0.25, 1.0])
def test_coincident_breakpoints_one_ulp_apart(chap, xbar):
    """3x >= 1 and 0.3x >= 0.1 become tight at 1/3 in exact arithmetic; their
    double breakpoints are 0.3333333333333333 and 0.33333333333333337.  At
    either point both rows are satisfied within eps, so both candidates score
    +4 (two rows from violated to satisfied) and the closer one wins; a third
    row x <= 0.5 is satisfied throughout."""
    rows = [0, 1, 2]
    cols = [0, 0, 0]
    vals = [3.0, 0.3, 1.0]
    prob = inst.from_triplets("ulp_apart", 1, 3, rows, cols, vals, [0.0], [10.0], [1.0], [1.0, 0.1, 0.5],
                              [inst.VAR_CONT], [inst.ROW_GE, inst.ROW_GE, inst.ROW_LE], x0=[xbar])
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=3)
    bs.set_state(np.array([xbar]))
    st = bs.state()
    g = _compare(bs, orc, st)
    if xbar < 1.0 / 3.0:
        assert int(g[1][0]) == 4 and abs(g[0][0] - 1.0 / 3.0) < 1e-15


@pytest.mark.parametrize("seed", range(120))
def test_rows_satisfied_within_eps(chap, seed):
    tol = 1e-9
    prob, x = fp_tiny(seed, tol)
    orc = Oracle(prob, feas_tol=tol)
    rng = np.random.default_rng(5000 + seed)
    bs = chap.BestShift(prob, tenure=3, feas_tol=tol)
    _, _, nv = orc.residuals(x)
    st = dict(x=x, w=rng.integers(1, 4, size=orc.mn).astype(np.int32),
              tabu_inc=rng.integers(0, 5, size=prob.n), tabu_dec=rng.integers(0, 5, size=prob.n), iter=2,
              best_nviol=max(0, nv - int(rng.integers(0, 2))))
    bs.set_checkpoint(st)
    s = bs.state()
    assert s["nviol"] == nv
    assert np.array_equal(bs.residuals(), orc.residuals(x)[0])
    _compare(bs, orc, s)
    bs.close()


def _tight_instance(seed, n=400, m=300):
    """Continuous and integer variables over N(0,1) rows where many rows hold
    with equality at the start point (rhs = a.x0 on every "=" row and a third
    of the others), so that a pass meets many rows with |r| <= eps: the
    short-column kernel's queue of undecided halves, and its list entries for
    tight rows, at a size that spans several CTAs."""
    rng = np.random.default_rng(seed)
    vt = np.where(rng.random(n) < 0.6, inst.VAR_CONT, inst.VAR_INT).astype(np.uint8)
    lb = np.zeros(n)
    ub = np.where(vt == inst.VAR_CONT, 10.0, 20.0)
    x0 = np.where(vt == inst.VAR_CONT, np.round(rng.random(n) * 10, 3), rng.integers(0, 21, size=n)).astype(float)
    rows, cols, vals = [], [], []
    for i in range(m):
        js = rng.choice(n, size=int(rng.integers(2, 9)), replace=False)
        for j in sorted(js.tolist()):
            rows.append(i); cols.append(j); vals.append(float(rng.normal()))
    ax = np.zeros(m)
    for r, c, v in zip(rows, cols, vals):
        ax[r] += v * x0[c]
    sense = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=m, p=[0.35, 0.35, 0.3])
    slack = np.where(rng.random(m) < 0.33, 0.0, rng.random(m) * 3 - 1.0)
    rhs = np.where(sense == 0, ax + slack, np.where(sense == 1, ax - slack, ax))
    return inst.from_triplets(f"tight_{seed}", n, m, rows, cols, vals, lb, ub, np.ones(n), rhs, vt, sense, x0=x0)


@pytest.mark.parametrize("seed", range(6))
def test_many_tight_rows_state_fed(chap, seed):
    prob = _tight_instance(seed)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=5)
    for _ in range(4):
        bs.set_checkpoint(bs.state())
        _compare(bs, orc, bs.state())
        bs.run(max_iters=10, stop_at_feasible=0)
    bs.close()
