"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (one handle, full passes), on sampled variables the oracle evaluates one
by one: the general 200k-var MIP (non-integral rows: scores and violation
changes equal, shifts within 1e-9 relative, state-fed after the run) and the
skewed 2M-var MIP (all rows integral: bit-exact, every dense column included)."""
import numpy as np
import pytest

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


def _sampled(chap, prob, vars_, states, exact):
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=10)
    bad_total = 0
    for it in states:
        if it:
            bs.run(max_iters=it, stop_at_feasible=0)
            if not exact:
                # state-fed: the device recomputes the residuals of the state it
                # reached (incremental FP64 residuals drift by rounding; the drift
                # is checked below), as the oracle does
                r_inc = bs.residuals()
                r_def, _, _ = orc.residuals(bs.state()["x"])
                b = np.abs(orc.norm_rows()[2])
                assert np.all(np.abs(r_inc - r_def) <= 1e-9 * np.maximum(1.0, b))
                bs.set_checkpoint(bs.state())
        st = bs.state()
        _, _, nv = orc.residuals(st["x"])
        assert nv == st["nviol"]
        gx, gs, gd = bs.best_shift()[:3]
        ox, os_, od = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"],
                                     st["best_nviol"], vars=vars_)
        gx, gs, gd = gx[vars_], gs[vars_], gd[vars_]
        if exact:
            bad = np.nonzero((gx != ox) | (gs != os_) | (gd != od))[0]
            assert len(bad) == 0, [(int(vars_[k]), gx[k], ox[k], int(gs[k]), int(os_[k])) for k in bad[:8]]
        else:
            ok = (np.abs(gx - ox) <= REL * np.maximum(1.0, np.abs(ox))) & (gs == os_) & (gd == od)
            bad_total += int(np.sum(~ok))
    bs.close()
    return bad_total


def test_general_200k_sampled(chap):
    prob = inst.make("general_200k")
    rng = np.random.default_rng(3)
    vt = prob.vtype
    vars_ = np.unique(np.concatenate([rng.choice(np.nonzero(vt == t)[0], 1500, replace=False) for t in (0, 1, 2)]))
    bad = _sampled(chap, prob, vars_.astype(np.int32), [0, 100], exact=False)
    assert bad == 0, bad


def test_skewed_2m_sampled(chap):
    prob = inst.make("skewed_2m")
    rng = np.random.default_rng(4)
    dense = np.array(prob.meta["dense_cols"], dtype=np.int64)
    vars_ = np.unique(np.concatenate([dense, rng.choice(prob.n, 4000, replace=False)])).astype(np.int32)
    _sampled(chap, prob, vars_, [0, 60], exact=True)
