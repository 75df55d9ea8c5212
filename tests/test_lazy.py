"""Selective re-evaluation of the binary flip scores (chap_options.lazy_binary).

The kept scores are recomputed only for the binary variables of rows whose
residual changed; tabu and aspiration are applied to them at every iteration.
Every result must equal the full pass: the move sequence against the CPU oracle
(integral instances, bit-exact) and against a handle without the option (mixed
instances: same moves, same per-variable outputs), through single steps, host
moves, checkpoints, graph runs split over several calls and the objective
cutoff.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
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


def same_outputs(a, b):
    ga, gb = a.best_shift(), b.best_shift()
    for k in range(3):
        assert np.array_equal(ga[k], gb[k]), k
    assert (ga[3].var, ga[3].score_half, ga[3].new_value) == (gb[3].var, gb[3].score_half, gb[3].new_value)


def same_state(a, b):
    sa, sb = a.state(), b.state()
    for k in ("x", "w", "tabu_inc", "tabu_dec"):
        assert np.array_equal(sa[k], sb[k]), k
    assert (sa["iter"], sa["nviol"], sa["best_nviol"]) == (sb["iter"], sb["nviol"], sb["best_nviol"])


def test_lazy_setcover_steps_bit_exact(chap):
    prob = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    bs = chap.BestShift(prob, tenure=10, lazy_binary=1)
    assert bs.info.launches_per_step == chap.BestShift(prob, tenure=10).info.launches_per_step + 2
    orc = Oracle(prob)
    ost = orc.initial_state()
    bumps = 0
    for k in range(1000):
        mv = bs.step()
        tr = orc.run(ost, tenure=10, n_iters=1, stop_at_feasible=False)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
        bumps += mv.var < 0
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    assert bumps > 0


@pytest.mark.parametrize("seed", range(8))
def test_lazy_tiny_integer_trajectory_exact(chap, seed):
    prob = inst.gen_tiny_mixed(100 + seed, n=14, m=12, max_len=6, dom=20, cont_frac=0.0, dyadic=False, eq_frac=0.3)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=4, lazy_binary=1)
    bs.set_state(prob.x0)
    ost = orc.initial_state(prob.x0)
    for k in range(150):
        mv = bs.step()
        tr = orc.run(ost, tenure=4, n_iters=1, stop_at_feasible=False)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k


def test_lazy_general_small_equals_full(chap):
    prob = inst.gen_general(seed=1, n=20_000, m=10_000, len_cap=500)
    a = chap.BestShift(prob, tenure=10, lazy_binary=1)
    b = chap.BestShift(prob, tenure=10)
    same_outputs(a, b)
    for k in range(400):
        ma, mb = a.step(), b.step()
        assert (ma.var, ma.score_half, ma.new_value) == (mb.var, mb.score_half, mb.new_value), k
        if k in (0, 57, 399):
            same_outputs(a, b)
    same_state(a, b)


def test_lazy_host_moves_checkpoint_and_graph_runs(chap):
    prob = inst.gen_setcover(seed=4, n=20_000, m=10_000, k=8)
    a = chap.BestShift(prob, tenure=12, lazy_binary=1, graph_iters=64)
    b = chap.BestShift(prob, tenure=12, graph_iters=64)
    # two host moves before the next pass: both columns' rows must be marked
    for bs in (a, b):
        bs.apply(5, 1.0)
        bs.apply(17, 1.0)
    same_outputs(a, b)
    # a run split over calls: the last iteration of each call is marked too
    for n_it in (333, 1, 64, 500):
        ra, rb = a.run(max_iters=n_it, stop_at_feasible=0), b.run(max_iters=n_it, stop_at_feasible=0)
        assert (ra.iters, ra.moves) == (rb.iters, rb.moves)
        same_state(a, b)
        same_outputs(a, b)
    # a checkpoint replaces every kept score
    ck = b.state()
    rng = np.random.default_rng(0)
    ck["x"] = (rng.random(prob.n) < 0.3).astype(np.float64)
    ck["w"] = rng.integers(1, 4, size=b.m_norm).astype(np.int32)
    ck["best_nviol"] = 10 ** 6
    a.set_checkpoint(ck)
    b.set_checkpoint(ck)
    same_outputs(a, b)
    ra, rb = a.run(max_iters=700, stop_at_feasible=1), b.run(max_iters=700, stop_at_feasible=1)
    assert (ra.iters, ra.feasible_iter) == (rb.iters, rb.feasible_iter)
    same_state(a, b)


def test_lazy_with_objective_cutoff(chap):
    prob = inst.with_objective_row(inst.gen_setcover(seed=0, n=2000, m=1000, k=8))
    bs = chap.BestShift(prob, tenure=10, lazy_binary=1)
    bs.set_cutoff(prob.m - 1, 1.0)
    orc = Oracle(prob)
    ost = orc.initial_state()
    cut = dict(row=prob.m - 1, delta=1.0)
    for k in range(1500):
        mv = bs.step()
        tr = orc.run_cutoff(ost, 10, 1, cut)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
    info, xb = bs.cutoff()
    assert info.solutions == cut["count"] >= 2 and info.best_objective == cut["obj"]
    assert np.array_equal(xb, cut["x_best"])


def test_lazy_option_validated(chap):
    prob = inst.gen_setcover(seed=0, n=200, m=100, k=8)
    with pytest.raises(chap.ChapError) as e:
        chap.BestShift(prob, lazy_binary=2)
    assert e.value.status == chap.CHAP_E_INVALID
    # no binary column: the option has nothing to keep
    tiny = inst.gen_tiny_mixed(5, n=6, m=4, max_len=3, dom=5, dyadic=False)
    tiny.vtype[:] = inst.VAR_INT
    tiny.ub[:] = np.maximum(tiny.ub, tiny.lb + 2)
    a = chap.BestShift(tiny, tenure=3, lazy_binary=1)
    b = chap.BestShift(tiny, tenure=3)
    assert a.info.launches_per_step == b.info.launches_per_step
    same_outputs(a, b)


def test_lazy_under_the_learned_loop(chap):
    """The learned loop (proposals between exact passes) over a handle with kept
    binary scores takes the moves of the same loop without them: the marks of
    the proposal iterations accumulate until the next exact pass."""
    torch = pytest.importorskip("torch")
    from paper_2605_05086_gb300 import learn
    prob = inst.gen_setcover(seed=8, n=3000, m=1500, k=8)
    w = learn.to_bf16_bits(torch.tensor(learn.init_params(3), device="cuda"))
    a = chap.BestShift(prob, tenure=7, lazy_binary=1)
    b = chap.BestShift(prob, tenure=7)
    ra = chap.chap_learned_run(a.h, w, topk=128, exact_every=9, propose_every=2, max_iters=400, stop_at_feasible=False)
    rb = chap.chap_learned_run(b.h, w, topk=128, exact_every=9, propose_every=2, max_iters=400, stop_at_feasible=False)
    assert (ra.iters, ra.misses, ra.exact_passes) == (rb.iters, rb.misses, rb.exact_passes)
    same_state(a, b)
    same_outputs(a, b)
