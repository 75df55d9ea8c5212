"""Parity of the CUDA best-shift path (through the C ABI) with the CPU oracle.

Bar: bit-exact results on integral instances (same per-variable best shift,
score and violation change; same selected move with ties broken by the lowest
variable and the smallest |delta|; same trajectory), and on non-integral rows
scores equal and shift values within 1e-9 relative (scores are integer
half-weight counts, so "within 1e-9 relative" means equal).
"""
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


def oracle_pass(orc, st, vars=None):
    return orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"],
                          st["best_nviol"], vars=vars)


def assert_exact(g, o, vars=None):
    gx, gs, gd = g
    if vars is not None:
        gx, gs, gd = gx[vars], gs[vars], gd[vars]
    ox, os_, od = o
    bad = np.nonzero((gx != ox) | (gs != os_) | (gd != od))[0]
    assert len(bad) == 0, [(int(k), gx[k], ox[k], int(gs[k]), int(os_[k]), int(gd[k]), int(od[k])) for k in bad[:10]]


def fp_mismatches(g, o, vars=None):
    gx, gs, gd = g
    if vars is not None:
        gx, gs, gd = gx[vars], gs[vars], gd[vars]
    ox, os_, od = o
    xok = np.abs(gx - ox) <= REL * np.maximum(1.0, np.abs(ox))
    sok = np.abs(gs - os_) <= REL * np.maximum(1.0, np.abs(os_))
    return np.nonzero(~(xok & sok & (gd == od)))[0]


def state_matches_oracle(st, orc):
    _, viol, nv = orc.residuals(st["x"])
    assert st["nviol"] == nv


# ------------------------------------------------------------------ config-1 set cover


def test_setcover_first_pass_exact(chap):
    prob = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    bs = chap.BestShift(prob, tenure=10)
    orc = Oracle(prob)
    st = bs.state()
    state_matches_oracle(st, orc)
    xh, sh, dc, mv = bs.best_shift()
    o = oracle_pass(orc, st)
    assert_exact((xh, sh, dc), o)
    j = int(np.argmax(o[1]))
    assert mv.var == (j if o[1][j] > 0 else -1)
    assert mv.score_half == o[1][j]


def test_setcover_1000_iterations_bit_exact(chap):
    prob = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    bs = chap.BestShift(prob, tenure=10)
    orc = Oracle(prob)
    ost = orc.initial_state()
    for k in range(1000):
        mv = bs.step()
        tr = orc.run(ost, tenure=10, n_iters=1, stop_at_feasible=False)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
        if mv.var >= 0:
            assert mv.new_value == tr["val"][0]
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    assert np.array_equal(st["tabu_inc"], ost["tabu_inc"]) and np.array_equal(st["tabu_dec"], ost["tabu_dec"])
    assert st["iter"] == ost["iter"] == 1000 and st["best_nviol"] == ost["best_nviol"]
    assert np.array_equal(bs.residuals(), orc.residuals(ost["x"])[0])


def test_setcover_graph_run_matches_oracle(chap):
    prob = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    orc = Oracle(prob)
    for stop in (0, 1):
        bs = chap.BestShift(prob, tenure=10, graph_iters=64)
        res = bs.run(max_iters=1000, stop_at_feasible=stop)
        ost = orc.initial_state()
        tr = orc.run(ost, tenure=10, n_iters=1000, stop_at_feasible=bool(stop))
        st = bs.state()
        assert res.iters == len(tr["var"]) == st["iter"]
        assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
        feas = np.nonzero(tr["nviol_after"] == 0)[0]
        assert res.feasible_iter == (int(feas[0]) + 1 if len(feas) else -1)
        if res.feasible_iter >= 0:
            assert res.time_to_feasible_s > 0 and res.final_nviol == 0 or not stop


def test_checkpoint_resume_bit_exact(chap):
    prob = inst.gen_setcover(seed=2, n=1500, m=900, k=8)
    a = chap.BestShift(prob, tenure=7)
    a.run(max_iters=600, stop_at_feasible=0)
    full = a.state()
    b = chap.BestShift(prob, tenure=7)
    b.run(max_iters=300, stop_at_feasible=0)
    ck = b.state()
    c = chap.BestShift(prob, tenure=7)
    c.set_checkpoint(ck)
    c.run(max_iters=300, stop_at_feasible=0)
    st = c.state()
    for k in ("x", "w", "tabu_inc", "tabu_dec"):
        assert np.array_equal(st[k], full[k]), k
    assert (st["iter"], st["nviol"], st["best_nviol"]) == (full["iter"], full["nviol"], full["best_nviol"])


# ------------------------------------------------------------------ tiny mixed instances


def _random_state(prob, orc, rng):
    x = prob.x0.copy()
    for j in range(prob.n):
        if prob.vtype[j] != inst.VAR_CONT:
            x[j] = rng.integers(int(prob.lb[j]), int(prob.ub[j]) + 1)
    w = rng.integers(1, 5, size=orc.mn).astype(np.int32)
    it = int(rng.integers(0, 6))
    ti = rng.integers(0, it + 4, size=prob.n)
    td = rng.integers(0, it + 4, size=prob.n)
    _, _, nv = orc.residuals(x)
    return dict(x=x, w=w, tabu_inc=ti, tabu_dec=td, iter=it, best_nviol=max(0, nv - int(rng.integers(0, 2))))


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("dyadic", [False, True])
def test_tiny_state_fed_exact(chap, seed, dyadic):
    prob = inst.gen_tiny_mixed(seed, n=10, m=8, max_len=6, dom=15, cont_frac=0.25 if dyadic else 0.0,
                               dyadic=dyadic, eq_frac=0.3)
    tol = 0.0 if dyadic else 1e-9
    orc = Oracle(prob, feas_tol=tol)
    bs = chap.BestShift(prob, tenure=3, feas_tol=tol)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        ck = _random_state(prob, orc, rng)
        bs.set_checkpoint(ck)
        st = bs.state()
        state_matches_oracle(st, orc)
        g = bs.best_shift()[:3]
        assert_exact(g, oracle_pass(orc, st))
        assert np.array_equal(bs.residuals(), orc.residuals(st["x"])[0])


@pytest.mark.parametrize("seed", range(12))
def test_tiny_integer_trajectory_exact(chap, seed):
    prob = inst.gen_tiny_mixed(100 + seed, n=14, m=12, max_len=6, dom=20, cont_frac=0.0, dyadic=False, eq_frac=0.3)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=4)
    bs.set_state(prob.x0)
    ost = orc.initial_state(prob.x0)
    for k in range(150):
        mv = bs.step()
        tr = orc.run(ost, tenure=4, n_iters=1, stop_at_feasible=False)
        assert (mv.var, mv.score_half) == (int(tr["var"][0]), int(tr["s_half"][0])), k
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])


def test_apply_host_moves_and_weight_updates(chap):
    prob = inst.gen_tiny_mixed(7, n=12, m=10, max_len=5, dom=10, dyadic=False)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=2)
    bs.set_state(prob.x0)
    rng = np.random.default_rng(0)
    x = prob.x0.copy()
    for k in range(40):
        j = int(rng.integers(-1, prob.n))
        if j >= 0:
            if prob.lb[j] == prob.ub[j]:
                continue
            v = float(rng.integers(int(prob.lb[j]), int(prob.ub[j]) + 1))
            if v == x[j]:
                continue
            x[j] = v
        bs.apply(j, x[j] if j >= 0 else 0.0)
        st = bs.state()
        assert np.array_equal(st["x"], x)
        assert np.array_equal(bs.residuals(), orc.residuals(x)[0])
        state_matches_oracle(st, orc)


# ------------------------------------------------------------------ larger workloads


@pytest.fixture(scope="module")
def general_small():
    return inst.gen_general(seed=1, n=20_000, m=10_000, len_cap=500)


def test_general_small_state_fed(chap, general_small):
    prob = general_small
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=10)
    rng = np.random.default_rng(5)
    vars_ = np.sort(rng.choice(prob.n, size=3000, replace=False)).astype(np.int32)
    for it in range(3):
        # state-fed: the residuals of the reached state recomputed on the device
        bs.set_checkpoint(bs.state())
        st = bs.state()
        state_matches_oracle(st, orc)
        g = bs.best_shift()[:3]
        o = oracle_pass(orc, st, vars=vars_)
        bad = fp_mismatches(g, o, vars_)
        assert len(bad) == 0, [(int(vars_[k]), g[0][vars_[k]], o[0][k], int(g[1][vars_[k]]), int(o[1][k]))
                               for k in bad[:8]]
        bs.run(max_iters=200, stop_at_feasible=0)
        # drift of the incremental FP64 residuals against the recomputed ones
        r_def, _, _ = orc.residuals(bs.state()["x"])
        _, _, rhs_n, _ = orc.norm_rows()
        assert np.all(np.abs(bs.residuals() - r_def) <= 1e-9 * np.maximum(1.0, np.abs(rhs_n)))


def test_general_small_trajectory_tracks_oracle(chap, general_small):
    """FP rows make long trajectories legitimately diverge; the first 100 moves agree."""
    prob = general_small
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=10)
    ost = orc.initial_state()
    agree = 0
    for k in range(100):
        mv = bs.step()
        tr = orc.run(ost, tenure=10, n_iters=1, stop_at_feasible=False)
        if mv.var != int(tr["var"][0]):
            break
        if mv.var >= 0:
            assert abs(mv.new_value - tr["val"][0]) <= REL * max(1.0, abs(tr["val"][0]))
            ost["x"][mv.var] = mv.new_value
        agree += 1
    assert agree == 100, agree


def test_skewed_sampled_exact(chap):
    prob = inst.gen_skewed(seed=3, n=200_000, m=100_000, n_dense=4, dense_len=20_000)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=10)
    assert bs.info.n_hist_cols == 4
    dense = np.array(prob.meta["dense_cols"], dtype=np.int32)
    rng = np.random.default_rng(9)
    vars_ = np.unique(np.concatenate([dense, rng.choice(prob.n, 4000, replace=False)])).astype(np.int32)
    for it in range(2):
        st = bs.state()
        state_matches_oracle(st, orc)
        g = bs.best_shift()[:3]
        assert_exact(g, oracle_pass(orc, st, vars=vars_), vars_)
        bs.run(max_iters=100, stop_at_feasible=0)


def test_long_continuous_column_cta_path(chap):
    """A continuous column with > 256 breakpoint entries takes the shared-memory CTA sort."""
    rng = np.random.default_rng(4)
    n, m = 50, 400
    rows, cols, vals = [], [], []
    for i in range(m):
        js = rng.choice(np.arange(1, n), size=3, replace=False)
        for j in [0, *js]:
            rows.append(i); cols.append(int(j)); vals.append(float(rng.choice([-2, -1, -0.5, 0.5, 1, 2])))
    vt = np.full(n, inst.VAR_INT); vt[0] = inst.VAR_CONT
    lb = np.zeros(n); ub = np.full(n, 8.0)
    x0 = np.floor(rng.random(n) * 9); x0[0] = 2.25
    sense = rng.choice([0, 1, 2], size=m, p=[0.4, 0.4, 0.2])
    ax = np.zeros(m)
    for r, c, v in zip(rows, cols, vals):
        ax[r] += v * x0[c]
    rhs = ax + rng.integers(-2, 3, size=m)
    prob = inst.from_triplets("longcol", n, m, rows, cols, vals, lb, ub, np.ones(n), rhs, vt, sense, x0=x0)
    orc = Oracle(prob, feas_tol=0.0)
    bs = chap.BestShift(prob, tenure=3, feas_tol=0.0)
    bs.set_state(x0)
    st = bs.state()
    assert_exact(bs.best_shift()[:3], oracle_pass(orc, st))


def _breakpoint_columns(seed, lengths, dom=200, eq_frac=0.2):
    """Integer columns j with lengths[j] single-variable rows each, whose
    breakpoints lie inside [0, dom]: every row contributes an entry to the
    column's list, so the lists have about lengths[j] entries (short lists,
    8/16/32-entry group sorts, lists longer than a group holds)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs, sense = [], [], [], [], []
    i = 0
    for j, L in enumerate(lengths):
        for _ in range(L):
            a = int(rng.choice([1, 2, 3, -1, -2]))
            t = int(rng.integers(0, dom + 1))
            s = int(rng.choice([0, 1, 2], p=[(1 - eq_frac) / 2, (1 - eq_frac) / 2, eq_frac]))
            rows.append(i); cols.append(j); vals.append(float(a))
            rhs.append(float(a * t + int(rng.integers(-1, 2))))
            sense.append(s)
            i += 1
    n, m = len(lengths), i
    vt = np.full(n, inst.VAR_INT)
    return inst.from_triplets(f"bp_columns_{seed}", n, m, rows, cols, vals, np.zeros(n), np.full(n, float(dom)),
                              np.ones(n), np.array(rhs), vt, np.array(sense, dtype=np.uint8), x0=np.zeros(n))


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("lengths,lanes", [([3, 7, 12, 20, 30, 45, 60, 100, 5], 8),
                                           ([1, 2, 3, 5, 7, 9, 12, 15, 18, 25, 4, 2, 3, 6, 11], 4)])
def test_list_lengths_group_and_warp_paths(chap, seed, lengths, lanes):
    """Columns whose lists take every sort of the short-column kernel (G, 2 G
    and 4 G entries per group of G lanes, the whole-warp path for lists longer
    than a group holds) and the counting sort, plus a partial last group of
    columns; G = 8 for long columns on average, 4 for short ones."""
    prob = _breakpoint_columns(seed, lengths)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=3)
    assert bs.info.nb_lanes == lanes
    for it in range(4):
        st = bs.state()
        assert_exact(bs.best_shift()[:3], oracle_pass(orc, st))
        bs.run(max_iters=7, stop_at_feasible=0)


def test_kernel_timing_api(chap, general_small):
    bs = chap.BestShift(general_small, tenure=10)
    with pytest.raises(chap.ChapError):
        chap.chap_bs_kernel_ms(bs.h)
    chap.chap_bs_profile(bs.h, True)
    bs.best_shift()
    ms = chap.chap_bs_kernel_ms(bs.h)
    info = bs.info
    assert ms[0] > 0 and ms[1] > 0 and ms[4] > 0
    assert info.grid_bin > 0 and info.grid_nb > 0 and info.bytes_bin > 0 and info.bytes_nb > 0
    chap.chap_bs_profile(bs.h, False)
    bs.close()


@pytest.mark.parametrize("n,k,lanes", [(40_000, 4, 2), (3_000, 8, 4), (2_000, 40, 8)])
def test_binary_lanes_per_column(chap, n, k, lanes):
    """The binary kernel's lanes per column follow the mean column length; every
    width is exact against the oracle over a few iterations."""
    prob = inst.gen_setcover(seed=n + k, n=n, m=n // 2, k=k)
    bs = chap.BestShift(prob, tenure=10)
    assert bs.info.bin_lanes == lanes
    orc = Oracle(prob)
    for _ in range(3):
        st = bs.state()
        assert_exact(bs.best_shift()[:3], oracle_pass(orc, st))
        bs.run(max_iters=5, stop_at_feasible=0)
    bs.close()


@pytest.mark.parametrize("which", ["general", "skewed"])
def test_pass_without_outputs_selects_the_full_pass_move(chap, general_small, which):
    """A pass that returns only the move skips the list sort of short columns
    whose score bound cannot reach an admissible score already found; the move
    must be the one of the full pass (which returns every variable's result)."""
    prob = general_small if which == "general" else \
        inst.gen_skewed(seed=7, n=100_000, m=50_000, n_dense=2, dense_len=5_000)
    bs = chap.BestShift(prob, tenure=10)
    for it in range(12):
        full = bs.best_shift()[3]
        _, _, _, quick = chap.chap_bs_best_shift(bs.h, want_vars=False)
        assert (quick.var, quick.score_half, quick.dnviol, quick.new_value) == \
            (full.var, full.score_half, full.dnviol, full.new_value), it
        bs.run(max_iters=25, stop_at_feasible=0)
    bs.close()


def _continuous_columns(seed, lengths, dom=64, eq_frac=0.2):
    """Continuous columns j with lengths[j] single-variable rows each (dyadic
    coefficients, breakpoints inside [0, dom]): a delta and a tight-point marker
    per half, so lists of up to about 2 * lengths[j] entries."""
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs, sense = [], [], [], [], []
    i = 0
    for j, L in enumerate(lengths):
        for _ in range(L):
            a = float(rng.choice([1, 2, 0.5, -1, -2, -0.5]))
            t = float(rng.integers(0, 4 * dom + 1)) / 4
            rows.append(i); cols.append(j); vals.append(a)
            rhs.append(a * t + float(rng.integers(-1, 2)) * 0.25)
            sense.append(int(rng.choice([0, 1, 2], p=[(1 - eq_frac) / 2, (1 - eq_frac) / 2, eq_frac])))
            i += 1
    n, m = len(lengths), i
    return inst.from_triplets(f"cont_columns_{seed}", n, m, rows, cols, vals, np.zeros(n), np.full(n, float(dom)),
                              np.ones(n), np.array(rhs), np.full(n, inst.VAR_CONT), np.array(sense, dtype=np.uint8),
                              x0=np.zeros(n))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_continuous_lists_whole_warp(chap, seed):
    """Continuous columns whose lists pass 128 entries (up to 256) stay on the
    short-column kernel: groups, then the whole-warp path over the warp's
    stage and queue memory (8 entries per lane); bit-exact on dyadic data."""
    lengths = [3, 20, 50, 70, 80, 90, 95, 40, 8, 64, 75]
    prob = _continuous_columns(seed, lengths, eq_frac=0.1)
    orc = Oracle(prob, feas_tol=0.0)
    bs = chap.BestShift(prob, tenure=3, feas_tol=0.0)
    assert bs.info.n_cta_cols == 0 and bs.info.n_long_cols == 0
    for it in range(4):
        st = bs.state()
        assert_exact(bs.best_shift()[:3], oracle_pass(orc, st))
        bs.run(max_iters=5, stop_at_feasible=0)


@pytest.mark.parametrize("which", ["setcover", "general"])
def test_run_objective_reduced_on_device(chap, which):
    """chap_tabu_run reports c^T x of the state it leaves, reduced on the device:
    exact on integer data, within the summation-order rounding otherwise."""
    prob = (inst.gen_setcover(seed=2, n=3000, m=1500, k=8) if which == "setcover"
            else inst.gen_general(seed=2, n=5000, m=2500, len_cap=60))
    bs = chap.BestShift(prob, tenure=5)
    for _ in range(3):
        r = bs.run(max_iters=40, stop_at_feasible=0)
        x = bs.state()["x"]
        want = float(np.dot(prob.obj, x))
        if which == "setcover":
            assert r.objective == want
        else:
            assert abs(r.objective - want) <= 1e-12 * max(1.0, float(np.abs(prob.obj) @ np.abs(x)))
    bs.close()
