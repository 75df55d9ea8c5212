"""Row-blocked binary flips (bin_kernel = 3: the rows cut into blocks whose
states a CTA holds in shared memory, the binary columns' entries of each block
scored against them, the blocks' partial sums met by device atomics and
finished per range of positions) against the oracle and against the
column-wise kernel (bin_kernel = 1): the same per-variable scores, violation
changes, moves and trajectories."""
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


def _same(a, b):
    for u, v in zip(a[:3], b[:3]):
        assert np.array_equal(u, v)
    assert (a[3].var, a[3].score_half, a[3].dnviol, a[3].new_value) == (b[3].var, b[3].score_half, b[3].dnviol,
                                                                         b[3].new_value)


def _binary_eq(seed, n=12_000, m=6_000):
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs = [], [], [], []
    sense = rng.choice([0, 1, 2], size=m, p=[0.4, 0.4, 0.2]).astype(np.uint8)
    xs = rng.integers(0, 2, size=n)
    for i in range(m):
        js = rng.choice(n, size=6, replace=False)
        a = rng.integers(1, 5, size=6) * np.where(rng.random(6) < 0.5, -1, 1)
        rows += [i] * 6; cols += list(js); vals += list(a.astype(float))
        rhs.append(float(a @ xs[js]) + (rng.integers(0, 3) if sense[i] == 0 else -rng.integers(0, 3) if sense[i] == 1 else 0))
    return inst.from_triplets("bineq", n, m, rows, cols, vals, np.zeros(n), np.ones(n), np.ones(n), np.array(rhs),
                              np.full(n, inst.VAR_BIN), sense, x0=np.zeros(n))


@pytest.mark.parametrize("block_rows", [128, 0])
def test_setcover_1000_iterations_bit_exact(chap, block_rows):
    """Set cover 2k: the first pass and 1,000 tabu iterations equal the
    oracle's, with 8 row blocks of 128 rows and with one block."""
    prob = inst.gen_setcover(seed=0, n=2000, m=1000, k=8)
    bs = chap.BestShift(prob, tenure=10, bin_kernel=3, bin_block_rows=block_rows)
    assert bs.info.bin_row_blocks == (8 if block_rows == 128 else 1)
    orc = Oracle(prob)
    ost = orc.initial_state()
    st = bs.state()
    g = bs.best_shift()
    o = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"], st["best_nviol"])
    assert all(np.array_equal(u, v) for u, v in zip(g[:3], o))
    orc.run(ost, tenure=10, n_iters=1000, stop_at_feasible=False)
    bs.run(max_iters=1000, stop_at_feasible=0)
    st = bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    bs.close()


@pytest.mark.parametrize("which,block_rows", [("setcover_20k", 1000), ("general_small", 0), ("general_small", 700),
                                              ("binary_eq", 333), ("skewed_small", 4096)])
def test_blocks_equal_columns(chap, which, block_rows):
    """Integral and N(0,1) rows, "=" rows, ragged last blocks: the row-blocked
    and column-wise kernels agree on every variable at several states, and
    their trajectories (graph runs, weight updates included) coincide."""
    if which == "setcover_20k":
        prob = inst.gen_setcover(seed=3, n=20_000, m=10_000, k=8)
    elif which == "general_small":
        prob = inst.gen_general(seed=1, n=20_000, m=10_000, len_cap=500)
    elif which == "binary_eq":
        prob = _binary_eq(5)
    else:
        prob = inst.gen_skewed(seed=3, n=100_000, m=50_000, n_dense=3, dense_len=10_000)
    a = chap.BestShift(prob, tenure=7, bin_kernel=1)
    b = chap.BestShift(prob, tenure=7, bin_kernel=3, bin_block_rows=block_rows)
    assert a.info.bin_row_blocks == 0
    assert b.info.bin_row_blocks == -(-prob.m // (block_rows or 8192))
    for _ in range(4):
        _same(a.best_shift(), b.best_shift())
        a.run(max_iters=25, stop_at_feasible=0)
        b.run(max_iters=25, stop_at_feasible=0)
        sa, sb = a.state(), b.state()
        assert np.array_equal(sa["x"], sb["x"]) and np.array_equal(sa["w"], sb["w"])
    a.close()
    b.close()


@pytest.mark.parametrize("seed", range(20))
def test_tiny_state_fed_exact(chap, seed):
    """Random states (weights, tabu stamps, best counts) of tiny mixed
    instances with "=" rows, rows cut into blocks of 2: the row-blocked binary
    scores equal the oracle's."""
    prob = inst.gen_tiny_mixed(seed, n=12, m=9, max_len=6, dom=10, cont_frac=0.0, dyadic=False, eq_frac=0.3)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=3, bin_kernel=3, bin_block_rows=2)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        x = prob.x0.copy()
        for j in range(prob.n):
            x[j] = float(rng.integers(int(prob.lb[j]), int(prob.ub[j]) + 1))
        _, _, nv = orc.residuals(x)
        st = dict(x=x, w=rng.integers(1, 5, size=orc.mn).astype(np.int32), tabu_inc=rng.integers(0, 6, size=prob.n),
                  tabu_dec=rng.integers(0, 6, size=prob.n), iter=3, best_nviol=max(0, nv - int(rng.integers(0, 2))))
        bs.set_checkpoint(st)
        s = bs.state()
        g = bs.best_shift()
        o = orc.best_shift(s["x"], s["w"], s["tabu_inc"], s["tabu_dec"], s["iter"], s["nviol"], s["best_nviol"])
        assert all(np.array_equal(u, v) for u, v in zip(g[:3], o))
    bs.close()


def test_host_moves_and_checkpoints(chap):
    """Moves applied from the host and states loaded mid-run keep the flip
    directions of the row-blocked store in step with x."""
    prob = inst.gen_general(seed=2, n=20_000, m=10_000, len_cap=300)
    a = chap.BestShift(prob, tenure=5, bin_kernel=1)
    b = chap.BestShift(prob, tenure=5, bin_kernel=3, bin_block_rows=2048)
    rng = np.random.default_rng(0)
    bins = np.flatnonzero(prob.vtype == inst.VAR_BIN)
    for k in range(6):
        j = int(rng.choice(bins))
        v = 1.0 - a.state()["x"][j]
        a.apply(j, v)
        b.apply(j, v)
        _same(a.best_shift(), b.best_shift())
    st = a.state()
    st["x"][bins[:500]] = 1.0 - st["x"][bins[:500]]
    a.set_checkpoint(st)
    b.set_checkpoint(st)
    _same(a.best_shift(), b.best_shift())
    a.run(max_iters=40, stop_at_feasible=0)
    b.run(max_iters=40, stop_at_feasible=0)
    assert np.array_equal(a.state()["x"], b.state()["x"])
    a.close()
    b.close()


def test_automatic_choice(chap):
    """With the default option the library takes the row-blocked flips on a
    general-family MIP with enough binary columns and few row blocks, and its
    results equal the column-wise kernel's."""
    prob = inst.gen_general(seed=6, n=40_000, m=20_000, len_cap=1000)
    a = chap.BestShift(prob, tenure=10, bin_kernel=1)
    b = chap.BestShift(prob, tenure=10)
    assert b.info.bin_row_blocks == 3
    for _ in range(3):
        _same(a.best_shift(), b.best_shift())
        a.run(max_iters=30, stop_at_feasible=0)
        b.run(max_iters=30, stop_at_feasible=0)
    assert np.array_equal(a.state()["x"], b.state()["x"])
    a.close()
    b.close()


def test_cutoff_row_blocked(chap):
    """The objective cutoff (its row's residual tightened on the device) under
    the row-blocked flips: the same trajectory and recorded solutions as the
    column-wise kernel."""
    prob = inst.with_objective_row(inst.gen_setcover(seed=7, n=4000, m=2000, k=8))
    a = chap.BestShift(prob, tenure=10, bin_kernel=1)
    b = chap.BestShift(prob, tenure=10, bin_kernel=3, bin_block_rows=256)
    for h in (a, b):
        h.set_cutoff(prob.meta["cutoff_row"], 1.0)
        h.run(max_iters=1500, stop_at_feasible=0)
    ca, cb = a.cutoff(), b.cutoff()
    assert ca[0].solutions == cb[0].solutions and ca[0].solutions > 0
    assert np.array_equal(ca[1], cb[1])
    assert np.array_equal(a.state()["x"], b.state()["x"])
    a.close()
    b.close()


def test_sharded_row_blocked(chap):
    """Two column shards, each scoring its binary columns row-blocked, take
    the whole-instance moves."""
    import torch
    prob = inst.gen_setcover(seed=4, n=40_000, m=20_000, k=8)
    whole = chap.BestShift(prob, tenure=5, bin_kernel=1)
    shards = [chap.ShardedSearch(prob, r, 2, tenure=5, bin_kernel=3, bin_block_rows=4096) for r in range(2)]
    assert all(s.bs.info.bin_row_blocks == 5 for s in shards)
    for k in range(30):
        recs = torch.cat([s.pass_record().clone() for s in shards])
        for s in shards:
            s.apply(recs)
        whole.step()
    st, wst = shards[0].bs.state(), whole.state()
    assert np.array_equal(st["x"], wst["x"]) and np.array_equal(st["w"], wst["w"])
    for s in shards:
        s.close()
    whole.close()


def test_block_rows_option_checked(chap):
    prob = inst.gen_setcover(seed=0, n=200, m=100, k=4)
    for bad in (-1, 8193):
        with pytest.raises(chap.ChapError):
            chap.BestShift(prob, bin_kernel=3, bin_block_rows=bad)
