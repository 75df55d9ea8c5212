"""Column-sharded pass: K handles, each evaluating every K-th column of each
class, exchange their 32-byte move records and all apply the winner.  On one
GPU the K ranks are emulated in one process (no kernel waits on another: the
passes run one after the other and the records are concatenated in rank
order), and the sharded search must take the same moves as one handle over
the whole instance, and as the oracle."""
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


def _sharded_steps(chap, prob, world, iters, **opts):
    import torch
    shards = [chap.ShardedSearch(prob, r, world, **opts) for r in range(world)]
    moves = []
    for _ in range(iters):
        recs = torch.cat([s.pass_record().clone() for s in shards])
        for s in shards:
            s.apply(recs)
        moves.append(recs)
    return shards, moves


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("which", ["setcover", "tiny_int", "general_small", "skewed_small"])
def test_sharded_equals_whole_instance(chap, world, which):
    if which == "setcover":
        prob, iters = inst.gen_setcover(seed=0, n=2000, m=1000, k=8), 200
    elif which == "tiny_int":
        prob, iters = inst.gen_tiny_mixed(7, n=14, m=12, max_len=6, dom=20, cont_frac=0.0, dyadic=False,
                                          eq_frac=0.3), 200
    elif which == "general_small":
        prob, iters = inst.gen_general(seed=1, n=20_000, m=10_000, len_cap=500), 60
    else:
        prob, iters = inst.gen_skewed(seed=3, n=100_000, m=50_000, n_dense=3, dense_len=10_000), 40
    whole = chap.BestShift(prob, tenure=5)
    shards, _ = _sharded_steps(chap, prob, world, 0, tenure=5)
    for k in range(iters):
        import torch
        recs = torch.cat([s.pass_record().clone() for s in shards])
        for s in shards:
            s.apply(recs)
        mv = whole.step()
        st = shards[0].bs.state()
        wst = whole.state()
        assert st["iter"] == wst["iter"] == k + 1
        assert np.array_equal(st["x"], wst["x"]), k
        assert st["nviol"] == wst["nviol"] and np.array_equal(st["w"], wst["w"]), k
    for s in shards[1:]:
        o = s.bs.state()
        assert np.array_equal(o["x"], st["x"]) and np.array_equal(o["w"], st["w"])
        assert np.array_equal(o["tabu_inc"], st["tabu_inc"]) and np.array_equal(o["tabu_dec"], st["tabu_dec"])
    for s in shards:
        s.close()
    whole.close()


def test_sharded_trajectory_equals_oracle(chap):
    prob = inst.gen_setcover(seed=2, n=1500, m=700, k=8)
    shards, _ = _sharded_steps(chap, prob, 2, 200, tenure=10)
    orc = Oracle(prob)
    ost = orc.initial_state()
    orc.run(ost, tenure=10, n_iters=200, stop_at_feasible=False)
    st = shards[0].bs.state()
    assert np.array_equal(st["x"], ost["x"]) and np.array_equal(st["w"], ost["w"])
    for s in shards:
        s.close()


def test_shard_pass_covers_its_columns(chap):
    """Each shard scores its own columns exactly as the whole-instance pass
    does and leaves the others at (x, 0, 0); together the shards cover every
    column once."""
    prob = inst.gen_general(seed=4, n=6_000, m=3_000, len_cap=300)
    whole = chap.BestShift(prob, tenure=5)
    g = whole.best_shift()
    seen = np.zeros(prob.n, dtype=int)
    for r in range(3):
        bs = chap.BestShift(prob, tenure=5, shard_rank=r, shard_count=3)
        x, s, d, mv = bs.best_shift()
        own = s != 0
        assert np.array_equal(s[own], g[1][own]) and np.array_equal(x[own], g[0][own])
        assert np.array_equal(d[own], g[2][own])
        seen += own
        st = bs.state()
        assert np.all(x[~own] == st["x"][~own])
        bs.close()
    # every variable with a positive score in the whole pass is scored by one shard
    assert np.array_equal(seen > 0, g[1] != 0) and seen.max() <= 1
    whole.close()


def test_sharded_handle_refuses_whole_instance_calls(chap):
    prob = inst.gen_setcover(seed=0, n=500, m=250, k=8)
    bs = chap.BestShift(prob, tenure=5, shard_rank=0, shard_count=2)
    for call in (lambda: bs.step(), lambda: bs.run(max_iters=3)):
        with pytest.raises(chap.ChapError) as ei:
            call()
        assert ei.value.status == chap.CHAP_E_STATE
    bad = (chap.chap_move_record * 1)()
    bad[0].score_half, bad[0].var, bad[0].new_value = 5, prob.n + 3, 1.0
    with pytest.raises(chap.ChapError) as ei:
        chap.chap_bs_apply_records(bs.h, bad)
    assert ei.value.status == chap.CHAP_E_INVALID
    # host records: a valid flip is applied as given
    ok = (chap.chap_move_record * 2)()
    ok[0].score_half, ok[0].var, ok[0].new_value = 3, 7, 1.0
    ok[1].score_half, ok[1].var, ok[1].new_value = 3, 4, 1.0
    chap.chap_bs_apply_records(bs.h, ok)
    st = bs.state()
    assert st["x"][4] == 1.0 and st["x"][7] == 0.0 and st["iter"] == 1
    bs.close()
