"""Batched tabu chains (chap_batch_*) against the single-handle path and the
oracle: every chain must follow exactly the trajectory of chap_bs_step on its
instance with its tenure (same moves, weights, stopping iteration), under both
schedules (three launches per iteration, one persistent launch with grid
barriers).  A barrier whose wait bound is set to 1 ns runs out: the run
returns CHAP_E_TIMEOUT, nothing faults, and the batch works again after a
reset."""
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


def binary_mixed(seed, n, m, k=5):
    """All-binary integral instance with <=, >= and = rows (coefficients +-1..4)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals, rhs = [], [], [], []
    sense = rng.choice([inst.ROW_LE, inst.ROW_GE, inst.ROW_EQ], size=m, p=[0.4, 0.4, 0.2]).astype(np.uint8)
    xstar = rng.integers(0, 2, size=n)
    for i in range(m):
        js = rng.choice(n, size=k, replace=False)
        a = rng.integers(1, 5, size=k) * np.where(rng.random(k) < 0.5, -1, 1)
        rows += [i] * k; cols += list(js); vals += list(a.astype(float))
        act = float(a @ xstar[js])
        rhs.append(act + (rng.integers(0, 3) if sense[i] == inst.ROW_LE else -rng.integers(0, 3) if sense[i] == inst.ROW_GE else 0))
    return inst.from_triplets(f"binmix_{seed}", n, m, rows, cols, vals, np.zeros(n), np.ones(n), np.ones(n),
                              np.array(rhs), np.full(n, inst.VAR_BIN), sense, x0=np.zeros(n))


def single_run(chap, prob, tenure, iters, stop):
    bs = chap.BestShift(prob, tenure=tenure)
    r = bs.run(max_iters=iters, stop_at_feasible=1 if stop else 0, graph_iters=32)
    st = bs.state()
    bs.close()
    return r, st


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("schedule", [(8, 4), (4, 2), (16, 8), (2, 4)])
def test_chains_follow_single_handles(chap, schedule, persistent):
    probs = [inst.gen_setcover(seed=5, n=300, m=150, k=6), binary_mixed(7, 500, 260),
             inst.gen_setcover(seed=6, n=1300, m=700, k=8)]
    chain_prob = [0, 0, 1, 1, 2, 2, 1]
    tenures = [3, 10, 3, 10, 5, 20, 0]
    b = chap.BatchChains(probs, chain_prob, tenures)
    b.set_schedule(*schedule)
    b.set_persistent(persistent)
    res, _ = b.run(max_iters=300, stop_at_feasible=False, graph_iters=32)
    for c, (k, t) in enumerate(zip(chain_prob, tenures)):
        r, st = single_run(chap, probs[k], t, 300, False)
        assert (res[c].iters, res[c].moves, res[c].final_nviol, res[c].best_nviol, res[c].feasible_iter) == \
            (st["iter"], st["moves"], st["nviol"], st["best_nviol"], st["feasible_iter"]), c
        assert np.array_equal(b.x(c), st["x"]), c
    b.close()


@pytest.mark.parametrize("persistent", [1, 0])
def test_stop_at_feasible_and_continue(chap, persistent):
    probs = [inst.gen_setcover(seed=s, n=400 + 300 * s, m=200 + 150 * s, k=6) for s in range(3)]
    chain_prob = [0, 1, 2, 0, 1, 2]
    tenures = [10, 10, 10, 2, 2, 2]
    b = chap.BatchChains(probs, chain_prob, tenures)
    b.set_persistent(persistent)
    res, secs = b.run(max_iters=5000, stop_at_feasible=True, graph_iters=64)
    for c, (k, t) in enumerate(zip(chain_prob, tenures)):
        r, st = single_run(chap, probs[k], t, 5000, True)
        assert res[c].feasible_iter == st["feasible_iter"] and res[c].iters == st["iter"], c
        assert np.array_equal(b.x(c), st["x"]), c
        if res[c].feasible_iter >= 0:
            assert res[c].final_nviol == 0 and res[c].time_to_feasible_s >= 0
    # a second run continues every chain (feasible ones are done at once)
    res2, _ = b.run(max_iters=50, stop_at_feasible=True)
    for c in range(len(chain_prob)):
        if res[c].feasible_iter >= 0:
            assert res2[c].iters == res[c].iters
        else:
            assert res2[c].iters == res[c].iters + 50
    b.close()


def test_chain_matches_oracle(chap):
    prob = binary_mixed(11, 60, 40, k=4)
    b = chap.BatchChains([prob], [0, 0], [4, 9])
    res, _ = b.run(max_iters=120, stop_at_feasible=False)
    orc = Oracle(prob)
    for c, t in enumerate([4, 9]):
        ost = orc.initial_state()
        tr = orc.run(ost, tenure=t, n_iters=120, stop_at_feasible=False)
        assert np.array_equal(b.x(c), ost["x"]), c
        assert res[c].moves == int(np.sum(tr["var"] >= 0)), c
    b.close()


def test_autotune_keeps_results(chap):
    probs = inst.gen_batch(n_instances=4, first_seed=1, n_min=1000, n_max=20_000)
    chain_prob = [k for k in range(4) for _ in range(2)]
    tenures = [5, 50] * 4
    b = chap.BatchChains(probs, chain_prob, tenures)
    res_a, _ = b.run(max_iters=200, stop_at_feasible=False)
    xa = [b.x(c) for c in range(len(chain_prob))]
    g, ctas, pers = b.autotune(iters=3)
    assert g in (2, 4, 8, 16) and ctas in (2, 4, 8) and pers in (0, 1)
    res_b, _ = b.run(max_iters=200, stop_at_feasible=False)
    for c in range(len(chain_prob)):
        assert (res_a[c].moves, res_a[c].final_nviol) == (res_b[c].moves, res_b[c].final_nviol)
        assert np.array_equal(xa[c], b.x(c))
    b.close()


def test_unsupported_instance_rejected(chap):
    prob = inst.gen_tiny_mixed(0, n=6, m=5)
    with pytest.raises(chap.ChapError):
        chap.BatchChains([prob], [0], [3])


def test_persistent_barrier_wait_runs_out(chap):
    """A barrier bound of 1 ns makes the first wait that is not met at once
    run out: every CTA leaves the launch, the run reports CHAP_E_TIMEOUT, the
    context stays usable, and after a reset the same batch (default bound)
    follows the single-handle trajectories again."""
    probs = [inst.gen_setcover(seed=5, n=3000, m=1500, k=6), binary_mixed(8, 2000, 1000)]
    chain_prob = [0, 1, 0, 1]
    tenures = [3, 3, 10, 10]
    b = chap.BatchChains(probs, chain_prob, tenures)
    b.set_schedule(8, 4)
    b.set_persistent(1, barrier_limit_ns=1)
    with pytest.raises(chap.ChapError) as ei:
        b.run(max_iters=64, stop_at_feasible=False, graph_iters=16)
    assert ei.value.status == chap.CHAP_E_TIMEOUT
    with pytest.raises(chap.ChapError) as ei:
        b.run(max_iters=8, stop_at_feasible=False)
    assert ei.value.status == chap.CHAP_E_STATE
    b.reset()
    b.set_persistent(1, barrier_limit_ns=2_000_000_000)
    res, _ = b.run(max_iters=100, stop_at_feasible=False, graph_iters=16)
    for c, (k, t) in enumerate(zip(chain_prob, tenures)):
        r, st = single_run(chap, probs[k], t, 100, False)
        assert res[c].moves == st["moves"] and np.array_equal(b.x(c), st["x"]), c
    b.close()
