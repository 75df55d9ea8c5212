"""Loading a state (chap_bs_set_state, chap_bs_set_checkpoint) recomputes every
row's residual on the device: integral rows in int64, the others as the double
sum of their products in CSR order, one lane per row with the products staged
128 entries at a time.  The residuals, margins and violation count must equal
the oracle's bit for bit, on rows shorter and longer than one staging phase,
with given weights, and with -0 in x (stored as +0)."""
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


def rows_of_lengths(seed, lengths, n=6000):
    """Mixed rows of the given lengths (N(0,1) coefficients, every kind of
    variable) next to integral rows of the same lengths; senses cycle."""
    rng = np.random.default_rng(seed)
    vt = rng.choice(np.array([B, I, C], dtype=np.uint8), size=n, p=[0.5, 0.3, 0.2])
    lb = np.zeros(n)
    ub = np.where(vt == B, 1.0, np.where(vt == I, 50.0, 300.0))
    rows, cols, vals, rhs, sense = [], [], [], [], []
    ints = np.nonzero(vt != C)[0]
    i = 0
    for L in lengths:
        for integral in (False, True):
            js = rng.choice(ints if integral else np.arange(n), size=L, replace=False)
            a = rng.integers(-9, 10, size=L).astype(float) if integral else rng.standard_normal(L)
            if integral:
                a[a == 0] = 1.0
            rows += [i] * L
            cols += list(js)
            vals += list(a)
            rhs.append(float(rng.integers(-20, 21)) if integral else float(rng.standard_normal() * 10))
            sense.append(i % 3)
            i += 1
    return inst.from_triplets(f"lens_{seed}", n, i, rows, cols, vals, lb, ub, np.ones(n), np.array(rhs), vt,
                              np.array(sense, dtype=np.uint8), x0=np.zeros(n))


def random_x(prob, rng):
    x = rng.random(prob.n) * prob.ub
    x = np.where(prob.vtype == C, x, np.floor(x + 0.5))
    return np.minimum(np.maximum(x, prob.lb), prob.ub)


def check(bs, orc, x):
    st = bs.state()
    r, _, nv = orc.residuals(x)
    assert np.array_equal(bs.residuals(), r)
    assert st["nviol"] == nv


@pytest.mark.parametrize("seed", [0, 1])
def test_residuals_across_phase_boundaries(chap, seed):
    lengths = [1, 2, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 255, 256, 257, 640, 1000, 2500] * 3
    prob = rows_of_lengths(seed, lengths)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=5)
    rng = np.random.default_rng(seed + 10)
    for _ in range(3):
        x = random_x(prob, rng)
        bs.set_state(x)
        check(bs, orc, x)
    bs.close()


def test_residuals_general_family_with_weights(chap):
    prob = inst.gen_general(seed=4, n=20_000, m=10_000, len_cap=3000)
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=5)
    rng = np.random.default_rng(3)
    x = random_x(prob, rng)
    w = rng.integers(1, 50, size=bs.m_norm).astype(np.int32)
    bs.set_state(x, w)
    check(bs, orc, x)
    assert np.array_equal(bs.state()["w"], w)
    # the next pass sees the loaded weights: same scores as the oracle's
    st = bs.state()
    vars_ = rng.choice(prob.n, 300, replace=False).astype(np.int32)
    gx, gs, gd = (a[vars_] for a in bs.best_shift()[:3])
    ox, os_, od = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["nviol"],
                                 st["best_nviol"], vars=vars_)
    # FP bar: scores and violation changes equal, shifts within 1e-9 relative
    assert np.array_equal(gs, os_) and np.array_equal(gd, od)
    bad = np.nonzero(np.abs(gx - ox) > 1e-9 * np.maximum(1.0, np.abs(ox)))[0]
    assert len(bad) == 0, [(int(vars_[k]), int(prob.vtype[vars_[k]]), gx[k], ox[k], st["x"][vars_[k]], int(gs[k]))
                           for k in bad[:8]]
    # a checkpoint with other weights replaces them
    st["w"] = np.ones_like(w)
    bs.set_checkpoint(st)
    assert np.array_equal(bs.state()["w"], st["w"])
    check(bs, orc, x)
    bs.close()


def test_negative_zero_stored_as_positive(chap):
    prob = rows_of_lengths(7, [5, 70, 300])
    orc = Oracle(prob)
    bs = chap.BestShift(prob, tenure=5)
    x = np.zeros(prob.n)
    x[::2] = -0.0
    bs.set_state(x)
    got = bs.state()["x"]
    assert not np.any(np.signbit(got))
    check(bs, orc, np.zeros(prob.n))
    bs.close()


def test_invalid_weights_keep_the_state(chap):
    prob = rows_of_lengths(8, [5, 70])
    bs = chap.BestShift(prob, tenure=5)
    x = random_x(prob, np.random.default_rng(1))
    bs.set_state(x)
    before = bs.state()
    w = np.ones(bs.m_norm, np.int32)
    w[-1] = 0
    with pytest.raises(chap.ChapError):
        bs.set_state(np.zeros(prob.n), w)
    after = bs.state()
    assert np.array_equal(after["x"], before["x"]) and np.array_equal(after["w"], before["w"])
    bs.close()
