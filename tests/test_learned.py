"""Learned proposal path: features, network forward / gradient / Adam against
the CPU oracle (oracle/mlp.py), the top-k rule, exactness of the learned loop,
and what training gains."""
import numpy as np
import pytest

from oracle import mlp
from oracle.oracle import Oracle
from paper_2605_05086_gb300 import instances as inst

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2605_05086_gb300 import chap, learn
    chap.load()
    return torch, chap, learn


def bf16(torch, a):
    """float64 numpy -> BF16-rounded float64 numpy (the values the kernels see)."""
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def test_features_match_oracle(env):
    torch, chap, learn = env
    prob = inst.gen_setcover(seed=3, n=400, m=220, k=6)
    bs = chap.BestShift(prob, tenure=7)
    orc = Oracle(prob)
    bs.run(max_iters=40, stop_at_feasible=0)
    chap.chap_bs_refresh_features(bs.h)
    st = bs.state()
    bs.run(max_iters=3, stop_at_feasible=0)   # features three iterations after the pass
    st2 = bs.state()
    f = torch.empty((prob.n, 12), dtype=torch.int16, device="cuda")
    t = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    chap.chap_bs_features(bs.h, f, t)
    got = f.view(torch.bfloat16).to(torch.float64).cpu().numpy()
    # oracle: scores and column features at the pass state, the rest at the current state
    _, _, nv = orc.residuals(st["x"])
    _, s_last, _ = orc.best_shift(st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], nv, st["best_nviol"])
    cv, cw = mlp.column_stats(prob, st["x"], st["w"])
    want = mlp.features(prob, st2["x"], st2["tabu_inc"], st2["tabu_dec"], st2["iter"], 7, cv, cw,
                        s_last.astype(float), 3)
    want = bf16(torch, want)
    # features are FP32 on the GPU, rounded once to BF16: at most one BF16 step apart
    assert np.all(np.abs(got - want) <= np.abs(want) / 128 + 1e-30), np.argwhere(np.abs(got - want) > np.abs(want) / 128)[:5]
    tgt = t.cpu().numpy()
    assert np.allclose(tgt, s_last / (1.0 + np.max(np.abs(s_last))), rtol=1e-6, atol=1e-7)
    bs.close()


def test_forward_and_gradient_match_oracle(env):
    torch, chap, learn = env
    rng = np.random.default_rng(0)
    p = bf16(torch, mlp.init_params(2))
    x = bf16(torch, rng.standard_normal((1000, 12)))
    t = rng.standard_normal(1000)
    w_d = torch.tensor(p, dtype=torch.float32).to(torch.bfloat16).view(torch.int16).cuda()
    x_d = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).view(torch.int16).cuda()
    y = torch.empty(1000, dtype=torch.float32, device="cuda")
    chap.chap_mlp_forward(w_d, x_d, y)
    y_ref = mlp.forward(p, x)
    assert np.allclose(y.cpu().numpy(), y_ref, rtol=1e-4, atol=1e-4 * np.max(np.abs(y_ref)))
    g = torch.zeros(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    t_d = torch.tensor(t, dtype=torch.float32, device="cuda")
    chap.chap_mlp_loss_grad(w_d, x_d, t_d, g, loss)
    l_ref, g_ref = mlp.loss_and_grad(p, x, t.astype(np.float32).astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    cos = gg @ g_ref / (np.linalg.norm(gg) * np.linalg.norm(g_ref))
    assert cos > 0.99999, cos
    assert np.max(np.abs(gg - g_ref)) <= 1e-3 * np.max(np.abs(g_ref))
    assert abs(loss.item() / 1000 - l_ref) <= 1e-4 * l_ref


def test_adam_step(env):
    torch, chap, learn = env
    rng = np.random.default_rng(1)
    w = rng.standard_normal(mlp.N_PARAMS).astype(np.float32)
    g = rng.standard_normal(mlp.N_PARAMS).astype(np.float32)
    w32 = torch.tensor(w, device="cuda")
    wbf = torch.zeros(mlp.N_PARAMS, dtype=torch.int16, device="cuda")
    m = torch.zeros_like(w32); v = torch.zeros_like(w32); gd = torch.tensor(g, device="cuda")
    chap.chap_mlp_adam(w32, wbf, m, v, gd, 1, 1e-2)
    # first step: m = 0.1 g, v = 0.001 g^2, corrected m/c1 = g, v/c2 = g^2: w - lr g / (|g| + eps)
    want = w - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.allclose(w32.cpu().numpy(), want, rtol=1e-5, atol=1e-6)
    assert np.all(gd.cpu().numpy() == 0)
    assert np.array_equal(wbf.view(torch.bfloat16).float().cpu().numpy(),
                          torch.tensor(want).to(torch.bfloat16).float().numpy())


def test_topk_is_the_k_largest_by_index_ties(env):
    torch, chap, learn = env
    prob = inst.gen_setcover(seed=4, n=3000, m=1500, k=8)
    bs = chap.BestShift(prob, tenure=10)
    chap.chap_bs_refresh_features(bs.h)
    w = learn.to_bf16_bits(torch.tensor(learn.init_params(5), device="cuda"))
    for k in (1, 100, 777, 3000):
        lst = torch.empty(k, dtype=torch.int32, device="cuda")
        pred = torch.empty(prob.n, dtype=torch.float32, device="cuda")
        chap.chap_bs_propose(bs.h, w, k, lst, pred)
        got = np.sort(lst.cpu().numpy())
        assert np.array_equal(got, mlp.topk(pred.cpu().numpy(), k)), k
    bs.close()


@pytest.mark.parametrize("mode", ["all_vars", "exact_every_iteration"])
def test_learned_loop_reduces_to_exact(env, mode):
    """With k = n (or an exact pass every iteration) the learned loop must take
    exactly the moves of the plain exact driver."""
    torch, chap, learn = env
    prob = inst.gen_setcover(seed=8, n=900, m=500, k=7)
    w = learn.to_bf16_bits(torch.tensor(learn.init_params(1), device="cuda"))
    a = chap.BestShift(prob, tenure=5)
    b = chap.BestShift(prob, tenure=5)
    kw = dict(topk=prob.n, exact_every=7, propose_every=3) if mode == "all_vars" else \
        dict(topk=10, exact_every=1, propose_every=1)
    r = chap.chap_learned_run(a.h, w, max_iters=300, stop_at_feasible=False, **kw)
    b.run(max_iters=300, stop_at_feasible=0)
    sa, sb = a.state(), b.state()
    assert r.iters == 300
    assert np.array_equal(sa["x"], sb["x"]) and np.array_equal(sa["w"], sb["w"])
    assert (sa["moves"], sa["nviol"], sa["best_nviol"]) == (sb["moves"], sb["nviol"], sb["best_nviol"])
    if mode == "all_vars":
        assert r.misses == 0 and r.exact_passes == 300 // 7 + 1


def test_training_lowers_the_miss_rate(env):
    """What the trained network gains over the same path with an untrained one:
    fewer top-1 misses at the exact passes."""
    torch, chap, learn = env
    prob = inst.gen_setcover(seed=11, n=20_000, m=10_000, k=8)
    bs = chap.BestShift(prob, tenure=10)
    x, t = learn.log_pairs(bs, passes=12, iters_between=25)
    wbf, _, curve = learn.train(x, t, epochs=4, batch=2048, lr=3e-3, seed=0)
    assert curve[-1] < curve[0]
    rates = {}
    for name, w in (("trained", wbf), ("untrained", learn.to_bf16_bits(torch.tensor(learn.init_params(0), device="cuda")))):
        h = chap.BestShift(prob, tenure=10)
        r = chap.chap_learned_run(h.h, w, topk=256, exact_every=10, propose_every=1, max_iters=600,
                                  stop_at_feasible=False)
        rates[name] = r.misses / max(1, r.exact_passes)
        h.close()
    assert rates["trained"] < rates["untrained"], rates


def test_tensor_core_forward_in_proposals(env):
    """The proposal's forward pass runs its second layer on the tensor cores with
    BF16 first-layer activations: within BF16 rounding of the FP64 oracle."""
    torch, chap, learn = env
    prob = inst.gen_setcover(seed=6, n=5000, m=2500, k=8)
    bs = chap.BestShift(prob, tenure=10)
    bs.run(max_iters=30, stop_at_feasible=0)
    chap.chap_bs_refresh_features(bs.h)
    p = bf16(torch, mlp.init_params(7))
    w = torch.tensor(p, dtype=torch.float32).to(torch.bfloat16).view(torch.int16).cuda()
    pred = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    chap.chap_bs_propose(bs.h, w, 64, None, pred)
    f = torch.empty((prob.n, 12), dtype=torch.int16, device="cuda")
    chap.chap_bs_features(bs.h, f, None)
    x = f.view(torch.bfloat16).to(torch.float64).cpu().numpy()
    ref = mlp.forward(p, x)
    got = pred.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 2e-2 * np.max(np.abs(ref)), np.max(np.abs(got - ref))
    # with the first-layer activations rounded to BF16 as the kernel does, the
    # rest is FP32 accumulation against FP64: agreement to ~1e-5
    q = mlp.unpack(p)
    h1 = bf16(torch, np.maximum(x @ q["W1"] + q["b1"], 0.0))
    ref16 = np.maximum(h1 @ q["W2"] + q["b2"], 0.0) @ q["w3"] + q["b3"][0]
    assert np.max(np.abs(got - ref16)) <= 1e-4 * max(1.0, np.max(np.abs(ref16))), np.max(np.abs(got - ref16))
    bs.close()


def _mixed_small(seed):
    """General-family instance (binary, integer and continuous variables, integral
    and N(0,1) rows) with short columns only: every non-binary column is
    evaluated by the proposal's Algorithm 1 kernel."""
    return inst.gen_general(seed=seed, n=6000, m=3000, len_cap=40)


@pytest.mark.parametrize("mode", ["all_vars", "exact_every_iteration"])
def test_learned_loop_reduces_to_exact_mixed(env, mode):
    """Mixed instance: with k = n the proposal evaluates every column exactly
    (flips and Algorithm 1), so the learned loop takes the plain driver's
    moves, shift values included."""
    torch, chap, learn = env
    prob = _mixed_small(3)
    w = learn.to_bf16_bits(torch.tensor(learn.init_params(1), device="cuda"))
    a = chap.BestShift(prob, tenure=5)
    b = chap.BestShift(prob, tenure=5)
    assert a.info.n_int > 0 and a.info.n_cont > 0
    assert a.info.n_cta_cols == 0 and a.info.n_hist_cols == 0 and a.info.n_long_cols == 0
    kw = dict(topk=prob.n, exact_every=7, propose_every=3) if mode == "all_vars" else \
        dict(topk=50, exact_every=1, propose_every=1)
    r = chap.chap_learned_run(a.h, w, max_iters=200, stop_at_feasible=False, **kw)
    b.run(max_iters=200, stop_at_feasible=0)
    sa, sb = a.state(), b.state()
    assert r.iters == 200
    assert np.array_equal(sa["x"], sb["x"]) and np.array_equal(sa["w"], sb["w"])
    assert (sa["moves"], sa["nviol"], sa["best_nviol"]) == (sb["moves"], sb["nviol"], sb["best_nviol"])
    if mode == "all_vars":
        assert r.misses == 0


def test_training_on_both_families_lowers_the_miss_rate_on_mixed(env):
    """Pairs logged from a set-cover and a general-family instance (the two
    workloads' families), trained on the GPU: fewer top-1 misses at the exact
    passes on a mixed instance than the untrained network."""
    torch, chap, learn = env
    xs, ts = [], []
    for prob in (inst.gen_setcover(seed=12, n=20_000, m=10_000, k=8), inst.gen_general(seed=13, n=20_000, m=10_000,
                                                                                         len_cap=60)):
        bs = chap.BestShift(prob, tenure=10)
        x, t = learn.log_pairs(bs, passes=8, iters_between=25)
        xs.append(x); ts.append(t)
        bs.close()
    wbf, _, curve = learn.train(torch.cat(xs), torch.cat(ts), epochs=4, batch=2048, lr=3e-3, seed=0)
    assert curve[-1] < curve[0]
    prob = inst.gen_general(seed=14, n=20_000, m=10_000, len_cap=60)
    rates = {}
    for name, w in (("trained", wbf), ("untrained", learn.to_bf16_bits(torch.tensor(learn.init_params(0), device="cuda")))):
        h = chap.BestShift(prob, tenure=10)
        r = chap.chap_learned_run(h.h, w, topk=512, exact_every=10, propose_every=1, max_iters=400,
                                  stop_at_feasible=False)
        rates[name] = r.misses / max(1, r.exact_passes)
        h.close()
    assert rates["trained"] < rates["untrained"], rates
