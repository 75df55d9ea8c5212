"""CPU oracle of the learned move-proposal network (test infrastructure only:
imported by tests/ and never by the library).

The network is not in the paper: it is the growth path that proposes a top-k
subset of variables for the exact best-shift pass.  Definition (plain FP64):
    h1 = relu(x W1 + b1)        x: [B, 12], W1: [12, 64]
    h2 = relu(h1 W2 + b2)       W2: [64, 64]
    y  = h2 w3 + b3             w3: [64]
    loss = mean((y - t)^2)
Parameters are one flat vector in the order W1 (row-major, input x output), b1,
W2, b2, w3, b3: 12*64 + 64 + 64*64 + 64 + 64 + 1 = 5057 values.

Also the per-variable features and the top-k rule of the proposal step.
"""
import numpy as np

F, H = 12, 64
SIZES = [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p):
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def forward(p, x):
    """Network output for each row of x."""
    q = unpack(p)
    h1 = np.maximum(x @ q["W1"] + q["b1"], 0.0)
    h2 = np.maximum(h1 @ q["W2"] + q["b2"], 0.0)
    return h2 @ q["w3"] + q["b3"][0]


def loss_and_grad(p, x, t):
    """Mean squared error and its gradient with respect to the flat parameters
    (backpropagation through the three layers)."""
    q = unpack(p)
    x = np.asarray(x, np.float64)
    a1 = x @ q["W1"] + q["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ q["W2"] + q["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ q["w3"] + q["b3"][0]
    B = x.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    gy = 2.0 * r / B
    g = {}
    g["w3"] = h2.T @ gy
    g["b3"] = np.array([gy.sum()])
    ga2 = np.outer(gy, q["w3"]) * (a2 > 0)
    g["W2"] = h1.T @ ga2
    g["b2"] = ga2.sum(0)
    ga1 = (ga2 @ q["W2"].T) * (a1 > 0)
    g["W1"] = x.T @ ga1
    g["b1"] = ga1.sum(0)
    return loss, np.concatenate([g[name].ravel() for name, _ in SIZES])


def init_params(seed):
    """He-uniform initial weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = []
    for name, shape in SIZES:
        if name.startswith("W") or name == "w3":
            fan_in = shape[0]
            lim = np.sqrt(6.0 / fan_in)
            p.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            p.append(np.zeros(int(np.prod(shape))))
    return np.concatenate(p)


def features(prob, x, tabu_inc, tabu_dec, it, tenure, colviol, colwv, s_last, iters_since_exact):
    """The 12 per-variable features of the proposal step (one row per variable):
    x/(u-l), (x-l)/(u-l), (u-x)/(u-l), min(tabu age, 64)/64, violated share of
    the column, violated weighted share, last exact score / (1 + max |score|),
    iterations since the last exact pass / 50, log2(1 + column length) / 16,
    is_binary, is_integer, c_j / max |c|.  colviol, colwv and s_last are the
    values recorded at the last exact pass."""
    n = prob.n
    lb, ub = prob.lb, prob.ub
    width = np.where(np.isfinite(ub - lb) & (ub > lb), ub - lb, 0.0)
    safe = np.where(width > 0, width, 1.0)
    f = np.zeros((n, 12))
    f[:, 0] = np.where(width > 0, x / safe, 0.0)
    f[:, 1] = np.where(width > 0, (x - lb) / safe, 0.0)
    f[:, 2] = np.where(width > 0, (ub - x) / safe, 0.0)
    last = np.maximum(tabu_inc, tabu_dec) - 1 - tenure
    moved = np.maximum(tabu_inc, tabu_dec) > 0
    age = np.where(moved, it - last, 64)
    f[:, 3] = np.minimum(age, 64) / 64.0
    f[:, 4] = colviol
    f[:, 5] = colwv
    smax = np.max(np.abs(s_last)) if n else 0
    f[:, 6] = s_last / (1.0 + smax)
    f[:, 7] = iters_since_exact / 50.0
    length = np.diff(prob.col_ptr)
    f[:, 8] = np.log2(1.0 + length) / 16.0
    f[:, 9] = (prob.vtype == 0).astype(float)
    f[:, 10] = (prob.vtype == 1).astype(float)
    cmax = np.max(np.abs(prob.obj)) if n else 0
    f[:, 11] = prob.obj / cmax if cmax > 0 else 0.0
    return f


def topk(scores, k):
    """Indices of the k largest scores, ties broken by the lower index."""
    order = np.lexsort((np.arange(len(scores)), -np.asarray(scores, np.float64)))
    return np.sort(order[:k])


def column_stats(prob, x, w, feas_tol=0.0):
    """Pass-time column features of every variable at assignment x with the
    normalised rows' weights w (canonical order): the share of the column's
    normalised halves that are violated, and their share of sum w |a|."""
    from oracle import definition as D
    rows = D.normalised_rows(prob, feas_tol)
    halves = np.zeros(prob.n)
    viol = np.zeros(prob.n)
    wall = np.zeros(prob.n)
    wviol = np.zeros(prob.n)
    xs = [D.F(float(v)) for v in x]
    for k, (coeffs, b, eps) in enumerate(rows):
        v = D.activity(coeffs, xs) - b > eps
        for j, a in coeffs.items():
            halves[j] += 1
            wall[j] += w[k] * abs(float(a))
            if v:
                viol[j] += 1
                wviol[j] += w[k] * abs(float(a))
    colviol = np.where(halves > 0, viol / np.maximum(halves, 1), 0.0)
    colwv = np.where(wall > 0, wviol / np.where(wall > 0, wall, 1.0), 0.0)
    return colviol, colwv
