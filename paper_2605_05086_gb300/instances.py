"""Seeded synthetic MIP instances for the best-shift tabu search.

This module only draws problem data: sparsity patterns, coefficients, bounds,
variable types, row senses and right-hand sides.  It contains none of the
method's arithmetic (no residuals, scores, breakpoints or moves), so both the
CPU oracle and the CUDA path may use it as their common input source.

The MIP form is the one of Sec. 3.1: min c^T x  s.t.  rows of A x (<=, >=, =) b,
l <= x <= u, x_j integer for j in I.  Instances are returned with both CSR and
CSC copies of A (the CSC copy is the exact transpose, rows ascending inside each
column), bounds, objective, variable types and row senses.

The paper evaluates on competition instances that are not available here; the
workloads below are synthetic stand-ins whose shapes follow the five workload
descriptions this library is measured on (set-cover-like binary, general
integer with power-law rows, skewed large with dense columns, a batch of uneven
set-cover-like instances, and a large set-cover-like instance).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

VAR_BIN, VAR_INT, VAR_CONT = 0, 1, 2
ROW_LE, ROW_GE, ROW_EQ = 0, 1, 2


@dataclass
class Problem:
    """A MIP in CSR + CSC form (0-based, int64 pointers, int32 indices, float64 values)."""

    name: str
    n: int
    m: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    row_val: np.ndarray
    col_ptr: np.ndarray
    row_idx: np.ndarray
    col_val: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    obj: np.ndarray
    rhs: np.ndarray
    vtype: np.ndarray
    sense: np.ndarray
    x0: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def csc_from_csr(n, row_ptr, col_idx, row_val):
    """Transpose a CSR matrix; rows stay ascending inside each column (stable sort)."""
    m = len(row_ptr) - 1
    rows = np.repeat(np.arange(m, dtype=np.int32), np.diff(row_ptr))
    order = np.argsort(col_idx, kind="stable")
    counts = np.bincount(col_idx, minlength=n)
    col_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=col_ptr[1:])
    return col_ptr, rows[order].astype(np.int32), row_val[order].astype(np.float64)


def from_triplets(name, n, m, rows, cols, vals, lb, ub, obj, rhs, vtype, sense, x0=None, meta=None):
    """Build a Problem from (row, col, value) triplets (duplicates are not allowed)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.argsort(rows * np.int64(max(n, 1)) + cols, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    if len(rows) > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate (row, col) entries")
    counts = np.bincount(rows, minlength=m) if len(rows) else np.zeros(m, dtype=np.int64)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = cols.astype(np.int32)
    row_val = vals
    col_ptr, row_idx, col_val = csc_from_csr(n, row_ptr, col_idx, row_val)
    lb = np.asarray(lb, dtype=np.float64)
    ub = np.asarray(ub, dtype=np.float64)
    if x0 is None:
        x0 = np.clip(np.zeros(n), lb, ub)
    return Problem(
        name=name, n=n, m=m,
        row_ptr=row_ptr, col_idx=col_idx, row_val=row_val,
        col_ptr=col_ptr, row_idx=row_idx, col_val=col_val,
        lb=lb, ub=ub,
        obj=np.asarray(obj, dtype=np.float64),
        rhs=np.asarray(rhs, dtype=np.float64),
        vtype=np.asarray(vtype, dtype=np.uint8),
        sense=np.asarray(sense, dtype=np.uint8),
        x0=np.asarray(x0, dtype=np.float64),
        meta=dict(meta or {}),
    )


def with_objective_row(prob, rhs=None):
    """The problem with one more row, c^T x <= rhs, appended last (index m): the
    row an objective cutoff tightens.  Default rhs: the largest value of c^T x
    over the bounds (the row starts satisfied); a variable with c_j = 0 has no
    entry in it."""
    c = np.asarray(prob.obj, dtype=np.float64)
    nzc = np.flatnonzero(c != 0.0)
    if rhs is None:
        hi = np.where(c[nzc] > 0, prob.ub[nzc], prob.lb[nzc])
        rhs = float(np.sum(c[nzc] * hi)) if len(nzc) else 0.0
        if not np.isfinite(rhs):
            raise ValueError("an unbounded objective term: give rhs")
    rows = np.repeat(np.arange(prob.m, dtype=np.int64), np.diff(prob.row_ptr))
    rows = np.concatenate([rows, np.full(len(nzc), prob.m, dtype=np.int64)])
    cols = np.concatenate([prob.col_idx.astype(np.int64), nzc.astype(np.int64)])
    vals = np.concatenate([prob.row_val, c[nzc]])
    return from_triplets(prob.name + "+obj", prob.n, prob.m + 1, rows, cols, vals, prob.lb, prob.ub, prob.obj,
                         np.append(prob.rhs, rhs), prob.vtype, np.append(prob.sense, ROW_LE), x0=prob.x0,
                         meta=dict(prob.meta, cutoff_row=prob.m))


def _distinct_segments(rng, lengths, pool_size):
    """For segment s draw lengths[s] distinct values uniformly from range(pool_size).

    Returns (segment_id, value) arrays sorted by (segment, value).  Duplicates
    inside a segment are redrawn until none remain, so each segment is a uniform
    sample without replacement.
    """
    lengths = np.asarray(lengths, dtype=np.int64)
    if (lengths > pool_size).any():
        raise ValueError("segment longer than its pool")
    seg = np.repeat(np.arange(len(lengths), dtype=np.int64), lengths)
    val = rng.integers(0, pool_size, size=len(seg), dtype=np.int64)
    P = np.int64(pool_size)
    while True:
        key = np.sort(seg * P + val)
        dup = np.zeros(len(key), dtype=bool)
        if len(key) > 1:
            dup[1:] = key[1:] == key[:-1]
        seg, val = key // P, key % P
        k = int(dup.sum())
        if k == 0:
            return seg, val
        val[dup] = rng.integers(0, pool_size, size=k, dtype=np.int64)


def _rhs_from_hidden_point(rng, m, row_ptr, col_idx, row_val, xstar, sense, integral_row):
    """rhs = a.x* +/- slack (<= rows: +s, >= rows: -s, = rows: 0); integral rows get integer slack."""
    rows = np.repeat(np.arange(m), np.diff(row_ptr))
    ax = np.bincount(rows, weights=row_val * xstar[col_idx], minlength=m)
    s_int = rng.integers(0, 11, size=m).astype(np.float64)
    s_fp = rng.random(m)
    s = np.where(integral_row, s_int, s_fp)
    rhs = np.where(sense == ROW_LE, ax + s, np.where(sense == ROW_GE, ax - s, ax))
    return rhs


def gen_setcover(seed=0, n=2000, m=1000, k=8, name=None):
    """Set-cover-like binary MIP: m >= rows over k distinct uniform columns,
    integer coefficients U{1..5}, rhs = ceil(0.3 * row sum), objective U{1..10},
    x0 = 0 (the 2,000-var / 1,000-row / 8-per-row workload at the default sizes)."""
    rng = np.random.default_rng(seed)
    seg, cols = _distinct_segments(rng, np.full(m, k), n)
    vals = rng.integers(1, 6, size=len(seg)).astype(np.float64)
    rowsum = np.bincount(seg, weights=vals, minlength=m)
    rhs = np.ceil(0.3 * rowsum)
    obj = rng.integers(1, 11, size=n).astype(np.float64)
    return from_triplets(
        name or f"setcover_n{n}_m{m}_k{k}_s{seed}", n, m, seg, cols, vals,
        lb=np.zeros(n), ub=np.ones(n), obj=obj, rhs=rhs,
        vtype=np.full(n, VAR_BIN), sense=np.full(m, ROW_GE), x0=np.zeros(n),
        meta={"kind": "setcover", "seed": seed},
    )


def gen_general(seed=0, n=200_000, m=100_000, len_cap=5000, name=None):
    """General integer MIP: 70% binary / 20% integer in [0,100] / 10% continuous in
    [0,1e3]; senses 40% <=, 40% >=, 20% =; row lengths Zipf(1.5) clipped to
    [2, len_cap]; half the rows integral (columns from binary/integer vars,
    coefficients U{-20..20}\\{0}), half mixed (columns from all vars, N(0,1)
    coefficients); rhs from a hidden point plus slack (U{0..10} on integral rows,
    U[0,1) on mixed rows); x0 = 0."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    n_bin, n_int = int(0.7 * n), int(0.2 * n)
    vtype = np.empty(n, dtype=np.uint8)
    vtype[perm[:n_bin]] = VAR_BIN
    vtype[perm[n_bin:n_bin + n_int]] = VAR_INT
    vtype[perm[n_bin + n_int:]] = VAR_CONT
    lb = np.zeros(n)
    ub = np.where(vtype == VAR_BIN, 1.0, np.where(vtype == VAR_INT, 100.0, 1000.0))
    sense = rng.choice(np.array([ROW_LE, ROW_GE, ROW_EQ], dtype=np.uint8), size=m, p=[0.4, 0.4, 0.2])
    lengths = np.clip(rng.zipf(1.5, size=m), 2, len_cap).astype(np.int64)
    integral_row = rng.random(m) < 0.5
    int_pool = np.sort(np.nonzero(vtype != VAR_CONT)[0])
    all_pool = np.arange(n)
    lengths = np.where(integral_row, np.minimum(lengths, len(int_pool)), lengths)
    rows_i = np.nonzero(integral_row)[0]
    rows_m = np.nonzero(~integral_row)[0]
    seg_i, c_i = _distinct_segments(rng, lengths[rows_i], len(int_pool))
    seg_m, c_m = _distinct_segments(rng, lengths[rows_m], len(all_pool))
    mag = rng.integers(1, 21, size=len(seg_i))
    sgn = np.where(rng.random(len(seg_i)) < 0.5, -1, 1)
    v_i = (mag * sgn).astype(np.float64)
    v_m = rng.standard_normal(len(seg_m))
    rows = np.concatenate([rows_i[seg_i], rows_m[seg_m]])
    cols = np.concatenate([int_pool[c_i], all_pool[c_m]])
    vals = np.concatenate([v_i, v_m])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    xstar = np.where(vtype == VAR_BIN, rng.integers(0, 2, size=n),
                     np.where(vtype == VAR_INT, rng.integers(0, 101, size=n), 0)).astype(np.float64)
    cont = vtype == VAR_CONT
    xstar[cont] = rng.random(int(cont.sum())) * 1000.0
    rhs = _rhs_from_hidden_point(rng, m, row_ptr, cols.astype(np.int32), vals, xstar, sense, integral_row)
    obj = rng.integers(1, 11, size=n).astype(np.float64)
    return from_triplets(
        name or f"general_n{n}_m{m}_cap{len_cap}_s{seed}", n, m, rows, cols, vals,
        lb=lb, ub=ub, obj=obj, rhs=rhs, vtype=vtype, sense=sense, x0=np.zeros(n),
        meta={"kind": "general", "seed": seed, "len_cap": len_cap},
    )


def gen_skewed(seed=0, n=2_000_000, m=1_000_000, col_cap=14, n_dense=50, dense_len=100_000, name=None):
    """Skewed large integral MIP: 90% binary / 10% integer in [0,1000]; column
    lengths Zipf(1.3) clipped to [1, col_cap] plus n_dense integer columns of
    exactly dense_len entries; coefficients U{-50..50}\\{0}; senses 40/40/20;
    rhs from a hidden point plus integer slack U{0..10}; x0 = 0."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    n_bin = int(0.9 * n)
    vtype = np.empty(n, dtype=np.uint8)
    vtype[perm[:n_bin]] = VAR_BIN
    vtype[perm[n_bin:]] = VAR_INT
    lb = np.zeros(n)
    ub = np.where(vtype == VAR_BIN, 1.0, 1000.0)
    lengths = np.clip(rng.zipf(1.3, size=n), 1, col_cap).astype(np.int64)
    lengths = np.minimum(lengths, m)
    int_vars = perm[n_bin:]
    dense = np.sort(rng.choice(int_vars, size=min(n_dense, len(int_vars)), replace=False))
    lengths[dense] = min(dense_len, m)
    seg, rws = _distinct_segments(rng, lengths, m)
    mag = rng.integers(1, 51, size=len(seg))
    sgn = np.where(rng.random(len(seg)) < 0.5, -1, 1)
    vals = (mag * sgn).astype(np.float64)
    sense = rng.choice(np.array([ROW_LE, ROW_GE, ROW_EQ], dtype=np.uint8), size=m, p=[0.4, 0.4, 0.2])
    rows, cols = rws, seg
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    xstar = np.where(vtype == VAR_BIN, rng.integers(0, 2, size=n), rng.integers(0, 1001, size=n)).astype(np.float64)
    rhs = _rhs_from_hidden_point(rng, m, row_ptr, cols.astype(np.int32), vals, xstar, sense, np.ones(m, dtype=bool))
    obj = rng.integers(1, 11, size=n).astype(np.float64)
    return from_triplets(
        name or f"skewed_n{n}_m{m}_s{seed}", n, m, rows, cols, vals,
        lb=lb, ub=ub, obj=obj, rhs=rhs, vtype=vtype, sense=sense, x0=np.zeros(n),
        meta={"kind": "skewed", "seed": seed, "dense_cols": dense.tolist()},
    )


def gen_batch(n_instances=64, first_seed=1, n_min=1000, n_max=200_000, nnz_per_var=10, k=8):
    """Uneven batch of set-cover-like instances: n log-uniform in [n_min, n_max],
    nnz = nnz_per_var * n, m = nnz / k rows of k entries, seeds first_seed..."""
    out = []
    for s in range(first_seed, first_seed + n_instances):
        rng = np.random.default_rng(10_000 + s)
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        m = max(1, (nnz_per_var * n) // k)
        out.append(gen_setcover(seed=s, n=n, m=m, k=k, name=f"batch_{s}_n{n}_m{m}"))
    return out


def gen_tiny_mixed(seed, n=6, m=5, max_len=4, dom=12, cont_frac=0.0, dyadic=True, eq_frac=0.2):
    """Tiny mixed instances for exhaustive checks: integer (and optionally
    continuous) variables with small domains, short rows, all three senses.
    With dyadic=True every coefficient, bound, rhs and start value is a small
    dyadic rational, so double arithmetic on them is exact."""
    rng = np.random.default_rng(seed)
    vtype = np.where(rng.random(n) < 0.3, VAR_BIN, VAR_INT).astype(np.uint8)
    if cont_frac > 0:
        vtype[rng.random(n) < cont_frac] = VAR_CONT
    lb = np.where(vtype == VAR_BIN, 0.0, rng.integers(-3, 2, size=n).astype(np.float64))
    width = rng.integers(1, dom, size=n).astype(np.float64)
    ub = np.where(vtype == VAR_BIN, 1.0, lb + width)
    lengths = rng.integers(1, max_len + 1, size=m)
    lengths = np.minimum(lengths, n)
    seg, cols = _distinct_segments(rng, lengths, n)
    if dyadic:
        choices = np.array([-4, -2, -1, -0.5, 0.5, 1, 2, 4], dtype=np.float64)
        vals = rng.choice(choices, size=len(seg))
    else:
        vals = rng.integers(1, 6, size=len(seg)) * np.where(rng.random(len(seg)) < 0.5, -1, 1)
        vals = vals.astype(np.float64)
    sense = rng.choice(np.array([ROW_LE, ROW_GE, ROW_EQ], dtype=np.uint8), size=m,
                       p=[(1 - eq_frac) / 2, (1 - eq_frac) / 2, eq_frac])
    x0 = np.where(vtype == VAR_CONT, lb, lb + np.floor(rng.random(n) * (ub - lb + 1)))
    x0 = np.minimum(x0, ub)
    cont = vtype == VAR_CONT
    if cont.any():
        x0[cont] = lb[cont] + np.floor(rng.random(int(cont.sum())) * 4 * (ub[cont] - lb[cont])) / 4
    rows = seg
    rowsum_x = np.bincount(rows, weights=vals * x0[cols], minlength=m)
    shift = rng.integers(-3, 4, size=m).astype(np.float64)
    rhs = rowsum_x + shift
    obj = rng.integers(1, 5, size=n).astype(np.float64)
    return from_triplets(
        f"tiny_s{seed}", n, m, rows, cols, vals, lb=lb, ub=ub, obj=obj, rhs=rhs,
        vtype=vtype, sense=sense, x0=x0, meta={"kind": "tiny", "seed": seed},
    )


WORKLOADS = {
    "setcover_2k": dict(fn=gen_setcover, kw=dict(seed=0, n=2000, m=1000, k=8)),
    "general_200k": dict(fn=gen_general, kw=dict(seed=0, n=200_000, m=100_000, len_cap=5000)),
    "skewed_2m": dict(fn=gen_skewed, kw=dict(seed=0)),
    "setcover_200k": dict(fn=gen_setcover, kw=dict(seed=5, n=200_000, m=100_000, k=8)),
}


def make(name):
    spec = WORKLOADS[name]
    return spec["fn"](**spec["kw"])
