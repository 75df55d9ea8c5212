"""Exhaustive definition of the best shift, in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY (tiny instances; pure Python loops).  It pins the C
oracle: for every variable it scores EVERY integer value of the domain D_j
(Eq. best_move, Sec. 3.1) -- not just breakpoints -- by recomputing the row
activities with fractions.Fraction and applying the penalty p_ij of
Sec. 3.1 ("Scoring Functions").  The C oracle's score must equal this maximum
and its value must be one of the maximisers: that checks the step-function
claim of Sec. 3.1 (the maximum over the domain is attained at a bound or a
breakpoint) together with the oracle's arithmetic.  When a whole interval ties,
the method (and the oracle) return the closest tying bound or breakpoint, which
need not be the closest tying domain value.

Rows are normalised to "<=" form in the same canonical order as the library's
interface ("<=": (a, b); ">=": (-a, -b); "=": (a, b) then (-a, -b)).
Violation: r = ybar - b > eps with eps = 0 on integral rows and
feas_tol * max(1, |b|) otherwise.
"""
from __future__ import annotations

from fractions import Fraction as F
import math

BIN, INT, CONT = 0, 1, 2
LE, GE, EQ = 0, 1, 2


def normalised_rows(prob, feas_tol=0.0):
    """List of (coeffs {j: Fraction}, rhs Fraction, eps Fraction) in canonical order."""
    out = []
    for i in range(prob.m):
        lo, hi = int(prob.row_ptr[i]), int(prob.row_ptr[i + 1])
        coeffs = {int(prob.col_idx[e]): F(float(prob.row_val[e])) for e in range(lo, hi)}
        b = F(float(prob.rhs[i]))
        integral = b.denominator == 1 and all(
            a.denominator == 1 and prob.vtype[j] != CONT
            and math.isfinite(prob.lb[j]) and math.isfinite(prob.ub[j])
            for j, a in coeffs.items())
        eps = F(0) if integral else F(feas_tol) * max(F(1), abs(b))
        s = int(prob.sense[i])
        if s in (LE, EQ):
            out.append((coeffs, b, eps))
        if s in (GE, EQ):
            out.append(({j: -a for j, a in coeffs.items()}, -b, eps))
    return out


def activity(coeffs, x):
    return sum((a * x[j] for j, a in coeffs.items()), F(0))


def penalty_half(r0, r1, eps, w):
    """2 * p_ij from the residuals before (r0) and after (r1) the move (Sec. 3.1)."""
    v0, v1 = r0 > eps, r1 > eps
    if not v0 and v1:
        return -2 * w
    if v0 and not v1:
        return 2 * w
    if v0 and v1 and r1 < r0:
        return w
    if v0 and v1 and r1 > r0:
        return -w
    return 0


def score(rows, x, w, j, v):
    """(2 * s_j(v, xbar), change in the number of violated rows) for moving x_j to v."""
    s, dc = 0, 0
    xv = list(x)
    xv[j] = F(v)
    for k, (coeffs, b, eps) in enumerate(rows):
        if j not in coeffs:
            continue
        r0 = activity(coeffs, x) - b
        r1 = activity(coeffs, xv) - b
        s += penalty_half(r0, r1, eps, int(w[k]))
        dc += int(r1 > eps) - int(r0 > eps)
    return s, dc


def admissible(v, xbar, j, dc, tabu_inc, tabu_dec, it, nviol, best_nviol):
    tabu = (it < tabu_inc[j]) if v > xbar else (it < tabu_dec[j])
    return (not tabu) or (nviol + dc < best_nviol)


def exhaustive_max(prob, x, w, tabu_inc, tabu_dec, it, nviol, best_nviol, feas_tol=0.0):
    """Per variable: (max admissible score over the WHOLE integer domain minus xbar,
    {value: dnviol} of every admissible maximiser); (None, {}) when no value is admissible.

    Only for instances whose variables are all binary or integer with small domains.
    """
    rows = normalised_rows(prob, feas_tol)
    xf = [F(float(v)) for v in x]
    out = []
    for j in range(prob.n):
        if prob.vtype[j] == CONT:
            raise ValueError("exhaustive enumeration needs integer domains")
        lo, hi = int(prob.lb[j]), int(prob.ub[j])
        xbar = xf[j]
        best, arg = None, {}
        for v in range(lo, hi + 1):
            if v == xbar:
                continue
            s, dc = score(rows, xf, w, j, v)
            if not admissible(v, xbar, j, dc, tabu_inc, tabu_dec, it, nviol, best_nviol):
                continue
            if best is None or s > best:
                best, arg = s, {v: dc}
            elif s == best:
                arg[v] = dc
        out.append((best, arg))
    return out


def candidate_values(prob, x, j, feas_tol=0.0):
    """Bounds and breakpoints of variable j (exact), the values Algorithm 1 scores.

    A cross-check of the oracle's candidate arithmetic, not an independent pin.
    """
    rows = normalised_rows(prob, feas_tol)
    xf = [F(float(v)) for v in x]
    c = set()
    if prob.vtype[j] == BIN:
        return {1 - xf[j]}
    for v in (prob.lb[j], prob.ub[j]):
        if math.isfinite(v):
            c.add(F(float(v)))
    for coeffs, b, eps in rows:
        if j not in coeffs:
            continue
        rest = activity({k: a for k, a in coeffs.items() if k != j}, xf)
        if prob.vtype[j] == INT:
            t = (b + eps - rest) / coeffs[j]
            t = F(math.floor(t)) if coeffs[j] > 0 else F(math.ceil(t))
        else:
            r = activity(coeffs, xf) - b
            if r <= eps and abs(r) <= eps:
                continue
            t = (b - rest) / coeffs[j]
        if F(float(prob.lb[j])) <= t <= F(float(prob.ub[j])):
            c.add(t)
    c.discard(xf[j])
    return c


def residual_state(prob, x, feas_tol=0.0):
    """(residuals, violated flags, nviol) of the normalised rows, exactly."""
    rows = normalised_rows(prob, feas_tol)
    xf = [F(float(v)) for v in x]
    r = [activity(c, xf) - b for c, b, _ in rows]
    viol = [ri > e for ri, (_, _, e) in zip(r, rows)]
    return r, viol, sum(viol)
