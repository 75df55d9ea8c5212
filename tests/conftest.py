import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_05086_gb300 import instances as inst  # noqa: E402
from oracle import definition  # noqa: E402
from fractions import Fraction as F  # noqa: E402


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 GPU and the CUDA library")


def golden_cases():
    with open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")) as f:
        return json.load(f)["cases"]


def problem_from_case(case):
    """Problem from a golden case: rows are [[ [col, coef], ... ], sense, rhs]."""
    n = len(case["vtype"])
    rows, cols, vals, sense, rhs = [], [], [], [], []
    for i, (entries, s, b) in enumerate(case["rows"]):
        for j, a in entries:
            rows.append(i)
            cols.append(j)
            vals.append(float(a))
        sense.append(s)
        rhs.append(float(b))
    return inst.from_triplets(case["name"], n, len(case["rows"]), rows, cols, vals,
                              lb=case["lb"], ub=case["ub"], obj=np.ones(n), rhs=rhs,
                              vtype=case["vtype"], sense=sense, x0=case["x"])


@pytest.fixture(scope="session")
def setcover_small():
    return inst.gen_setcover(seed=0, n=2000, m=1000, k=8)


def fp_tiny(seed, tol):
    """Tiny MIP with N(0,1) rows (|a| >= 0.1) over continuous and integer
    variables, and a state in which some rows are satisfied within eps without
    being exactly tight: a continuous value is moved onto a row's tight point
    plus an offset of 0.3 eps / |a| (exact rationals, rounded once to double)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 6))
    vt = np.array([inst.VAR_CONT, inst.VAR_CONT] + [int(rng.choice([inst.VAR_INT, inst.VAR_CONT]))
                                                   for _ in range(n - 2)], dtype=np.uint8)
    lb = rng.integers(-3, 1, size=n).astype(float)
    ub = lb + rng.integers(2, 9, size=n)
    xs = np.where(vt == inst.VAR_CONT, lb + rng.random(n) * (ub - lb), np.floor(lb + rng.random(n) * (ub - lb + 1)))
    xs = np.minimum(xs, ub)
    m = int(rng.integers(4, 8))
    rows, cols, vals = [], [], []
    for i in range(m):
        for j in sorted(rng.choice(n, size=int(rng.integers(1, 4)), replace=False).tolist()):
            a = 0.0
            while abs(a) < 0.1:
                a = float(rng.normal())
            rows.append(i); cols.append(j); vals.append(a)
    ax = np.zeros(m)
    for r, c, v in zip(rows, cols, vals):
        ax[r] += v * xs[c]
    sense = rng.choice(np.array([0, 1, 2], dtype=np.uint8), size=m, p=[0.4, 0.4, 0.2])
    slack = np.where(rng.random(m) < 0.3, 0.0, rng.random(m))
    rhs = np.where(sense == 0, ax + slack, np.where(sense == 1, ax - slack, ax))
    prob = inst.from_triplets(f"fptiny_{seed}", n, m, rows, cols, vals, lb, ub, np.ones(n), rhs, vt, sense,
                              x0=np.clip(np.zeros(n), lb, ub))
    x = np.where(vt == inst.VAR_CONT, lb + rng.random(n) * (ub - lb), np.floor(lb + rng.random(n) * (ub - lb + 1)))
    x = np.minimum(x, ub)
    nrows = definition.normalised_rows(prob, tol)
    for _ in range(2):
        # a continuous value on a row's tight point, nudged by 0.3 eps / |a|
        k = int(rng.integers(0, len(nrows)))
        coeffs, b, eps = nrows[k]
        js = [j for j in coeffs if vt[j] == inst.VAR_CONT]
        if not js or eps == 0:
            continue
        j = js[0]
        xf = [F(float(v)) for v in x]
        rest = sum((a * xf[q] for q, a in coeffs.items() if q != j), F(0))
        t = (b - rest) / coeffs[j] + F(int(rng.choice([-1, 1]))) * F(3, 10) * eps / abs(coeffs[j])
        if F(float(lb[j])) <= t <= F(float(ub[j])):
            x[j] = float(t)
    return prob, x
