import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2605_05086_gb300 import instances as inst  # noqa: E402


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
