"""The C-ABI library builds, loads and exports every entry point of include/chap.h,
and its host-side validation rejects malformed problems before any device call
(these tests run without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2605_05086_gb300 import build, chap
from paper_2605_05086_gb300 import instances as inst


def declared_symbols():
    with open(os.path.join(ROOT, "include", "chap.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"CHAP_API\s+[\w\s\*]+?\b(chap_\w+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = C.CDLL(build.LIB)
    names = declared_symbols()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(chap.EXPORTED)


def test_status_strings_and_defaults():
    lib = chap.load()
    assert lib.chap_status_str(chap.CHAP_E_INVALID) == b"invalid argument"
    o = chap.chap_options_default()
    assert o.feas_tol == 1e-9 and o.tenure == 10 and o.graph_iters == 64 and o.stop_at_feasible == 1


def _bad(prob, **changes):
    import copy
    p = copy.deepcopy(prob)
    for k, v in changes.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("case", ["unsorted_row", "csc_mismatch", "nan", "zero_coef", "l_gt_u",
                                  "binary_bounds", "fractional_int_bound", "bad_sense", "row_ptr_end"])
def test_create_rejects_invalid_problems(case):
    prob = inst.gen_tiny_mixed(3, n=6, m=5, max_len=4)
    if case == "unsorted_row":
        i = int(np.argmax(np.diff(prob.row_ptr) >= 2))
        ci = prob.col_idx.copy()
        a, b = prob.row_ptr[i], prob.row_ptr[i] + 1
        ci[a], ci[b] = ci[b], ci[a]
        p = _bad(prob, col_idx=ci)
    elif case == "csc_mismatch":
        cv = prob.col_val.copy(); cv[0] += 1.0
        p = _bad(prob, col_val=cv)
    elif case == "nan":
        rv = prob.row_val.copy(); rv[0] = np.nan
        p = _bad(prob, row_val=rv)
    elif case == "zero_coef":
        rv = prob.row_val.copy(); rv[0] = 0.0
        cv = prob.col_val.copy()
        cv[np.nonzero((prob.row_idx == 0))[0][0]] = 0.0
        p = _bad(prob, row_val=rv, col_val=cv)
    elif case == "l_gt_u":
        lb = prob.lb.copy(); lb[0] = prob.ub[0] + 1
        p = _bad(prob, lb=lb)
    elif case == "binary_bounds":
        vt = prob.vtype.copy(); vt[:] = inst.VAR_BIN
        ub = prob.ub.copy(); ub[:] = 2.0
        p = _bad(prob, vtype=vt, ub=ub)
    elif case == "fractional_int_bound":
        vt = prob.vtype.copy(); vt[0] = inst.VAR_INT
        ub = prob.ub.copy(); ub[0] = prob.lb[0] + 2.5
        p = _bad(prob, vtype=vt, ub=ub)
    elif case == "bad_sense":
        s = prob.sense.copy(); s[0] = 7
        p = _bad(prob, sense=s)
    else:
        rp = prob.row_ptr.copy(); rp[-1] += 1
        p = _bad(prob, row_ptr=rp)
    with pytest.raises(chap.ChapError) as e:
        chap.chap_bs_create(p)
    assert e.value.status == chap.CHAP_E_INVALID


def test_python_binding_has_no_cpu_path():
    """The binding only marshals arguments: no oracle import, no numpy scoring."""
    src = open(os.path.join(ROOT, "paper_2605_05086_gb300", "chap.py")).read()
    assert "oracle" not in src.replace("no oracle", "")
