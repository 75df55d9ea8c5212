"""ctypes wrapper of the C oracle (chap_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg; the library under paper_2605_05086_gb300 never
imports it.  build() compiles the C file with gcc (OpenMP when available).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chap_oracle.c")
_LIB = os.path.join(_HERE, "libchap_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile chap_oracle.c into oracle/libchap_oracle.so (no fused multiply-add)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", _LIB, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", _LIB, "-lm"], check=True, capture_output=True)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    P = C.c_void_p
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, P, P, P, P, C.c_double]
    lib.orc_destroy.argtypes = [P]
    lib.orc_num_norm_rows.restype = C.c_int32
    lib.orc_num_norm_rows.argtypes = [P]
    lib.orc_norm_row_info.argtypes = [P, P, P, P, P]
    lib.orc_residuals.restype = C.c_int64
    lib.orc_residuals.argtypes = [P, P, P, P]
    lib.orc_best_shift.argtypes = [P, P, P, P, P, C.c_int64, C.c_int64, C.c_int64, P, C.c_int32,
                                   P, P, P, C.c_int32]
    lib.orc_max_threads.restype = C.c_int32
    lib.orc_run.restype = C.c_int64
    lib.orc_run.argtypes = [P, P, P, P, P, P, P, C.c_int32, C.c_int64, C.c_int32, P, P, P, P, C.c_int32]
    lib.orc_run_cutoff.restype = C.c_int64
    lib.orc_run_cutoff.argtypes = [P, P, P, P, P, P, P, C.c_int32, C.c_int64, C.c_int32, C.c_double,
                                   P, P, P, P, P, P, P, P, C.c_int32]
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """The oracle bound to one problem (arrays are kept alive by this object)."""

    def __init__(self, prob, feas_tol: float = 1e-9):
        lib = _load()
        self.prob = prob
        self._keep = [np.ascontiguousarray(a) for a in (
            prob.row_ptr.astype(np.int64), prob.col_idx.astype(np.int32), prob.row_val.astype(np.float64),
            prob.col_ptr.astype(np.int64), prob.row_idx.astype(np.int32),
            prob.lb.astype(np.float64), prob.ub.astype(np.float64), prob.rhs.astype(np.float64),
            prob.vtype.astype(np.uint8), prob.sense.astype(np.uint8))]
        k = self._keep
        self.h = lib.orc_create(prob.n, prob.m, _p(k[0]), _p(k[1]), _p(k[2]), _p(k[3]), _p(k[4]),
                                _p(k[5]), _p(k[6]), _p(k[7]), _p(k[8]), _p(k[9]), float(feas_tol))
        if not self.h:
            raise MemoryError("oracle allocation failed")
        self.n = prob.n
        self.mn = lib.orc_num_norm_rows(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_destroy(self.h)
            self.h = None

    def norm_rows(self):
        orig = np.zeros(self.mn, np.int32)
        sign = np.zeros(self.mn)
        rhs = np.zeros(self.mn)
        eps = np.zeros(self.mn)
        _load().orc_norm_row_info(self.h, _p(orig), _p(sign), _p(rhs), _p(eps))
        return orig, sign, rhs, eps

    def residuals(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        r = np.zeros(self.mn)
        v = np.zeros(self.mn, np.uint8)
        nv = _load().orc_residuals(self.h, _p(x), _p(r), _p(v))
        return r, v.astype(bool), int(nv)

    def best_shift(self, x, w, tabu_inc, tabu_dec, it, nviol, best_nviol, vars=None, nthreads=0):
        """Per-variable best shift: (xhat, s_half, dnviol) for `vars` (all when None)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.int32)
        ti = np.ascontiguousarray(tabu_inc, dtype=np.int64)
        td = np.ascontiguousarray(tabu_dec, dtype=np.int64)
        vv = None if vars is None else np.ascontiguousarray(vars, dtype=np.int32)
        cnt = self.n if vv is None else len(vv)
        xh = np.zeros(cnt)
        sh = np.zeros(cnt, np.int64)
        dc = np.zeros(cnt, np.int32)
        _load().orc_best_shift(self.h, _p(x), _p(w), _p(ti), _p(td), int(it), int(nviol), int(best_nviol),
                               _p(vv), 0 if vv is None else len(vv), _p(xh), _p(sh), _p(dc), int(nthreads))
        return xh, sh, dc

    def run(self, state, tenure, n_iters, stop_at_feasible=True, nthreads=0):
        """Run tabu iterations on a state dict (x, w, tabu_inc, tabu_dec, iter, best_nviol), in place.

        Returns a dict of per-iteration traces (var, val, s_half, nviol_after)."""
        x = state["x"]; w = state["w"]; ti = state["tabu_inc"]; td = state["tabu_dec"]
        it = C.c_int64(int(state["iter"]))
        bn = C.c_int64(int(state["best_nviol"]))
        mv = np.full(n_iters, -2, np.int32)
        mval = np.zeros(n_iters)
        ms = np.zeros(n_iters, np.int64)
        na = np.zeros(n_iters, np.int64)
        done = _load().orc_run(self.h, _p(x), _p(w), _p(ti), _p(td), C.addressof(it), C.addressof(bn),
                               int(tenure), int(n_iters), int(bool(stop_at_feasible)),
                               _p(mv), _p(mval), _p(ms), _p(na), int(nthreads))
        state["iter"] = it.value
        state["best_nviol"] = bn.value
        return dict(var=mv[:done], val=mval[:done], s_half=ms[:done], nviol_after=na[:done])

    def run_cutoff(self, state, tenure, n_iters, cut, nthreads=0):
        """`run` under the objective cutoff (Sec. 3.2).  `cut` is a dict with the
        cutoff row `row` and `delta`, updated in place: `obj`, `count`, `best_iter`
        and `x_best` of the best solution recorded, `rhs` the row's rhs after the
        run.  Never stops at feasibility."""
        x = state["x"]; w = state["w"]; ti = state["tabu_inc"]; td = state["tabu_dec"]
        it = C.c_int64(int(state["iter"]))
        bn = C.c_int64(int(state["best_nviol"]))
        obj = C.c_double(float(cut.get("obj", float("nan"))))
        cnt = C.c_int64(int(cut.get("count", 0)))
        bi = C.c_int64(int(cut.get("best_iter", -1)))
        if "x_best" not in cut:
            cut["x_best"] = np.zeros(self.n)
        xb = cut["x_best"]
        mv = np.full(n_iters, -2, np.int32)
        mval = np.zeros(n_iters)
        ms = np.zeros(n_iters, np.int64)
        na = np.zeros(n_iters, np.int64)
        done = _load().orc_run_cutoff(self.h, _p(x), _p(w), _p(ti), _p(td), C.addressof(it), C.addressof(bn),
                                      int(tenure), int(n_iters), int(cut["row"]), float(cut["delta"]),
                                      C.addressof(obj), C.addressof(cnt), C.addressof(bi), _p(xb),
                                      _p(mv), _p(mval), _p(ms), _p(na), int(nthreads))
        state["iter"] = it.value
        state["best_nviol"] = bn.value
        cut.update(obj=obj.value, count=cnt.value, best_iter=bi.value)
        orig, _, rhs, _ = self.norm_rows()
        cut["rhs"] = float(rhs[np.flatnonzero(orig == cut["row"])[0]])
        return dict(var=mv[:done], val=mval[:done], s_half=ms[:done], nviol_after=na[:done])

    def initial_state(self, x=None):
        x = np.array(self.prob.x0 if x is None else x, dtype=np.float64)
        _, _, nv = self.residuals(x)
        return dict(x=x, w=np.ones(self.mn, np.int32), tabu_inc=np.zeros(self.n, np.int64),
                    tabu_dec=np.zeros(self.n, np.int64), iter=0, best_nviol=nv)


def max_threads() -> int:
    return int(_load().orc_max_threads())
