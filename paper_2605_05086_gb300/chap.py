"""Python binding of libchap.so (include/chap.h): argument marshalling only.

Every step of the best-shift tabu search runs in the library's CUDA kernels;
this module converts numpy arrays / torch CUDA tensors to pointers and status
codes to exceptions.  There is no CPU fallback: when the library is missing or
no GPU is present, loading fails with an exception.

Function names follow the C ABI (chap_bs_create, chap_bs_best_shift,
chap_bs_apply, chap_tabu_run, ...); the BestShift class is a thin handle wrapper.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

CHAP_OK, CHAP_E_INVALID, CHAP_E_OOM, CHAP_E_CUDA, CHAP_E_TIMEOUT, CHAP_E_STATE, CHAP_E_UNSUPPORTED = range(7)
CHAP_MEM_HOST, CHAP_MEM_DEVICE = 0, 1

EXPORTED = [
    "chap_options_default", "chap_bs_create", "chap_bs_destroy", "chap_bs_info", "chap_bs_set_state",
    "chap_bs_set_checkpoint", "chap_bs_get_state", "chap_bs_residuals", "chap_bs_best_shift",
    "chap_bs_apply", "chap_bs_step", "chap_tabu_run", "chap_status_str", "chap_last_error",
    "chap_bs_profile", "chap_bs_kernel_ms", "chap_bs_best_shift_static_scratch",
    "chap_batch_create", "chap_batch_destroy", "chap_batch_run", "chap_batch_autotune", "chap_batch_set_schedule",
    "chap_batch_reset", "chap_batch_get_x", "chap_batch_last_error",
    "chap_bs_refresh_features", "chap_bs_features", "chap_bs_propose", "chap_learned_run", "chap_mlp_forward",
    "chap_mlp_loss_grad", "chap_mlp_adam", "chap_bs_set_cutoff", "chap_bs_get_cutoff",
    "chap_bs_move_record", "chap_bs_apply_records", "chap_batch_set_persistent", "chap_batch_autotune_mode",
]


class ChapError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class chap_problem(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("row_val", C.c_void_p),
                ("col_ptr", C.c_void_p), ("row_idx", C.c_void_p), ("col_val", C.c_void_p),
                ("lb", C.c_void_p), ("ub", C.c_void_p), ("obj", C.c_void_p), ("rhs", C.c_void_p),
                ("vtype", C.c_void_p), ("sense", C.c_void_p)]


class chap_options(C.Structure):
    _fields_ = [("feas_tol", C.c_double), ("tenure", C.c_int32), ("graph_iters", C.c_int32),
                ("max_iters", C.c_int64), ("stop_at_feasible", C.c_int32), ("lazy_binary", C.c_int32),
                ("static_scratch_only", C.c_int32), ("shard_rank", C.c_int32), ("shard_count", C.c_int32),
                ("bin_kernel", C.c_int32), ("bin_block_rows", C.c_int32), ("reserved", C.c_int32)]


class chap_move(C.Structure):
    _fields_ = [("var", C.c_int32), ("dnviol", C.c_int32), ("score_half", C.c_int64),
                ("old_value", C.c_double), ("new_value", C.c_double)]


class chap_move_record(C.Structure):
    _fields_ = [("score_half", C.c_int64), ("var", C.c_int32), ("dnviol", C.c_int32),
                ("new_value", C.c_double), ("old_value", C.c_double)]


MOVE_RECORD_BYTES = 32


class chap_tabu_result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("moves", C.c_int64), ("feasible_iter", C.c_int64),
                ("final_nviol", C.c_int64), ("best_nviol", C.c_int64), ("seconds", C.c_double),
                ("time_to_feasible_s", C.c_double), ("objective", C.c_double)]


class chap_cutoff_info(C.Structure):
    _fields_ = [("solutions", C.c_int64), ("best_iter", C.c_int64), ("best_objective", C.c_double),
                ("rhs", C.c_double), ("row", C.c_int32), ("reserved", C.c_int32)]


class chap_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("m_norm", C.c_int32),
                ("n_bin", C.c_int32), ("n_int", C.c_int32), ("n_cont", C.c_int32), ("n_fixed", C.c_int32),
                ("nnz", C.c_int64), ("nnz_int_rows", C.c_int64), ("nnz_fp_rows", C.c_int64),
                ("bytes_per_pass", C.c_int64), ("eval_blocks", C.c_int32), ("n_hist_cols", C.c_int32),
                ("launches_per_step", C.c_int32), ("grid_bin", C.c_int32), ("grid_nb", C.c_int32),
                ("bytes_bin", C.c_int64), ("bytes_nb", C.c_int64), ("bytes_cta", C.c_int64),
                ("bytes_hist", C.c_int64), ("bin_lanes", C.c_int32), ("nb_lanes", C.c_int32),
                ("n_long_cols", C.c_int32), ("n_cta_cols", C.c_int32), ("bin_rows", C.c_int32),
                ("bin_row_blocks", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libchap.so (building it first when missing).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"{_build.LIB} is missing; build it with paper_2605_05086_gb300.build.build()")
        _build.build()
    lib = C.CDLL(_build.LIB)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "chap_options_default": (None, [P]),
        "chap_bs_create": (I32, [P, P, P, P]),
        "chap_bs_destroy": (I32, [P]),
        "chap_bs_info": (I32, [P, P]),
        "chap_bs_set_state": (I32, [P, P, P, I32]),
        "chap_bs_set_checkpoint": (I32, [P, P, P, P, P, I64, I64]),
        "chap_bs_get_state": (I32, [P, P, P, P, P, P, I32]),
        "chap_bs_residuals": (I32, [P, P, I32]),
        "chap_bs_best_shift": (I32, [P, P, P, P, P, I32]),
        "chap_bs_apply": (I32, [P, I32, D]),
        "chap_bs_step": (I32, [P, P]),
        "chap_tabu_run": (I32, [P, P, P]),
        "chap_status_str": (C.c_char_p, [I32]),
        "chap_last_error": (C.c_char_p, [P]),
        "chap_bs_profile": (I32, [P, I32]),
        "chap_bs_kernel_ms": (I32, [P, P]),
        "chap_bs_best_shift_static_scratch": (I32, [P, P, P, P, P, I32]),
        "chap_batch_create": (I32, [P, I32, P, P, I32, P, P]),
        "chap_batch_destroy": (I32, [P]),
        "chap_batch_run": (I32, [P, I64, I32, I32, P, P]),
        "chap_batch_autotune": (I32, [P, I32, P]),
        "chap_batch_set_schedule": (I32, [P, I32, I32]),
        "chap_batch_set_persistent": (I32, [P, I32, I64]),
        "chap_batch_autotune_mode": (I32, [P, I32, I32, P]),
        "chap_batch_reset": (I32, [P]),
        "chap_batch_get_x": (I32, [P, I32, P]),
        "chap_batch_last_error": (C.c_char_p, [P]),
        "chap_bs_refresh_features": (I32, [P]),
        "chap_bs_features": (I32, [P, P, P]),
        "chap_bs_propose": (I32, [P, P, I32, P, P]),
        "chap_learned_run": (I32, [P, P, P, P]),
        "chap_mlp_forward": (I32, [P, P, I64, P, P]),
        "chap_mlp_loss_grad": (I32, [P, P, P, I64, P, P, P]),
        "chap_mlp_adam": (I32, [P, P, P, P, P, I32, C.c_float, P]),
        "chap_bs_set_cutoff": (I32, [P, I32, D]),
        "chap_bs_move_record": (I32, [P, P, I32]),
        "chap_bs_apply_records": (I32, [P, P, I32, I32]),
        "chap_bs_get_cutoff": (I32, [P, P, P, I32]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _check(h, status):
    if status != CHAP_OK:
        lib = load()
        msg = lib.chap_last_error(h).decode() if h else lib.chap_status_str(status).decode()
        raise ChapError(status, msg or lib.chap_status_str(status).decode())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def chap_options_default() -> chap_options:
    o = chap_options()
    load().chap_options_default(C.byref(o))
    return o


def chap_bs_create(prob, opts: chap_options | None = None, stream=None):
    """Create a handle over a Problem (instances.Problem-like, host numpy arrays)."""
    lib = load()
    keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
        (prob.row_ptr, np.int64), (prob.col_idx, np.int32), (prob.row_val, np.float64),
        (prob.col_ptr, np.int64), (prob.row_idx, np.int32), (prob.col_val, np.float64),
        (prob.lb, np.float64), (prob.ub, np.float64), (prob.obj, np.float64), (prob.rhs, np.float64),
        (prob.vtype, np.uint8), (prob.sense, np.uint8))]
    p = chap_problem(prob.n, prob.m, int(prob.row_ptr[-1]), *[_ptr(a) for a in keep])
    h = C.c_void_p()
    st = lib.chap_bs_create(C.byref(p), None if opts is None else C.byref(opts), _stream(stream), C.byref(h))
    if st != CHAP_OK:
        raise ChapError(st, "chap_bs_create: " + lib.chap_status_str(st).decode())
    return h


def chap_bs_destroy(h):
    _check(None, load().chap_bs_destroy(h))


def chap_bs_info(h) -> chap_info:
    inf = chap_info()
    _check(h, load().chap_bs_info(h, C.byref(inf)))
    return inf


def chap_bs_set_state(h, x=None, w=None, mem=CHAP_MEM_HOST):
    if mem == CHAP_MEM_HOST:
        x = None if x is None else np.ascontiguousarray(x, dtype=np.float64)
        w = None if w is None else np.ascontiguousarray(w, dtype=np.int32)
    _check(h, load().chap_bs_set_state(h, _ptr(x), _ptr(w), mem))


def chap_bs_set_checkpoint(h, x, w, tabu_inc, tabu_dec, it, best_nviol):
    arrs = [np.ascontiguousarray(x, np.float64), np.ascontiguousarray(w, np.int32),
            np.ascontiguousarray(tabu_inc, np.int64), np.ascontiguousarray(tabu_dec, np.int64)]
    _check(h, load().chap_bs_set_checkpoint(h, *[_ptr(a) for a in arrs], int(it), int(best_nviol)))


def chap_bs_get_state(h, n, m_norm):
    """Host copies of x, w, tabu stamps and the scalars (iter, nviol, best_nviol,
    feasible_iter, moves, weight_updates)."""
    x = np.zeros(n)
    w = np.zeros(m_norm, np.int32)
    ti = np.zeros(n, np.int64)
    td = np.zeros(n, np.int64)
    sc = np.zeros(6, np.int64)
    _check(h, load().chap_bs_get_state(h, _ptr(x), _ptr(w), _ptr(ti), _ptr(td), _ptr(sc), CHAP_MEM_HOST))
    return dict(x=x, w=w, tabu_inc=ti, tabu_dec=td, iter=int(sc[0]), nviol=int(sc[1]),
                best_nviol=int(sc[2]), feasible_iter=int(sc[3]), moves=int(sc[4]), weight_updates=int(sc[5]))


def chap_bs_profile(h, enable=True):
    _check(h, load().chap_bs_profile(h, 1 if enable else 0))


def chap_bs_kernel_ms(h):
    """Durations (ms) of the kernels of the last profiled pass: binary flips,
    short columns, CTA sort, counting sort, selection."""
    ms = np.zeros(5, np.float32)
    _check(h, load().chap_bs_kernel_ms(h, _ptr(ms)))
    return ms


def chap_bs_residuals(h, m_norm, out=None, mem=CHAP_MEM_HOST):
    r = np.zeros(m_norm) if out is None else out
    _check(h, load().chap_bs_residuals(h, _ptr(r), mem))
    return r


def chap_bs_best_shift(h, n=None, xhat=None, score_half=None, dnviol=None, mem=CHAP_MEM_HOST, want_vars=True):
    """Best-shift pass.  With mem=HOST and want_vars, returns numpy (xhat, score_half, dnviol, move)."""
    if mem == CHAP_MEM_HOST and want_vars and xhat is None:
        xhat = np.zeros(n)
        score_half = np.zeros(n, np.int64)
        dnviol = np.zeros(n, np.int32)
    mv = chap_move()
    _check(h, load().chap_bs_best_shift(h, _ptr(xhat), _ptr(score_half), _ptr(dnviol), C.byref(mv), mem))
    return xhat, score_half, dnviol, mv


def chap_bs_best_shift_static_scratch(h, n=None, xhat=None, score_half=None, dnviol=None, mem=CHAP_MEM_HOST,
                                      want_vars=True):
    """chap_bs_best_shift with the counting-sort columns on the library's fixed scratch."""
    if mem == CHAP_MEM_HOST and want_vars and xhat is None:
        xhat = np.zeros(n)
        score_half = np.zeros(n, np.int64)
        dnviol = np.zeros(n, np.int32)
    mv = chap_move()
    _check(h, load().chap_bs_best_shift_static_scratch(h, _ptr(xhat), _ptr(score_half), _ptr(dnviol),
                                                       C.byref(mv), mem))
    return xhat, score_half, dnviol, mv


def chap_bs_apply(h, var, new_value):
    _check(h, load().chap_bs_apply(h, int(var), float(new_value)))


def chap_bs_step(h, want_move=True):
    mv = chap_move()
    _check(h, load().chap_bs_step(h, C.byref(mv) if want_move else None))
    return mv


def chap_tabu_run(h, opts: chap_options | None = None) -> chap_tabu_result:
    res = chap_tabu_result()
    _check(h, load().chap_tabu_run(h, None if opts is None else C.byref(opts), C.byref(res)))
    return res


def chap_bs_set_cutoff(h, row, delta=1.0):
    _check(h, load().chap_bs_set_cutoff(h, int(row), float(delta)))


def chap_bs_get_cutoff(h, n):
    """(chap_cutoff_info, x_best as a host array)."""
    info = chap_cutoff_info()
    xb = np.zeros(n)
    _check(h, load().chap_bs_get_cutoff(h, C.byref(info), _ptr(xb), CHAP_MEM_HOST))
    return info, xb


class BestShift:
    """Handle wrapper: BestShift(problem, tenure=10, feas_tol=1e-9, ...)."""

    def __init__(self, prob, stream=None, **opts):
        o = chap_options_default()
        for k, v in opts.items():
            setattr(o, k, v)
        self.opts = o
        self.h = chap_bs_create(prob, o, stream)
        self.info = chap_bs_info(self.h)
        self.n, self.m_norm = prob.n, self.info.m_norm

    def close(self):
        if getattr(self, "h", None):
            chap_bs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, x=None, w=None, mem=CHAP_MEM_HOST):
        chap_bs_set_state(self.h, x, w, mem)

    def set_checkpoint(self, st):
        chap_bs_set_checkpoint(self.h, st["x"], st["w"], st["tabu_inc"], st["tabu_dec"], st["iter"], st["best_nviol"])

    def state(self):
        return chap_bs_get_state(self.h, self.n, self.m_norm)

    def residuals(self):
        return chap_bs_residuals(self.h, self.m_norm)

    def best_shift(self):
        return chap_bs_best_shift(self.h, self.n)

    def apply(self, var, value):
        chap_bs_apply(self.h, var, value)

    def step(self):
        return chap_bs_step(self.h)

    def set_cutoff(self, row, delta=1.0):
        """Objective cutoff on `row` (-1: off); see chap_bs_set_cutoff."""
        chap_bs_set_cutoff(self.h, row, delta)

    def cutoff(self):
        return chap_bs_get_cutoff(self.h, self.n)

    def run(self, **kw):
        o = chap_options()
        C.memmove(C.byref(o), C.byref(self.opts), C.sizeof(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return chap_tabu_run(self.h, o)


def chap_bs_move_record(h, rec=None, mem=CHAP_MEM_HOST):
    """The move of the handle's last pass: a chap_move_record (host), or written
    into `rec` (a device buffer of 32 bytes, e.g. a torch uint8 tensor) when
    mem=CHAP_MEM_DEVICE."""
    if mem == CHAP_MEM_HOST:
        r = chap_move_record()
        _check(h, load().chap_bs_move_record(h, C.byref(r), mem))
        return r
    _check(h, load().chap_bs_move_record(h, _ptr(rec), mem))
    return rec


def chap_bs_apply_records(h, recs, k=None, mem=CHAP_MEM_HOST):
    """Apply the winner of k move records: a ctypes array of chap_move_record
    (host) or a device buffer of k * 32 bytes (mem=CHAP_MEM_DEVICE)."""
    if mem == CHAP_MEM_HOST:
        k = len(recs) if k is None else k
        _check(h, load().chap_bs_apply_records(h, recs, int(k), mem))
    else:
        _check(h, load().chap_bs_apply_records(h, _ptr(recs), int(k), mem))


def exchange_records(local, world, group=None):
    """All-gather of the ranks' 32-byte move records: returns the world's
    records in rank order as one uint8 tensor of world * 32 bytes on local's
    device (NCCL for CUDA tensors; gloo takes host tensors)."""
    import torch
    import torch.distributed as dist
    out = torch.empty(world * MOVE_RECORD_BYTES, dtype=torch.uint8, device=local.device)
    parts = list(out.split(MOVE_RECORD_BYTES))
    dist.all_gather(parts, local.contiguous(), group=group)
    return out


class ShardedSearch:
    """One rank of the column-sharded tabu search: a handle that evaluates every
    world-th column, and the exchange of the 32-byte move records.

    exchange(local) must return the world's records in rank order as a device
    uint8 tensor of world * 32 bytes (an all-gather: NCCL across GPUs); the
    default is exchange_records on the current process group.  Every rank then
    applies the same winning move."""

    def __init__(self, prob, rank, world, stream=None, exchange=None, **opts):
        import torch
        self.bs = BestShift(prob, stream=stream, shard_rank=int(rank), shard_count=int(world), **opts)
        self.rank, self.world = int(rank), int(world)
        self.rec = torch.zeros(MOVE_RECORD_BYTES, dtype=torch.uint8, device="cuda")
        self.exchange = exchange or (lambda local: exchange_records(local, self.world))

    def pass_record(self):
        """The shard's pass and its move record (device)."""
        lib = load()
        _check(self.bs.h, lib.chap_bs_best_shift(self.bs.h, None, None, None, None, CHAP_MEM_DEVICE))
        chap_bs_move_record(self.bs.h, self.rec, CHAP_MEM_DEVICE)
        return self.rec

    def apply(self, records):
        chap_bs_apply_records(self.bs.h, records, self.world, CHAP_MEM_DEVICE)

    def step(self):
        self.apply(self.exchange(self.pass_record()))

    def close(self):
        self.bs.close()


class chap_chain_result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("moves", C.c_int64), ("feasible_iter", C.c_int64),
                ("final_nviol", C.c_int64), ("best_nviol", C.c_int64), ("time_to_feasible_s", C.c_double)]


class BatchChains:
    """Independent tabu chains over several all-binary integral instances (chap_batch_*)."""

    def __init__(self, probs, chain_prob, chain_tenure, stream=None):
        lib = load()
        self._keep = []
        arr = (chap_problem * len(probs))()
        for k, prob in enumerate(probs):
            keep = [np.ascontiguousarray(a, dtype=t) for a, t in (
                (prob.row_ptr, np.int64), (prob.col_idx, np.int32), (prob.row_val, np.float64),
                (prob.col_ptr, np.int64), (prob.row_idx, np.int32), (prob.col_val, np.float64),
                (prob.lb, np.float64), (prob.ub, np.float64), (prob.obj, np.float64), (prob.rhs, np.float64),
                (prob.vtype, np.uint8), (prob.sense, np.uint8))]
            self._keep.append(keep)
            arr[k] = chap_problem(prob.n, prob.m, int(prob.row_ptr[-1]), *[_ptr(a) for a in keep])
        self.chain_prob = np.ascontiguousarray(chain_prob, np.int32)
        self.chain_tenure = np.ascontiguousarray(chain_tenure, np.int32)
        self.n_chains = len(self.chain_prob)
        self.n_of = [p.n for p in probs]
        self.h = C.c_void_p()
        st = lib.chap_batch_create(arr, len(probs), _ptr(self.chain_prob), _ptr(self.chain_tenure), self.n_chains,
                                   _stream(stream), C.byref(self.h))
        if st != CHAP_OK:
            raise ChapError(st, "chap_batch_create: " + lib.chap_status_str(st).decode())

    def _check(self, st):
        if st != CHAP_OK:
            lib = load()
            raise ChapError(st, lib.chap_batch_last_error(self.h).decode() or lib.chap_status_str(st).decode())

    def run(self, max_iters, stop_at_feasible=True, graph_iters=64):
        res = (chap_chain_result * self.n_chains)()
        secs = C.c_double()
        self._check(load().chap_batch_run(self.h, int(max_iters), 1 if stop_at_feasible else 0, int(graph_iters),
                                          res, C.byref(secs)))
        return list(res), secs.value

    def autotune(self, iters=5, mode=-1):
        """(lanes per column, CTAs per SM, persistent) of the fastest schedule
        (mode 0: three launches per iteration only, 1: persistent only)."""
        ch = np.zeros(3, np.int32)
        self._check(load().chap_batch_autotune_mode(self.h, int(iters), int(mode), _ptr(ch)))
        return int(ch[0]), int(ch[1]), int(ch[2])

    def set_persistent(self, on=True, barrier_limit_ns=0):
        self._check(load().chap_batch_set_persistent(self.h, 1 if on else 0, int(barrier_limit_ns)))

    def set_schedule(self, lanes_per_column, ctas_per_sm):
        self._check(load().chap_batch_set_schedule(self.h, int(lanes_per_column), int(ctas_per_sm)))

    def reset(self):
        self._check(load().chap_batch_reset(self.h))

    def x(self, chain):
        out = np.zeros(self.n_of[self.chain_prob[chain]])
        self._check(load().chap_batch_get_x(self.h, int(chain), _ptr(out)))
        return out

    def close(self):
        if self.h:
            load().chap_batch_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 5057


class chap_learned_options(C.Structure):
    _fields_ = [("topk", C.c_int32), ("exact_every", C.c_int32), ("propose_every", C.c_int32),
                ("stop_at_feasible", C.c_int32), ("max_iters", C.c_int64)]


class chap_learned_result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("moves", C.c_int64), ("feasible_iter", C.c_int64),
                ("final_nviol", C.c_int64), ("best_nviol", C.c_int64), ("exact_passes", C.c_int64),
                ("misses", C.c_int64), ("seconds", C.c_double), ("time_to_feasible_s", C.c_double)]


def _dptr(t):
    """Device pointer of a torch tensor (None passes NULL)."""
    return None if t is None else C.c_void_p(t.data_ptr())


def chap_bs_refresh_features(h):
    _check(h, load().chap_bs_refresh_features(h))


def chap_bs_features(h, feat=None, target=None):
    """feat: torch int16 [n, 12] (BF16 bits), target: torch float32 [n] (device)."""
    _check(h, load().chap_bs_features(h, _dptr(feat), _dptr(target)))


def chap_bs_propose(h, weights, k, lst=None, pred=None):
    _check(h, load().chap_bs_propose(h, _dptr(weights), int(k), _dptr(lst), _dptr(pred)))


def chap_learned_run(h, weights, topk=4096, exact_every=50, propose_every=1, max_iters=1000, stop_at_feasible=True):
    lo = chap_learned_options(int(topk), int(exact_every), int(propose_every), 1 if stop_at_feasible else 0,
                              int(max_iters))
    res = chap_learned_result()
    _check(h, load().chap_learned_run(h, _dptr(weights), C.byref(lo), C.byref(res)))
    return res


def _stream_of(stream):
    return _stream(stream)


def chap_mlp_forward(weights, x, y, stream=None):
    st = load().chap_mlp_forward(_dptr(weights), _dptr(x), int(x.shape[0]), _dptr(y), _stream(stream))
    if st != CHAP_OK:
        raise ChapError(st, "chap_mlp_forward")


def chap_mlp_loss_grad(weights, x, target, grad, loss, stream=None):
    st = load().chap_mlp_loss_grad(_dptr(weights), _dptr(x), _dptr(target), int(x.shape[0]), _dptr(grad),
                                   _dptr(loss), _stream(stream))
    if st != CHAP_OK:
        raise ChapError(st, "chap_mlp_loss_grad")


def chap_mlp_adam(w32, wbf, m, v, grad, step, lr, stream=None):
    st = load().chap_mlp_adam(_dptr(w32), _dptr(wbf), _dptr(m), _dptr(v), _dptr(grad), int(step), float(lr),
                              _stream(stream))
    if st != CHAP_OK:
        raise ChapError(st, "chap_mlp_adam")
