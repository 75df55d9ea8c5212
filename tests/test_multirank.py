"""The N > 1 bench path (independent replicas, weak scaling): two gloo ranks on
the CPU check the whole-job reduction (slowest rank's time, summed moves) and
that the reference arm's non-zero ranks exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, mv = bench.reduce_over_ranks([1.0, 2.5][rank], [10, 20][rank], "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, mv))


def test_replica_reduction_two_ranks():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2.5, 30), (1, 2.5, 30)]


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_json_line():
    """The reference arm (the oracle timed on the host) prints one JSON line with
    the contract's keys, on the small set-cover workload."""
    import json
    import time
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    t0 = time.perf_counter()
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "setcover_2k", "--steps", "2", "--warmup", "1"], env=env, capture_output=True, text=True,
                       timeout=300)
    wall = time.perf_counter() - t0
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # ms_per_step is measured, not extrapolated: the timed steps fit in the run
    assert d["steps"] * d["ms_per_step"] * 1e-3 <= wall
    assert d["extrapolation"]["vars_per_step"] >= 16 * 16 * d["cpu_baseline"]["cores"] or \
        d["extrapolation"]["vars_per_step"] == d["config"]["n"]


def _record_worker(rank, world, port, q):
    import ctypes
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2605_05086_gb300 import chap
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rec = chap.chap_move_record(score_half=10 * (rank + 1), var=100 + rank, dnviol=-rank, new_value=0.5 * rank,
                                old_value=1.0)
    local = torch.frombuffer(bytearray(ctypes.string_at(ctypes.addressof(rec), ctypes.sizeof(rec))),
                             dtype=torch.uint8)
    out = chap.exchange_records(local, world)
    got = []
    for r in range(world):
        b = bytes(out[r * chap.MOVE_RECORD_BYTES:(r + 1) * chap.MOVE_RECORD_BYTES].numpy())
        x = chap.chap_move_record.from_buffer_copy(b)
        got.append((x.score_half, x.var, x.dnviol, x.new_value, x.old_value))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_move_record_exchange_two_gloo_ranks():
    """The column-sharded search's exchange step: every rank receives every
    rank's 32-byte move record, in rank order, with the fields intact (the
    layout of chap_move_record)."""
    mp = pytest.importorskip("torch.multiprocessing")
    sys.path.insert(0, ROOT)
    from paper_2605_05086_gb300 import chap
    import ctypes
    assert ctypes.sizeof(chap.chap_move_record) == chap.MOVE_RECORD_BYTES == 32
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_record_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [(10, 100, 0, 0.0, 1.0), (20, 101, -1, 0.5, 1.0)]
    assert out == [(0, want), (1, want)]
