"""The multi-rank path of bench.py on the CPU: two gloo ranks on 127.0.0.1 (the GPU machine
runs one rank per GPU over NCCL, replicas only).  Each rank transforms its own synthetic
batch (disjoint seeds, weak scaling) and the step time is the maximum over ranks."""

import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    try:
        import bench
        from synth.signals import device_signal
        r, w, local, dist = bench.init_ranks("gloo")
        t = bench.max_over_ranks(1.0 + 2.5 * r, dist, "cpu")
        _, f, _ = device_signal(2**12, 8, bench.rank_seed0(r), None, "cpu")
        dist.barrier()
        dist.destroy_process_group()
        q.put((r, w, local, t, bench.rank_seed0(r), f.tolist()))
    except Exception as e:  # report instead of hanging the parent
        q.put(("error", rank, repr(e)))


def test_two_gloo_ranks_max_time_and_disjoint_batches():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
    assert not any(r[0] == "error" for r in res), res
    res.sort()
    (r0, w0, l0, t0, s0, f0), (r1, w1, l1, t1, s1, f1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2 and (l0, l1) == (0, 1)
    assert t0 == t1 == 3.5                      # max over ranks
    assert s0 != s1 and f0 != f1                # replicas transform different signals
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    sys.path.insert(0, ROOT)
    import bench
    r, w, local, dist = bench.init_ranks("gloo")
    assert (r, w, local, dist) == (0, 1, 0, None)
    assert bench.max_over_ranks(2.0, None, "cpu") == 2.0


def test_reference_arm_other_ranks_do_no_work(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        steps, warmup, snr = 1, 3, 20.0
    assert bench.reference_arm(Args(), 1, 2) is None
    assert capsys.readouterr().out == ""
