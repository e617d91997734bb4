"""Asynchronous batched executes (sfft4_execute_batched_async / sfft4_wait), on a GB300.

Consecutive asynchronous calls use the plan's workspaces in turn (two for a uniform batch,
three for a batch of uneven signals) on the plan's own streams, so batch k's decode chain
overlaps batch k+1's gather.  Every batch must give,
bit for bit, the results of a synchronous execute of the same batch (same kernels, same
reduction orders), whatever the interleaving: four batches in flight through two
workspaces, a synchronous execute issued behind asynchronous ones, CUDA-graph replay, and
inputs rewritten after wait().  Noiseless batches must also match the FP64 oracle.
"""

import numpy as np
import pytest

from oracle import plan as OP, sfft4 as O
from synth import sparse_signal

pytestmark = pytest.mark.gpu

N, K, L_, Q_ = 2**18, 100, 16, 1.0


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def batch(seeds, snr):
    import torch
    return torch.from_numpy(np.stack([sparse_signal(N, K, s, snr).x for s in seeds])).to("cuda")


def host(out):
    return tuple(t.cpu().numpy() for t in out)


def same(a, b):
    return all(np.array_equal(u, v) for u, v in zip(a, b))


@pytest.mark.parametrize("graph", [False, True])
def test_async_batches_equal_synchronous(s4, graph):
    import torch
    xs = [batch(range(6 * k, 6 * k + 6), 20.0) for k in range(4)]
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=6, precision="bf16x3", graph=graph)
    want = [host(p.execute_batched(x)) for x in xs]
    outs = [p._outputs(6) for _ in xs]
    for x, o in zip(xs, outs):
        p.execute_batched(x, o, asynchronous=True)
    p.wait()
    torch.cuda.synchronize()
    for w, o in zip(want, outs):
        assert same(w, host(o))
    st = p.stats()
    assert st["executes"] == 8 and st["transforms"] == 48
    p.sync_status()
    p.close()


def test_sync_execute_behind_async(s4):
    """A synchronous execute on the plan's own workspace waits for the asynchronous one."""
    import torch
    xa, xb = batch(range(3), 20.0), batch(range(10, 13), 20.0)
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=3, precision="bf16x3")
    wa, wb = host(p.execute_batched(xa)), host(p.execute_batched(xb))
    oa = p._outputs(3)
    p.execute_batched(xa, oa, asynchronous=True)   # workspace 0
    ob = host(p.execute_batched(xb))               # synchronous, workspace 0 again
    p.wait()
    torch.cuda.synchronize()
    assert same(wa, host(oa))
    assert same(wb, ob)
    p.close()


def test_async_inputs_rewritten_after_wait(s4):
    import torch
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=4, precision="fp32")
    x = batch(range(4), None)
    o1, o2 = p._outputs(4), p._outputs(4)
    p.execute_batched(x, o1, asynchronous=True)
    p.wait()
    x.copy_(batch(range(20, 24), None))
    p.execute_batched(x, o2, asynchronous=True)
    p.wait()
    torch.cuda.synchronize()
    op = OP.make_plan(N, K, L_, Q_, seed=5)
    for o, seeds in ((o1, range(4)), (o2, range(20, 24))):
        idx, val, nf, _ = host(o)
        for i, sd in enumerate(seeds):
            sig = sparse_signal(N, K, sd, None)
            r = O.run(sig.x.astype(np.complex128), op, signal=i)
            n = int(nf[i])
            assert np.array_equal(idx[i, :n], r["f"])
            assert np.array_equal(idx[i, :n], sig.freqs)
            assert np.linalg.norm(val[i, :n] - r["v"]) <= 1e-5 * np.linalg.norm(r["v"])
    p.close()


def test_async_rejects_trace_plans(s4):
    from paper_2011_05698_gb300 import Sfft4Error
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=2, trace=True)
    with pytest.raises(Sfft4Error):
        p.execute_batched(batch(range(2), None), asynchronous=True)
    p.close()


def test_uneven_batch_async_equals_synchronous(s4):
    """Batches of signals of different N and K (sfft4_execute_batched_v_async): three batches
    of different contents in flight through three workspaces, each bit-identical to a
    synchronous execute, with and without graph replay."""
    import torch
    from synth.signals import device_signal
    sizes = [(2**14, 16), (2**16, 50), (2**12, 8), (2**18, 200), (2**14, 256), (2**20, 100)]
    Ns, Ks = [n for n, _ in sizes], [k for _, k in sizes]
    for graph in (False, True):
        bp = s4.BatchPlan(Ns, Ks, L_, Q_, seed=9, precision="bf16x3", graph=graph)
        sets = [[device_signal(n, k, 1000 * b + i, 20.0, "cuda")[0] for i, (n, k) in enumerate(sizes)]
                for b in range(3)]
        ptrs = [bp.pointers(xs) for xs in sets]
        want = [host(bp.execute(xs, ptrs=pt)) for xs, pt in zip(sets, ptrs)]
        outs = [bp.outputs() for _ in sets]
        for xs, pt, o in zip(sets, ptrs, outs):
            bp.execute(xs, out=o, ptrs=pt, asynchronous=True)
        bp.wait()
        torch.cuda.synchronize()
        for w, o in zip(want, outs):
            assert same(w, host(o))
        st = bp.stats()
        assert st["executes"] == 6 and st["transforms"] == 6 * len(sizes)
        bp.close()
