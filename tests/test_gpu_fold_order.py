"""The two fold orders of a batched execute (opts.fold_order), on a GB300.

Signal-major order folds every iteration of the batch in one launch, the CTAs of one
signal's iterations adjacent; iteration-major order folds one iteration at a time.  Each
(signal, iteration, residue slice) is folded by the same code with the same thread mapping
and the same reduction order in both, so:
  * the bucket arrays of every iteration and the outputs are bit-identical between the orders;
  * the signal-major bucket arrays (execute path, traced for signal 0) match the FP64 oracle's
    within the bucketization bar of the parity tests (5e-6 relative l2 per round);
  * against the oracle (each signal with its own Philox signal index), the noiseless support
    is the oracle's and the generator's and the values are within 1e-5 relative l2.
Cases cover single-group iterations (l = 16), iterations of several fold groups with
different round counts (l = 4, q = 2: up to 41 rounds, groups of up to 8), and bucket counts
from 16 to 4096 (N = 2^20, K = 2000: B_1 = 4096).
"""

import math

import numpy as np
import pytest

from oracle import philox, plan as OP, sfft4 as O, window as OW
from synth import sparse_signal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def batch(N, K, seeds, snr):
    import torch
    xs = np.stack([sparse_signal(N, K, s, snr).x for s in seeds])
    return torch.from_numpy(xs).to("cuda")


def run(s4, order, N, K, l, q, xs, precision, trace=False):
    p = s4.Plan(N, K, l, q, seed=11, max_batch=xs.shape[0], precision=precision, fold_order=order,
                trace=trace)
    idx, val, nf, votes = p.execute_batched(xs)
    p.sync_status()
    out = (idx.cpu().numpy(), val.cpu().numpy(), nf.cpu().numpy(), votes.cpu().numpy())
    ys = [p.trace(m)[0] for m in range(1, p.info["n_iters"] + 1)] if trace else None
    info = dict(p.info)
    p.close()
    return out, ys, info


CASES = [(2**16, 40, 16, 1.0, 20.0), (2**18, 300, 4, 2.0, 20.0), (2**20, 2000, 16, 1.0, None)]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("N,K,l,q,snr", CASES)
def test_orders_bit_identical(s4, N, K, l, q, snr, precision):
    xs = batch(N, K, range(5), snr)
    a, ya, ia = run(s4, "signal_major", N, K, l, q, xs, precision, trace=True)
    b, yb, ib = run(s4, "iteration_major", N, K, l, q, xs, precision, trace=True)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    for m, (u, v) in enumerate(zip(ya, yb), 1):
        assert np.array_equal(u.view(np.uint32), v.view(np.uint32)), m
    # one fold launch instead of one per (iteration, fold group)
    assert ia["kernels_per_execute"] < ib["kernels_per_execute"]


@pytest.mark.parametrize("N,K,l,q,snr", CASES[:2])
def test_signal_major_buckets_match_oracle(s4, N, K, l, q, snr):
    """Traced bucket arrays of the execute path against the oracle's bucketization."""
    sig = sparse_signal(N, K, 0, snr)
    xs = batch(N, K, [0, 1], snr)
    _, ys, _ = run(s4, "signal_major", N, K, l, q, xs, "fp32", trace=True)
    op = OP.make_plan(N, K, l, q, seed=11)
    wc = OW.WindowCache(N, op.delta)
    x128 = sig.x.astype(np.complex128)
    for m in sorted({1, 2, len(op.iters)}):
        it = op.iters[m - 1]
        sigma, a_ = philox.permutation_draw(11, 0, m, N)
        G, h, _ = wc.get(it.B)
        Yo = O.bucketize(x128, N, it.B, G, h, sigma, O.round_offsets(sigma, a_, it, N))
        Yg = ys[m - 1].astype(np.complex128)
        for s in range(it.R):
            rel = np.linalg.norm(Yg[s] - Yo[s]) / np.linalg.norm(Yo[s])
            assert rel < 5e-6, (m, s, rel)
            assert np.max(np.abs(Yg[s] - Yo[s])) < 2e-5 * np.linalg.norm(Yo[s]) / math.sqrt(it.B), (m, s)


def test_signal_major_noiseless_matches_oracle(s4):
    N, K, l, q = 2**18, 300, 4, 2.0
    seeds = [3, 4, 5]
    xs = batch(N, K, seeds, None)
    (idx, val, nf, votes), _, _ = run(s4, "signal_major", N, K, l, q, xs, "bf16x3")
    for i, sd in enumerate(seeds):
        sig = sparse_signal(N, K, sd, None)
        r = O.run(sig.x.astype(np.complex128), OP.make_plan(N, K, l, q, seed=11), signal=i)
        n = int(nf[i])
        assert np.array_equal(idx[i, :n], r["f"])
        assert np.array_equal(idx[i, :n], sig.freqs)
        assert np.linalg.norm(val[i, :n] - r["v"]) <= 1e-5 * np.linalg.norm(r["v"])



@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_fold_rounds_regroup_without_changing_sums(s4, precision):
    """opts.fold_rounds only regroups the fold's tiles (every thread still adds a round's
    samples in increasing t, and the copies of a slot in copy order), so every bucket array
    and every output is bit-identical whatever the group size, in both fold orders."""
    import torch
    N, K, l, q = 2**20, 100, 16, 1.0
    xs = batch(N, K, [50, 51, 52], 20.0)
    ref = None
    for order in ("signal_major", "iteration_major"):
        for rnd in (1, 3, 6, 8):
            p = s4.Plan(N, K, l, q, seed=9, max_batch=3, precision=precision, fold_order=order, fold_rounds=rnd,
                        trace=True, trace_signal=1)
            out = [t.cpu() for t in p.execute_batched(xs)]
            ys = [p.trace(m)[0] for m in range(1, p.info["n_iters"] + 1)]
            p.sync_status()
            p.close()
            if ref is None:
                ref = (out, ys)
                continue
            for u, w in zip(out, ref[0]):
                assert torch.equal(u, w), (order, rnd)
            for m, (u, w) in enumerate(zip(ys, ref[1])):
                assert np.array_equal(u.view(np.uint32), w.view(np.uint32)), (order, rnd, m + 1)
