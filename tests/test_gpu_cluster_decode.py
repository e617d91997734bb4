"""The one-signal low-latency path: the decode of each signal spread over a thread-block
cluster (opts.decode_cluster CTAs sharing the update's buckets and the candidates of Section
3.1's iteration steps 2-5), on a GB300.

Every item of the decode (an update bucket's sum, a candidate's location, votes and estimate)
is computed as by one CTA, and the int64 bucket sums of several ranks add exactly, so outputs
must be bit-identical for every cluster size; against the FP64 oracle the single-signal bar
holds (noiseless: support exact and equal to the generator's, values within 1e-5; 20 dB:
exact support and votes or a fragile parting explained by replay, values within 1e-4).
"""

import numpy as np
import pytest

from oracle import plan as OP, sfft4 as O
from synth import sparse_signal

import parity_helpers as PH

pytestmark = pytest.mark.gpu

CASES = {
    # name: (N, K, l, q, B1) -- B up to 512 uses the gather-form update, larger B the scatter form
    "c1": (2**14, 16, 4, 0.5, 64),
    "c2": (2**20, 100, 16, 1.0, 128),
    "c3": (2**22, 1000, 16, 1.0, 0),
    "l4q2": (2**20, 100, 4, 2.0, 0),
}


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def run(s4, name, x, seed, cluster, precision="fp32", nsig=None):
    N, K, l, q, B1 = CASES[name]
    p = s4.Plan(N, K, l, q, seed=seed, B1=B1, precision=precision, decode_cluster=cluster,
                max_batch=1 if nsig is None else nsig)
    out = p.execute(x) if nsig is None else p.execute_batched(x)
    out = [t.cpu() for t in out]
    p.sync_status()
    p.close()
    return out


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "l4q2"])
@pytest.mark.parametrize("snr", [None, 20.0])
def test_cluster_sizes_bit_identical(s4, name, snr):
    import torch
    N, K, l, q, B1 = CASES[name]
    sig = sparse_signal(N, K, 41, snr)
    x = to_dev(sig.x)
    ref = run(s4, name, x, 41, 1)
    for c in (2, 4, 8, 16):
        got = run(s4, name, x, 41, c)
        for u, w in zip(ref, got):
            assert torch.equal(u, w), (name, snr, c)


def test_cluster_sizes_bit_identical_batched_bf16x3(s4):
    import torch
    N, K = 2**20, 100
    xs = torch.stack([to_dev(sparse_signal(N, K, 60 + i, 20.0).x) for i in range(5)])
    ref = run(s4, "c2", xs, 7, 1, "bf16x3", nsig=5)
    for c in (4, 8):
        got = run(s4, "c2", xs, 7, c, "bf16x3", nsig=5)
        for u, w in zip(ref, got):
            assert torch.equal(u, w), c


@pytest.mark.parametrize("name,snr,seeds", [("c1", None, range(3)), ("c3", None, range(2)), ("c2", 20.0, range(2)),
                                            ("c3", 20.0, range(1))])
def test_cluster_decode_matches_oracle(s4, name, snr, seeds):
    N, K, l, q, B1 = CASES[name]
    for seed in seeds:
        sig = sparse_signal(N, K, seed, snr)
        # the default (4 CTAs for one signal) on even seeds, 8 CTAs on odd ones
        p = s4.Plan(N, K, l, q, seed=seed, B1=B1, decode_cluster=(0, 8)[seed % 2], trace=True)
        idx, val, nf, votes = p.execute(to_dev(sig.x))
        n = int(nf.item())
        f, v, vt = idx[:n].cpu().numpy(), val[:n].cpu().numpy(), votes[:n].cpu().numpy()
        r = O.run(sig.x.astype(np.complex128), OP.make_plan(N, K, l, q, seed=seed, B1=B1), trace=True)
        if snr is None:
            assert np.array_equal(f, sig.freqs)
        PH.assert_oracle_parity(f, v, vt, r, lambda: PH.explain_divergence(p, r, N, K, l, q, seed, B1),
                                1e-5 if snr is None else 1e-4)
        p.close()


def test_decode_cluster_option_validation(s4):
    with pytest.raises(s4.Sfft4Error):
        s4.Plan(2**14, 16, 4, 0.5, decode_cluster=3)
    with pytest.raises(s4.Sfft4Error):
        s4.Plan(2**14, 16, 4, 0.5, decode_cluster=32)
