"""The location's phase measurement (Section 3.2, Eq. 16-19; the Monte Carlo of Fig. 5) and the
permutation draws the library exposes, on a GB300."""

import os
import sys

import numpy as np
import pytest

from oracle import philox, plan as OP, sfft4 as O, window as OW
from synth import sparse_signal

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def to_dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def test_permutation_matches_oracle_philox(s4):
    N, K = 2**20, 100
    p = s4.Plan(N, K, 16, 1.0, seed=1234567, B1=128)
    for m in (1, 2, p.info["n_iters"]):
        for sig in (0, 1, 37, 2**40 + 5):
            assert p.permutation(m, signal=sig) == philox.permutation_draw(1234567, sig, m, N)
    p.close()


def gpu_and_oracle_errors(s4, bench, N, B, K, snr, seed, signal):
    sig = sparse_signal(N, K, seed, snr)
    p = s4.Plan(N, K, 16, 1.0, seed=11, B1=B)
    taus = p.iter_info(1)["tau"]
    Yg = p.bucketize(to_dev(sig.x), 1, signal=signal).cpu().numpy().astype(np.complex128)
    sigma, a = p.permutation(1, signal=signal)
    p.close()
    op = OP.make_plan(N, K, 16, 1.0, seed=11, B1=B)
    it = op.iters[0]
    G, h, _ = OW.WindowCache(N, op.delta).get(it.B)
    Yo = O.bucketize(sig.x.astype(np.complex128), N, it.B, G, h, sigma, O.round_offsets(sigma, a, it, N))
    eg = bench.phase_errors(Yg, sig.freqs, np.uint64(sigma), N, B, taus)
    eo = bench.phase_errors(Yo, sig.freqs, np.uint64(sigma), N, B, taus)
    return eg, eo


def test_noiseless_isolated_tones_have_no_phase_error(s4, bench):
    eg, eo = gpu_and_oracle_errors(s4, bench, 2**17, 64, 50, None, 3, 0)
    assert eg.size > 0
    assert np.max(eo) < 1e-6           # the oracle: e^{2 pi i u tau / N} up to complex64 input and leakage
    assert np.max(eg) < 2e-5           # FP32 buckets


@pytest.mark.parametrize("snr", [0.0, 40.0])
def test_phase_errors_match_oracle_buckets(s4, bench, snr):
    eg, eo = gpu_and_oracle_errors(s4, bench, 2**17, 64, 50, snr, 5, 2)
    assert eg.size == eo.size and eg.size > 0
    assert np.max(np.abs(eg - eo)) < 1e-4


def test_phase_error_falls_with_snr(s4, bench):
    q = []
    for snr in (0.0, 20.0, 40.0):
        e = np.concatenate([gpu_and_oracle_errors(s4, bench, 2**17, 64, 50, snr, 7 + t, t)[0] for t in range(4)])
        q.append(np.quantile(e, 0.99))
    assert q[0] > q[1] > q[2]
