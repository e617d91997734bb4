"""The bench line's accuracy report (bench.accuracy_vs_oracle) on planted results, on the host:
it counts a signal as support- and vote-identical only when the GPU's lists equal the oracle's
exactly, and reports the values' relative l2 error over the signals whose support is equal."""

import os
import sys
import types

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def planted(n, K, seed=0):
    """Oracle-like results (time, nfound, f, v, votes) of n signals."""
    rng = np.random.default_rng(seed)
    res = []
    for _ in range(n):
        k = K - int(rng.integers(0, 5))
        f = np.sort(rng.choice(1 << 20, size=k, replace=False)).astype(np.int64)
        v = rng.standard_normal(k) + 1j * rng.standard_normal(k)
        vt = rng.integers(1, 5, size=k).astype(np.int8)
        res.append((1.0, k, f, v, vt))
    return res


def fake_s4(res, K, mutate):
    import torch

    class Plan:
        def __init__(self, N, K_, l, q, seed, max_batch, precision):
            self.n, self.precision = max_batch, precision

        def execute_batched(self, xs):
            idx = np.full((self.n, K), -1, np.int64)
            val = np.zeros((self.n, K), np.complex128)
            nf = np.zeros(self.n, np.int64)
            vt = np.zeros((self.n, K), np.int8)
            for i, (_, k, f, v, t) in enumerate(res):
                f2, v2, t2 = mutate(i, f.copy(), v.copy(), t.copy(), self.precision)
                idx[i, :len(f2)], val[i, :len(f2)], vt[i, :len(f2)], nf[i] = f2, v2, t2, len(f2)
            return [torch.from_numpy(a) for a in (idx, val, nf, vt)]

        def close(self):
            pass

    return types.SimpleNamespace(Plan=Plan)


def test_accuracy_report_counts_exact_matches(monkeypatch):
    import torch
    K, n = 40, 4
    monkeypatch.setattr(bench, "K_DEF", K)
    monkeypatch.setattr(bench, "N_DEF", 1 << 10)   # the synthesised inputs only feed the stand-in
    res = planted(n, K)

    def mutate(i, f, v, t, precision):
        if i == 1:
            t[0] = t[0] + 1                        # one vote differs: support equal, votes not
        if i == 2:
            f[0] = f[0] + 1                        # support differs
        if i == 3:
            v = v * (1 + (2e-5 if precision == "bf16x3" else 1e-6))
        return f, v, t

    out = bench.accuracy_vs_oracle(fake_s4(res, K, mutate), res, n, 20.0, 7_000, 1234, torch.device("cpu"))
    for prec, err in (("bf16x3", 2e-5), ("fp32", 1e-6)):
        r = out[prec]
        assert r["support_identical"] == 3 and r["votes_identical"] == 2, r
        assert abs(r["value_rel_l2_max"] - err) <= 1e-6 * err   # v (1 + e) against v: exactly e
        assert r["value_rel_l2_median"] == 0.0
