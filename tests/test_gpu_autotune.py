"""The B1 autotuner and per-signal B1 in a batch of uneven signals (GB300)."""

import numpy as np
import pytest

from synth import sparse_signal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def test_tune_one_picks_fastest_exact_candidate(s4):
    from paper_2011_05698_gb300 import autotune
    rec = autotune.tune_one(2**16, 50, 16, 1.0, "bf16x3", batch=8)
    tried = rec["tried"]
    assert {t["B1"] for t in tried} <= set(autotune.candidates(2**16, 50))
    good = [t for t in tried if t["exact_support"]]
    assert good, tried
    best = min(good, key=lambda t: t["ms_per_transform"])
    default = next(t for t in good if t["B1"] == autotune._pow2ceil(2 * 50))
    # the default stays unless another candidate is at least 3 % faster
    want = best if best["ms_per_transform"] <= 0.97 * default["ms_per_transform"] else default
    assert rec["B1"] == want["B1"]


def test_choose_b1_caches(s4, tmp_path):
    from paper_2011_05698_gb300 import autotune
    path = str(tmp_path / "tune.json")
    Ns, Ks = [2**16, 2**16, 2**14], [50, 40, 16]
    a = autotune.choose_b1(Ns, Ks, 16, 1.0, "fp32", cache_path=path, batch=4)
    assert a[0] == a[1]  # one (N, pow2ceil(K)) class
    b = autotune.choose_b1(Ns, Ks, 16, 1.0, "fp32", cache_path=path, batch=4)
    assert a == b and autotune.choose_b1.last_seconds < 1.0


def test_per_signal_b1_matches_uniform_plan(s4):
    """A batch member with an explicit B1 equals the uniform plan with that B1, bit for bit."""
    import torch
    sizes = [(2**16, 50, 64), (2**16, 50, 0), (2**14, 16, 32)]
    sigs = [sparse_signal(N, K, 40 + i, None) for i, (N, K, _) in enumerate(sizes)]
    xs = [torch.from_numpy(s.x).to("cuda") for s in sigs]
    bp = s4.BatchPlan([n for n, _, _ in sizes], [k for _, k, _ in sizes], 16, 1.0, seed=6,
                      B1s=[b for _, _, b in sizes])
    assert bp.info["n_classes"] == 3
    idx, val, nf, _ = bp.execute(xs)
    for i, (N, K, b) in enumerate(sizes):
        p = s4.Plan(N, K, 16, 1.0, seed=6, B1=b, max_batch=i + 1)
        batch = torch.zeros((i + 1, N), dtype=torch.complex64, device="cuda")
        batch[i] = xs[i]
        ui, uv, un, _ = p.execute_batched(batch)
        assert int(un[i]) == int(nf[i])
        assert torch.equal(ui[i], idx[i, :K]) and torch.equal(uv[i], val[i, :K])
        assert np.array_equal(idx[i, :int(nf[i])].cpu().numpy(), sigs[i].freqs)
        p.close()
    bp.close()


def test_tile_shape_tuning_and_oracle_parity(s4, tmp_path):
    """The fold tile shape (residues per fold CTA, rounds per fold group): the tuner keeps the
    fastest exact candidate (or the default within 3 %), and a plan with a non-default shape
    still matches the oracle (its fold sums in another order: FP32-rounding differences)."""
    from oracle import plan as OP, sfft4 as O
    from paper_2011_05698_gb300 import autotune
    rec = autotune.tune_one(2**16, 50, 16, 1.0, "bf16x3", batch=8)
    assert rec["fold_residues"] in autotune.RESIDUES and rec["fold_rounds"] in autotune.ROUNDS
    assert rec["tried_shape"] and all(t["exact_support"] for t in rec["tried_shape"])
    B1s, res, rnd = autotune.choose([2**16, 2**14], [50, 16], 16, 1.0, "fp32", cache_path=str(tmp_path / "t.json"),
                                    batch=4)
    # a batch keeps the batched plans' rounds per fold group; the residues come from the tuner
    assert len(B1s) == 2 and res in autotune.RESIDUES and rnd == autotune.BATCH_ROUNDS
    import torch
    N, K = 2**20, 100
    sig = sparse_signal(N, K, 3, None)
    for res, rnd in ((16, 4), (64, 8)):
        p = s4.Plan(N, K, 4, 1.0, seed=3, fold_residues=res, fold_rounds=rnd)
        idx, val, nf, _ = p.execute(torch.from_numpy(sig.x).to("cuda"))
        n = int(nf)
        r = O.run(sig.x.astype(np.complex128), OP.make_plan(N, K, 4, 1.0, seed=3))
        assert np.array_equal(idx[:n].cpu().numpy(), r["f"]) and np.array_equal(r["f"], sig.freqs)
        v = val[:n].cpu().numpy()
        assert np.linalg.norm(v - r["v"]) <= 1e-5 * np.linalg.norm(r["v"])
        p.close()
