"""Launch accounting of the plan profile (opts.profile) on a GB300: the launches it records per
execute, by kernel kind, add up to the plan's own count of kernels per execute, and the
tensor-core DFT's grouped call counts both of its stage launches."""

import pytest

from synth import sparse_signal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("order", ["signal_major", "iteration_major"])
def test_profile_launches_add_up(s4, precision, order):
    import numpy as np
    import torch
    N, K, nsig, reps = 2**18, 100, 4, 3
    xs = torch.from_numpy(np.stack([sparse_signal(N, K, 70 + i, 20.0).x for i in range(nsig)])).to("cuda")
    p = s4.Plan(N, K, 16, 1.0, seed=5, max_batch=nsig, precision=precision, fold_order=order, profile=True)
    out = p._outputs(nsig)
    p.execute_batched(xs, out)
    torch.cuda.synchronize()
    p.profile(reset=True)
    for _ in range(reps):
        p.execute_batched(xs, out)
    torch.cuda.synchronize()
    pr = p.profile(reset=True)
    info = p.info
    p.close()
    per = {k: pr[k + "_launches"] / reps for k in ("fold", "fft", "decode", "finalize")}
    assert sum(per.values()) == info["kernels_per_execute"], (per, info["kernels_per_execute"])
    n_iters = info["n_iters"]
    assert per["finalize"] == 1 and per["decode"] == n_iters
    if order == "signal_major":
        assert per["fold"] == 1
    if precision == "bf16x3" and order == "signal_major":
        assert per["fft"] == 2   # first stages of every iteration, then the second stages (B1 = 256)
    elif precision == "fp32":
        assert per["fft"] == n_iters
