"""The allocation-free window entry point (sfft4_window_noalloc), through the C ABI.

For callers that cannot allocate device memory where they need the window tables, the
library computes them into caller buffers with a static device array as its only scratch.
Its output must match the tables the allocating path (sfft4_plan / sfft4_get_window)
builds, on consecutive calls that reuse the shared scratch.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _window_noalloc(lib, torch, N, B, delta, G_cap, Gh_cap):
    G = torch.full((G_cap,), float("nan"), dtype=torch.float32, device="cuda")
    Gh = torch.full((Gh_cap,), float("nan"), dtype=torch.float32, device="cuda")
    rc = lib.sfft4_window_noalloc(N, B, delta, ctypes.c_void_p(G.data_ptr()), G_cap,
                                  ctypes.c_void_p(Gh.data_ptr()), Gh_cap,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, G.cpu().numpy(), Gh.cpu().numpy()


def test_window_noalloc_matches_allocating_path(cuda_device):
    import torch
    from paper_2011_05698_gb300 import build, _lib
    build.build()
    import paper_2011_05698_gb300 as s4
    lib = _lib.load()
    N, K = 2**22, 1000
    p = s4.Plan(N, K, 16, 1.0, seed=3)
    Bs = sorted({p.iter_info(m)["B"] for m in range(1, p.info["n_iters"] + 1)}, reverse=True)[:2]
    refs = {B: p.window(B) for B in Bs}
    p.close()
    # two calls in a row on different B (the second reuses the scratch), then the first again
    for B in Bs + Bs[:1]:
        G_ref, Gh_ref = refs[B]
        rc, G, Gh = _window_noalloc(lib, torch, N, B, 1e-8, G_ref.size + 7, Gh_ref.size + 5)
        assert rc == 0, lib.sfft4_strerror(rc)
        assert np.max(np.abs(G[:G_ref.size] - G_ref)) <= 2.0**-23 * np.max(np.abs(G_ref))
        assert np.max(np.abs(Gh[:Gh_ref.size] - Gh_ref)) < 2e-6
        assert np.all(np.isnan(G[G_ref.size:])) and np.all(np.isnan(Gh[Gh_ref.size:]))


def test_window_noalloc_rejects_sizes_beyond_its_scratch(cuda_device):
    import torch
    from paper_2011_05698_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    # B = 4096 at delta = 1e-8 needs w = 181,415 > 131,072 coefficients of scratch
    rc, _, _ = _window_noalloc(lib, torch, 2**22, 4096, 1e-8, 200_000, 2000)
    assert rc == _lib.SFFT4_EINVAL
    # capacities too small for the requested window
    rc, _, _ = _window_noalloc(lib, torch, 2**22, 1024, 1e-8, 100, 100)
    assert rc == _lib.SFFT4_EINVAL
