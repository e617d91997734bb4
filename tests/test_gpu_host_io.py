"""Executes on host buffers (sfft4_execute_batched_host) on a GB300: the inputs staged from
page-locked host memory by the library's zero-copy kernel, the batch run as an asynchronous
execute and the results copied back must equal, bit for bit, what sfft4_execute_batched gives
for the same rows already in device memory (the transforms are those of Section 3.1 in both
cases; only the inputs' and outputs' memory differs)."""

import ctypes

import numpy as np
import pytest

from synth import sparse_signal

pytestmark = pytest.mark.gpu

N, K, L_, Q_ = 2**18, 100, 16, 1.0


@pytest.fixture(scope="module")
def s4(cuda_device):
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4
    return s4


def pinned_rows(seeds, stride):
    """Pinned (len(seeds), stride) complex64 buffer holding the signals in its first N columns;
    returns the (len(seeds), N) view (row stride `stride`)."""
    import torch
    buf = torch.zeros((len(seeds), stride), dtype=torch.complex64, pin_memory=True)
    for i, s in enumerate(seeds):
        buf[i, :N] = torch.from_numpy(sparse_signal(N, K, s, 20.0).x)
    return buf[:, :N]


def device_reference(s4, xs_host, precision):
    import torch
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=8, precision=precision)
    out = p.execute_batched(xs_host.to("cuda").contiguous())
    out = [t.cpu() for t in out]
    p.sync_status()
    p.close()
    return out


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
@pytest.mark.parametrize("stride_pad", [0, 2, 1])
def test_host_execute_bit_identical(s4, precision, stride_pad):
    """Two calls in flight (distinct inputs and outputs), rows with a padded stride (stride_pad
    2: the 16-byte staging path on padded rows; 1: odd stride, the 8-byte path)."""
    import torch
    a = pinned_rows([11, 12, 13, 14, 15], N + stride_pad)
    b = pinned_rows([21, 22, 23], N + stride_pad)
    ra, rb = device_reference(s4, a, precision), device_reference(s4, b, precision)
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=8, precision=precision)
    oa, ob = p.host_outputs(5), p.host_outputs(3)
    p.execute_batched_host(a, oa)
    p.execute_batched_host(b, ob)
    p.wait()
    torch.cuda.synchronize()
    p.sync_status()
    for got, want in ((oa, ra), (ob, rb)):
        for u, w in zip(got, want):
            assert torch.equal(u, w)
    # the workspaces and staging buffers are reused: a second round of calls, swapped
    oa2, ob2 = p.host_outputs(3), p.host_outputs(5)
    p.execute_batched_host(b, oa2)
    p.execute_batched_host(a, ob2)
    p.wait()
    torch.cuda.synchronize()
    for got, want in ((oa2, rb), (ob2, ra)):
        for u, w in zip(got, want):
            assert torch.equal(u, w)
    p.close()


def test_host_execute_rejects_pageable_and_bad_sizes(s4):
    import torch
    from paper_2011_05698_gb300 import _lib
    lib = _lib.load()
    p = s4.Plan(N, K, L_, Q_, seed=5, max_batch=4)
    outs = p.host_outputs(2)
    ptr = [ctypes.c_void_p(t.data_ptr()) for t in outs]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    pageable = np.zeros((2, N), np.complex64)   # ordinary host memory: not page-locked
    rc = lib.sfft4_execute_batched_host(p._h, 2, ctypes.c_void_p(pageable.ctypes.data), N, *ptr, stream)
    assert rc == _lib.SFFT4_EINVAL
    good = pinned_rows([31, 32], N)
    gp = ctypes.c_void_p(good.data_ptr())
    assert lib.sfft4_execute_batched_host(p._h, 5, gp, N, *ptr, stream) == _lib.SFFT4_EINVAL      # > max_batch
    assert lib.sfft4_execute_batched_host(p._h, 0, gp, N, *ptr, stream) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched_host(p._h, 2, gp, N - 1, *ptr, stream) == _lib.SFFT4_EINVAL  # stride < N
    assert lib.sfft4_execute_batched_host(p._h, 2, None, N, *ptr, stream) == _lib.SFFT4_EINVAL
    with pytest.raises(ValueError):
        p.execute_batched_host(torch.zeros((2, N), dtype=torch.complex64))   # not pinned
    # a valid call still works after the rejected ones
    p.execute_batched_host(good, outs)
    p.wait()
    torch.cuda.synchronize()
    p.sync_status()
    assert bool((outs[2] > 0).all())
    p.close()
