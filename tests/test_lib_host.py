"""Host-side checks of the C ABI library (no GPU): it loads, exports every entry point the
header declares, its structs have the C layout, and argument validation rejects bad
input before any device work."""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sfft4.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2011_05698_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SFFT4_API\s+[\w\s\*]+?\b(sfft4_\w+)\s*\(", text)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for need in ("sfft4_plan", "sfft4_execute", "sfft4_execute_batched", "sfft4_destroy",
                 "sfft4_strerror", "sfft4_get_plan_info", "sfft4_bucketize", "sfft4_plan_batched",
                 "sfft4_execute_batched_v", "sfft4_get_batch_info", "sfft4_execute_batched_async",
                 "sfft4_execute_batched_host", "sfft4_wait", "sfft4_window_noalloc"):
        assert need in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2011_05698_gb300 import _lib
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
    declared_in_binding = {n for n, _, _ in _lib.SIGNATURES}
    assert declared_in_binding == set(declared_functions())


def test_struct_layouts_match_c(tmp_path):
    from paper_2011_05698_gb300 import _lib
    src = tmp_path / "sz.c"
    src.write_text('#include "sfft4.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sfft4_opts), '
                   'sizeof(sfft4_plan_info), sizeof(sfft4_iter_info), offsetof(sfft4_iter_info, tau), '
                   'offsetof(sfft4_iter_info, unique_samples), sizeof(sfft4_c128), '
                   'offsetof(sfft4_opts, graph), sizeof(sfft4_batch_info), '
                   'offsetof(sfft4_batch_info, samples_per_execute), sizeof(sfft4_run_stats), '
                   'offsetof(sfft4_run_stats, votes_hist), offsetof(sfft4_opts, location), '
                   'offsetof(sfft4_opts, fold_order), offsetof(sfft4_opts, trace_signal), '
                   'offsetof(sfft4_opts, batch_exec), offsetof(sfft4_opts, fold_rounds), '
                   'offsetof(sfft4_opts, decode_cluster)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(_lib.Opts), ctypes.sizeof(_lib.PlanInfo), ctypes.sizeof(_lib.IterInfo),
            _lib.IterInfo.tau.offset, _lib.IterInfo.unique_samples.offset, ctypes.sizeof(_lib.C128),
            _lib.Opts.graph.offset, ctypes.sizeof(_lib.BatchInfo), _lib.BatchInfo.samples_per_execute.offset,
            ctypes.sizeof(_lib.RunStats), _lib.RunStats.votes_hist.offset, _lib.Opts.location.offset,
            _lib.Opts.fold_order.offset, _lib.Opts.trace_signal.offset, _lib.Opts.batch_exec.offset,
            _lib.Opts.fold_rounds.offset, _lib.Opts.decode_cluster.offset]
    assert got == want


def test_opts_default_and_strerror(lib):
    from paper_2011_05698_gb300 import _lib
    o = _lib.Opts()
    assert lib.sfft4_opts_default(ctypes.byref(o)) == 0
    assert o.delta == 1e-8 and o.select_factor == 2.0 and o.mag_tol == 0.5 and o.max_batch == 1
    assert lib.sfft4_opts_default(None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_strerror(_lib.SFFT4_EINVAL) == b"invalid argument"
    assert lib.sfft4_strerror(12345) == b"unknown error"


@pytest.mark.parametrize("N,K,l,q,B1", [
    (1000, 4, 16, 1.0, 0),        # N not a power of two
    (128, 1, 16, 1.0, 0),         # N < 2^8
    (2**31, 4, 16, 1.0, 0),       # N > 2^30
    (2**14, 0, 16, 1.0, 0),       # K < 1
    (2**14, 300, 16, 1.0, 0),     # K > N / 64
    (2**20, 5000, 16, 1.0, 0),    # K > 4096
    (2**14, 16, 1, 0.0, 0),       # l < 2
    (2**14, 16, 33, 1.0, 0),      # l > 32
    (2**14, 16, 2, 1.0, 0),       # l <= q + 1
    (2**14, 16, 16, -0.5, 0),     # q < 0
    (2**14, 16, 16, 1.0, 48),     # B1 not a power of two
    (2**14, 16, 16, 1.0, 512),    # B1 > N / 64
])
def test_plan_rejects_invalid_parameters(lib, N, K, l, q, B1):
    from paper_2011_05698_gb300 import _lib
    o = _lib.Opts()
    lib.sfft4_opts_default(ctypes.byref(o))
    o.B1 = B1
    h = ctypes.c_void_p()
    assert lib.sfft4_plan(ctypes.byref(h), N, K, l, q, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL
    assert not h.value


def test_plan_rejects_bad_options(lib):
    from paper_2011_05698_gb300 import _lib
    for field, val in [("delta", 0.7), ("precision", 7), ("max_batch", -1), ("mag_tol", -1.0),
                       ("location", 3), ("fold_order", 2), ("fold_order", -1), ("decode_cluster", 3),
                       ("decode_cluster", 32), ("decode_cluster", -1), ("batch_exec", 2), ("batch_exec", -1),
                       ("fold_residues", 8), ("fold_residues", 48), ("fold_rounds", 9), ("fold_rounds", -1)]:
        o = _lib.Opts()
        lib.sfft4_opts_default(ctypes.byref(o))
        setattr(o, field, val)
        h = ctypes.c_void_p()
        assert lib.sfft4_plan(ctypes.byref(h), 2**14, 16, 4, 0.5, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL
    assert lib.sfft4_plan(None, 2**14, 16, 4, 0.5, 0, None) == _lib.SFFT4_EINVAL
    # the iteration-major fold puts the batch in grid.y: more than 65535 signals is rejected at
    # plan time (before any device work), not at the first launch
    o = _lib.Opts()
    lib.sfft4_opts_default(ctypes.byref(o))
    o.fold_order = _lib.SFFT4_FOLD_ITERATION_MAJOR
    o.max_batch = 65536
    h = ctypes.c_void_p()
    assert lib.sfft4_plan(ctypes.byref(h), 2**14, 16, 4, 0.5, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL
    assert not h.value
    # the traced signal must be a signal of the batch
    for ts in (-1, 4):
        o = _lib.Opts()
        lib.sfft4_opts_default(ctypes.byref(o))
        o.trace, o.max_batch, o.trace_signal = 1, 4, ts
        assert lib.sfft4_plan(ctypes.byref(h), 2**14, 16, 4, 0.5, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL


def test_execute_rejects_null_arguments(lib):
    from paper_2011_05698_gb300 import _lib
    assert lib.sfft4_execute(None, None, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched(None, 1, None, 0, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_get_plan_info(None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_trace_get(None, 1, None, 0, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched_v(None, None, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_get_batch_info(None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_stats(None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched_async(None, 1, None, 0, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched_host(None, 1, None, 0, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_wait(None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_execute_batched_v_async(None, None, None, None, None, None, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_sync_status(None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_inject_status(None, 1) == _lib.SFFT4_EINVAL
    lib.sfft4_destroy(None)


def test_plan_batched_rejects_invalid_sizes(lib):
    from paper_2011_05698_gb300 import _lib
    h = ctypes.c_void_p()

    def arr(v):
        return (ctypes.c_int64 * len(v))(*v)

    # one bad signal anywhere in the batch rejects the whole plan, before any device work
    for Ns, Ks in [([2**14, 1000], [16, 4]), ([2**14, 2**16], [16, 0]), ([2**14], [300])]:
        assert lib.sfft4_plan_batched(ctypes.byref(h), len(Ns), arr(Ns), arr(Ks), None, 16, 1.0, 0, None) \
            == _lib.SFFT4_EINVAL
        assert not h.value
    assert lib.sfft4_plan_batched(ctypes.byref(h), 0, arr([2**14]), arr([16]), None, 16, 1.0, 0, None) \
        == _lib.SFFT4_EINVAL
    assert lib.sfft4_plan_batched(ctypes.byref(h), 1, None, None, None, 16, 1.0, 0, None) == _lib.SFFT4_EINVAL
    assert lib.sfft4_plan_batched(None, 1, arr([2**14]), arr([16]), None, 16, 1.0, 0, None) == _lib.SFFT4_EINVAL
    # a per-signal B1 that is not a power of two, or whose window is wider than N/2
    b1 = (ctypes.c_int32 * 2)(0, 48)
    assert lib.sfft4_plan_batched(ctypes.byref(h), 2, arr([2**14, 2**14]), arr([16, 16]), b1, 16, 1.0, 0, None) \
        == _lib.SFFT4_EINVAL


def test_binding_fails_loudly_without_cuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import paper_2011_05698_gb300 as s4
    with pytest.raises(RuntimeError):
        s4.Plan(2**14, 16, 4, 0.5)


def test_autotune_candidates():
    from paper_2011_05698_gb300 import autotune
    assert autotune.candidates(2**22, 1000) == [512, 1024, 2048, 4096]
    assert autotune.candidates(2**16, 600) == [512, 1024]          # capped at N/64
    assert autotune.candidates(2**14, 4) == [16]                   # floor at 16
    assert all(b & (b - 1) == 0 for b in autotune.candidates(2**20, 77))


def test_two_round_location_limits(lib):
    from paper_2011_05698_gb300 import _lib
    o = _lib.Opts()
    lib.sfft4_opts_default(ctypes.byref(o))
    h = ctypes.c_void_p()
    o.location = 2
    assert lib.sfft4_plan(ctypes.byref(h), 2**14, 16, 4, 0.5, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL
    o.location = _lib.SFFT4_LOC_TWO_ROUND
    assert lib.sfft4_plan(ctypes.byref(h), 2**21, 16, 16, 1.0, 0, ctypes.byref(o)) == _lib.SFFT4_EINVAL
    assert not h.value
