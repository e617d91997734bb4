"""sFFT4.0 (multiscale flat-window sparse FFT, arXiv 2011.05698) on GB300 (sm_103a).

A thin Python binding over the C ABI of libsfft4.so (include/sfft4.h).  Every step of
the transform runs in the library's CUDA kernels; PyTorch only provides device memory and
the current stream.  There is no CPU fallback: without the built library or a CUDA device
every call raises.

    plan = Plan(N=2**22, K=1000, l=16, q=1.0, seed=7, max_batch=64)
    idx, val, nfound, votes = plan.execute(x)            # x: cuda complex64, length N
    idx, val, nfound, votes = plan.execute_batched(xs)   # xs: cuda complex64, (nsig, N)

    bp = BatchPlan(Ns, Ks, l=16, q=1.0, seed=7)          # signals of different N_i, K_i
    idx, val, nfound, votes = bp.execute(xs)             # xs: list of cuda complex64 tensors
"""

import ctypes

from . import _lib
from ._lib import Sfft4Error, check  # noqa: F401

__all__ = ["Plan", "BatchPlan", "Sfft4Error", "load", "gather_probe"]


def load():
    return _lib.load()


def gather_probe(xs, blocks=None, iters=64, threads=512, inflight=4, l2_fetch_bytes=0):
    """Random 8-byte gathers per second within each row of xs (CUDA complex64, (nsig, N)):
    the achievable rate of the gather's access pattern on this device, with `threads` per CTA,
    `inflight` loads per thread in flight (4, 8, 16) and the L2 fetch granularity (0 = as set)."""
    import torch
    lib = _lib.load()
    if blocks is None:
        blocks = torch.cuda.get_device_properties(xs.device).multi_processor_count * 8
    sink = torch.zeros(1, dtype=torch.float32, device=xs.device)
    out = ctypes.c_double()
    check(lib.sfft4_gather_probe_ex(ctypes.c_void_p(xs.data_ptr()), xs.shape[0], xs.shape[1], xs.stride(0),
                                    ctypes.c_void_p(sink.data_ptr()), blocks, threads, iters, inflight,
                                    l2_fetch_bytes, ctypes.byref(out), _stream_ptr(xs.device)),
          "sfft4_gather_probe_ex")
    return out.value


def _stream_ptr(device):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _opts(B1=0, delta=1e-8, precision="fp32", min_votes=0, select_factor=2.0, sig_floor=1e-10,
          mag_tol=0.5, max_iters=64, max_batch=1, trace=False, profile=False, graph=False,
          location="multiscale", fold_order="signal_major", l2_fetch_bytes=0, trace_signal=0,
          decode_cluster=0, batch_exec="persistent", fold_residues=0, fold_rounds=0):
    o = _lib.Opts()
    check(_lib.load().sfft4_opts_default(ctypes.byref(o)), "sfft4_opts_default")
    o.B1 = B1
    o.delta = delta
    o.precision = {"fp32": _lib.SFFT4_FP32, "bf16x3": _lib.SFFT4_BF16X3}[precision]
    o.min_votes = min_votes
    o.select_factor = select_factor
    o.sig_floor = sig_floor
    o.mag_tol = mag_tol
    o.max_iters = max_iters
    o.max_batch = max_batch
    o.trace = int(bool(trace))
    o.profile = int(bool(profile))
    o.graph = int(bool(graph))
    o.location = {"multiscale": _lib.SFFT4_LOC_MULTISCALE, "two_round": _lib.SFFT4_LOC_TWO_ROUND}[location]
    o.fold_order = {"signal_major": _lib.SFFT4_FOLD_SIGNAL_MAJOR,
                    "iteration_major": _lib.SFFT4_FOLD_ITERATION_MAJOR}[fold_order]
    o.l2_fetch_bytes = l2_fetch_bytes
    o.trace_signal = trace_signal
    o.decode_cluster = decode_cluster
    o.batch_exec = {"persistent": _lib.SFFT4_BATCH_PERSISTENT, "levels": _lib.SFFT4_BATCH_LEVELS}[batch_exec]
    o.fold_residues = fold_residues
    o.fold_rounds = fold_rounds
    return o


def _device(device):
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("sFFT4 needs a CUDA device")
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


class Plan:
    """A static sFFT4.0 plan (Section 3.1) for one (N, K, l, q, seed).  location="two_round"
    replaces the multiscale location by the two-round (tau = 0, 1) location of sFFT3.0 for
    exactly sparse signals.  fold_order="iteration_major" folds the batch one iteration at a
    time instead of all iterations of a signal together (same results, more DRAM reads).
    batch_exec="levels" decodes a batch iteration by iteration instead of in one persistent
    launch (same results)."""

    def __init__(self, N, K, l=16, q=1.0, seed=0, *, B1=0, delta=1e-8, precision="fp32",
                 min_votes=0, select_factor=2.0, sig_floor=1e-10, mag_tol=0.5, max_iters=64,
                 max_batch=1, trace=False, profile=False, graph=False, location="multiscale",
                 fold_order="signal_major", l2_fetch_bytes=0, trace_signal=0, decode_cluster=0,
                 batch_exec="persistent", fold_residues=0, fold_rounds=0, device=None):
        import torch
        lib = _lib.load()
        self.device = _device(device)
        o = _opts(B1, delta, precision, min_votes, select_factor, sig_floor, mag_tol, max_iters,
                  max_batch, trace, profile, graph, location, fold_order, l2_fetch_bytes, trace_signal,
                  decode_cluster, batch_exec, fold_residues, fold_rounds)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.sfft4_plan(ctypes.byref(h), N, K, l, q, seed, ctypes.byref(o)), "sfft4_plan")
        self._h = h
        self.N, self.K, self.l, self.q, self.seed = N, K, l, q, seed
        self.max_batch = max_batch
        inf = _lib.PlanInfo()
        check(lib.sfft4_get_plan_info(h, ctypes.byref(inf)), "sfft4_get_plan_info")
        self.info = {k: getattr(inf, k) for k, _ in _lib.PlanInfo._fields_}

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_h", None):
            _lib.load().sfft4_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ introspection
    def iter_info(self, m):
        it = _lib.IterInfo()
        check(_lib.load().sfft4_get_iter_info(self._h, m, ctypes.byref(it)), "sfft4_get_iter_info")
        S = it.S
        return {"B": it.B, "S": S, "R": S + 1, "n_c": it.n_c, "h": it.h, "L": it.L,
                "Lbar": list(it.Lbar[:S]), "tau": list(it.tau[:S + 1]), "H": list(it.H[:S]),
                "unique_samples": it.unique_samples}

    def permutation(self, m, signal=0):
        """(sigma, a) of iteration m for Philox signal index `signal` (f moves to sigma f mod N)."""
        s, a = ctypes.c_uint64(), ctypes.c_uint64()
        check(_lib.load().sfft4_get_permutation(self._h, signal, m, ctypes.byref(s), ctypes.byref(a)),
              "sfft4_get_permutation")
        return s.value, a.value

    def window(self, B):
        """(G, Ghat) host float32 arrays of bucket count B."""
        import numpy as np
        it = next(self.iter_info(m) for m in range(1, self.info["n_iters"] + 1)
                  if self.iter_info(m)["B"] == B)
        G = np.empty(2 * it["h"] + 1, np.float32)
        Gh = np.empty(3 * it["L"] // 2 + 1, np.float32)
        check(_lib.load().sfft4_get_window(self._h, B, G.ctypes.data_as(ctypes.c_void_p),
                                           Gh.ctypes.data_as(ctypes.c_void_p)), "sfft4_get_window")
        return G, Gh

    def sync_status(self):
        """Synchronise and raise if a bounded device wait of this plan gave up."""
        check(_lib.load().sfft4_sync_status(self._h), "sfft4_sync_status")

    def inject_status(self, value=1):
        """Test hook: set the plan's device status word as a bounded wait that gave up does."""
        check(_lib.load().sfft4_inject_status(self._h, value), "sfft4_inject_status")

    def stats(self):
        """Counters and the votes histogram of the last execute's found sets (synchronises)."""
        st = _lib.RunStats()
        check(_lib.load().sfft4_stats(self._h, ctypes.byref(st)), "sfft4_stats")
        d = {k: getattr(st, k) for k, _ in _lib.RunStats._fields_ if k not in ("votes_hist", "reserved")}
        d["votes_hist"] = list(st.votes_hist)
        return d

    def profile(self, reset=True):
        """Per-kernel launch counts and CUDA-event times since the last reset (profile=True)."""
        pr = _lib.Profile()
        check(_lib.load().sfft4_profile_get(self._h, ctypes.byref(pr), int(bool(reset))), "sfft4_profile_get")
        return {k: getattr(pr, k) for k, _ in _lib.Profile._fields_}

    # ------------------------------------------------------------------ execution
    def _outputs(self, nsig):
        import torch
        K, dev = self.K, self.device
        idx = torch.empty((nsig, K), dtype=torch.int64, device=dev)
        val = torch.empty((nsig, K), dtype=torch.complex128, device=dev)
        nf = torch.empty((nsig,), dtype=torch.int64, device=dev)
        votes = torch.empty((nsig, K), dtype=torch.int8, device=dev)
        return idx, val, nf, votes

    def _check_x(self, x, ndim):
        import torch
        if not isinstance(x, torch.Tensor) or x.device.type != "cuda" or x.dtype != torch.complex64:
            raise TypeError("x must be a CUDA complex64 tensor")
        if x.dim() != ndim or x.shape[-1] != self.N or x.stride(-1) != 1:
            raise ValueError(f"x must have shape (..., {self.N}) and unit inner stride")

    def execute(self, x, out=None):
        """One transform of x (length-N complex64 on the plan's device)."""
        self._check_x(x, 1)
        idx, val, nf, votes = out if out is not None else self._outputs(1)
        check(_lib.load().sfft4_execute(self._h, ctypes.c_void_p(x.data_ptr()),
                                        ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                        ctypes.c_void_p(nf.data_ptr()), ctypes.c_void_p(votes.data_ptr()),
                                        _stream_ptr(self.device)), "sfft4_execute")
        return idx[0], val[0], nf[0], votes[0]

    def execute_batched(self, xs, out=None, asynchronous=False):
        """Transforms of each row of xs (shape (nsig, N), complex64, on the device).  With
        asynchronous=True the batch runs on the plan's own streams and overlaps the next call
        (two workspaces in turn, up to two batches in flight); its results are complete after
        wait().  xs and the outputs must then stay untouched until wait(), and calls in flight
        together need distinct output buffers."""
        self._check_x(xs, 2)
        nsig = xs.shape[0]
        idx, val, nf, votes = out if out is not None else self._outputs(nsig)
        fn = "sfft4_execute_batched_async" if asynchronous else "sfft4_execute_batched"
        check(getattr(_lib.load(), fn)(self._h, nsig, ctypes.c_void_p(xs.data_ptr()), xs.stride(0),
                                       ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                       ctypes.c_void_p(nf.data_ptr()), ctypes.c_void_p(votes.data_ptr()),
                                       _stream_ptr(self.device)), fn)
        return idx, val, nf, votes

    def host_outputs(self, nsig):
        """Page-locked host output buffers (idx, val, nfound, votes) for execute_batched_host."""
        import torch
        K = self.K
        return (torch.empty((nsig, K), dtype=torch.int64, pin_memory=True),
                torch.empty((nsig, K), dtype=torch.complex128, pin_memory=True),
                torch.empty((nsig,), dtype=torch.int64, pin_memory=True),
                torch.empty((nsig, K), dtype=torch.int8, pin_memory=True))

    def execute_batched_host(self, xs, out=None):
        """Transforms of each row of xs, a page-locked (pinned) CPU complex64 tensor of shape
        (nsig, N): the library stages the rows into device memory, runs them as an asynchronous
        execute and copies the results into the host outputs (pinned CPU tensors, see
        host_outputs).  Consecutive calls overlap; results are complete after wait() and a
        synchronize of the current stream.  xs and the outputs must stay untouched until then."""
        import torch
        if not isinstance(xs, torch.Tensor) or xs.device.type != "cpu" or xs.dtype != torch.complex64:
            raise TypeError("xs must be a CPU complex64 tensor")
        if xs.dim() != 2 or xs.shape[-1] != self.N or xs.stride(-1) != 1:
            raise ValueError(f"xs must have shape (nsig, {self.N}) and unit inner stride")
        if not xs.is_pinned():
            raise ValueError("xs must be in page-locked (pinned) host memory")
        nsig = xs.shape[0]
        idx, val, nf, votes = out if out is not None else self.host_outputs(nsig)
        check(_lib.load().sfft4_execute_batched_host(self._h, nsig, ctypes.c_void_p(xs.data_ptr()), xs.stride(0),
                                                     ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                                     ctypes.c_void_p(nf.data_ptr()), ctypes.c_void_p(votes.data_ptr()),
                                                     _stream_ptr(self.device)), "sfft4_execute_batched_host")
        return idx, val, nf, votes

    def wait(self):
        """Makes the current stream wait for every asynchronous execute issued so far."""
        check(_lib.load().sfft4_wait(self._h, _stream_ptr(self.device)), "sfft4_wait")

    def bucketize(self, x, m, signal=0):
        """Raw bucket arrays (R, B) of iteration m for Philox signal index `signal` (Lemma 1)."""
        import torch
        self._check_x(x, 1)
        it = self.iter_info(m)
        y = torch.empty((it["R"], it["B"]), dtype=torch.complex64, device=self.device)
        check(_lib.load().sfft4_bucketize(self._h, ctypes.c_void_p(x.data_ptr()), signal, m,
                                          ctypes.c_void_p(y.data_ptr()), _stream_ptr(self.device)),
              "sfft4_bucketize")
        return y

    def trace(self, m):
        """(raw buckets (R, B) complex64, found f, found v, found votes) after iteration m
        of the traced signal (trace_signal, default 0) of the last execute (trace=True)."""
        import numpy as np
        it = self.iter_info(m)
        cap = self.info["found_capacity"]
        y = np.empty((it["R"], it["B"]), np.complex64)
        f = np.empty(cap, np.int64)
        v = np.empty(cap, np.complex128)
        vt = np.empty(cap, np.int8)
        nf = ctypes.c_int64()
        check(_lib.load().sfft4_trace_get(self._h, m, y.ctypes.data_as(ctypes.c_void_p), cap,
                                          f.ctypes.data_as(ctypes.c_void_p), v.ctypes.data_as(ctypes.c_void_p),
                                          vt.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nf)),
              "sfft4_trace_get")
        n = nf.value
        return y, f[:n], v[:n], vt[:n]


class BatchPlan:
    """Plan of a batch of signals of different sizes N_i and sparsities K_i, executed together
    (each signal follows its own static schedule, Section 3.1; signal i uses Philox counter
    (i, m, 0, 0)).  Outputs are rows of length Kmax = max K_i.  B1s optionally gives each
    signal's first-iteration bucket count (0 = default), e.g. from `autotune.choose_b1`.
    batch_exec="persistent" (default) runs all folds, all DFTs and one persistent decode launch
    (CTAs taking whole signals from a device queue); "levels" runs level by level.  The
    outputs are identical."""

    def __init__(self, Ns, Ks, l=16, q=1.0, seed=0, *, B1=0, B1s=None, delta=1e-8, precision="fp32",
                 min_votes=0, select_factor=2.0, sig_floor=1e-10, mag_tol=0.5, max_iters=64,
                 profile=False, graph=False, location="multiscale", batch_exec="persistent", fold_residues=0,
                 fold_rounds=0, device=None):
        import torch
        lib = _lib.load()
        self.device = _device(device)
        Ns = [int(n) for n in Ns]
        Ks = [int(k) for k in Ks]
        if len(Ns) != len(Ks) or not Ns:
            raise ValueError("Ns and Ks must be non-empty and of equal length")
        o = _opts(B1, delta, precision, min_votes, select_factor, sig_floor, mag_tol, max_iters,
                  1, False, profile, graph, location, batch_exec=batch_exec, fold_residues=fold_residues,
                  fold_rounds=fold_rounds)
        nsig = len(Ns)
        Na = (ctypes.c_int64 * nsig)(*Ns)
        Ka = (ctypes.c_int64 * nsig)(*Ks)
        Ba = None
        if B1s is not None:
            if len(B1s) != nsig:
                raise ValueError("B1s must have one entry per signal")
            Ba = (ctypes.c_int32 * nsig)(*[int(b) for b in B1s])
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(lib.sfft4_plan_batched(ctypes.byref(h), nsig, Na, Ka, Ba, l, q, seed, ctypes.byref(o)),
                  "sfft4_plan_batched")
        self._h = h
        self.Ns, self.Ks, self.l, self.q, self.seed = Ns, Ks, l, q, seed
        inf = _lib.BatchInfo()
        check(lib.sfft4_get_batch_info(h, ctypes.byref(inf)), "sfft4_get_batch_info")
        self.info = {k: getattr(inf, k) for k, _ in _lib.BatchInfo._fields_}
        self.Kmax = self.info["Kmax"]
        self._ptrs = None

    def close(self):
        if getattr(self, "_h", None):
            _lib.load().sfft4_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sync_status(self):
        check(_lib.load().sfft4_sync_status(self._h), "sfft4_sync_status")

    def stats(self):
        """Counters and the votes histogram of the last execute's found sets (synchronises)."""
        st = _lib.RunStats()
        check(_lib.load().sfft4_stats(self._h, ctypes.byref(st)), "sfft4_stats")
        d = {k: getattr(st, k) for k, _ in _lib.RunStats._fields_ if k not in ("votes_hist", "reserved")}
        d["votes_hist"] = list(st.votes_hist)
        return d

    def profile(self, reset=True):
        pr = _lib.Profile()
        check(_lib.load().sfft4_profile_get(self._h, ctypes.byref(pr), int(bool(reset))), "sfft4_profile_get")
        return {k: getattr(pr, k) for k, _ in _lib.Profile._fields_}

    def outputs(self):
        import torch
        n, K, dev = len(self.Ns), self.Kmax, self.device
        return (torch.empty((n, K), dtype=torch.int64, device=dev),
                torch.empty((n, K), dtype=torch.complex128, device=dev),
                torch.empty((n,), dtype=torch.int64, device=dev),
                torch.empty((n, K), dtype=torch.int8, device=dev))

    def pointers(self, xs):
        """Device array of the signals' base addresses (reused across calls: the kernels read
        it, so a captured graph sees new entries)."""
        import torch
        if len(xs) != len(self.Ns):
            raise ValueError(f"expected {len(self.Ns)} signals")
        for x, N in zip(xs, self.Ns):
            if (not isinstance(x, torch.Tensor) or x.device.type != "cuda" or x.dtype != torch.complex64
                    or x.dim() != 1 or x.shape[0] != N or x.stride(0) != 1):
                raise ValueError(f"each signal must be a contiguous CUDA complex64 tensor of its N ({N})")
        host = torch.tensor([x.data_ptr() for x in xs], dtype=torch.int64)
        if self._ptrs is None:
            self._ptrs = torch.empty(len(xs), dtype=torch.int64, device=self.device)
        self._ptrs.copy_(host, non_blocking=False)
        return self._ptrs

    def execute(self, xs, out=None, ptrs=None, asynchronous=False):
        """Transforms of the signals xs (list of CUDA complex64 tensors, xs[i] of length N_i).
        Returns (idx, val, nfound, votes), rows of length Kmax; row i past K_i holds -1 / 0.
        asynchronous=True: the batch runs on the plan's own streams and overlaps the next
        call (three workspaces in turn, up to three batches in flight); results are complete
        after wait(), and xs, ptrs and the outputs must stay untouched until then."""
        if ptrs is None:
            ptrs = self.pointers(xs)
        idx, val, nf, votes = out if out is not None else self.outputs()
        fn = "sfft4_execute_batched_v_async" if asynchronous else "sfft4_execute_batched_v"
        check(getattr(_lib.load(), fn)(self._h, ctypes.c_void_p(ptrs.data_ptr()),
                                       ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(val.data_ptr()),
                                       ctypes.c_void_p(nf.data_ptr()), ctypes.c_void_p(votes.data_ptr()),
                                       _stream_ptr(self.device)), fn)
        return idx, val, nf, votes

    def wait(self):
        """Makes the current stream wait for every asynchronous execute issued so far."""
        check(_lib.load().sfft4_wait(self._h, _stream_ptr(self.device)), "sfft4_wait")
