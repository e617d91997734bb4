"""Autotuner of the first-iteration bucket count B1 per (N, K class).

B1 sets the whole static schedule (Section 3.1): more buckets isolate more coefficients per
iteration but widen the window (w ~ 44 B1 samples at delta = 1e-8) and the DFT; fewer buckets
read fewer samples per iteration but need more iterations.  The default is pow2ceil(2K).  For
each (N, pow2ceil(K)) class the tuner times the candidates pow2ceil(2K) x {1/4, 1/2, 1, 2}
(those the planner accepts) on noiseless probe signals of the class's largest K, in batches
large enough to fill the GPU (about 2^27 signal samples per execute, so the time is throughput,
not the latency of one schedule), keeps those that recover every probe's support exactly, and
picks the fastest, keeping the default unless another candidate is at least 3 % faster.
Choices are cached in a JSON file keyed by device, precision, N, K class, l and q.

    from paper_2011_05698_gb300 import autotune
    B1s = autotune.choose_b1(Ns, Ks, l=16, q=1.0, precision="bf16x3")
    plan = BatchPlan(Ns, Ks, 16, 1.0, seed, B1s=B1s, precision="bf16x3")
"""

import json
import math
import os
import time

from . import Plan, Sfft4Error

B_MIN, B_MAX = 16, 4096


def _pow2ceil(v):
    return 1 << max(0, int(math.ceil(math.log2(max(1, v)))))


def default_cache_path():
    return os.environ.get("SFFT4_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "sfft4_gb300", "autotune.json"))


def candidates(N, K):
    """B1 values tried for (N, K): pow2ceil(2K) x {1/4, 1/2, 1, 2} within [16, min(4096, N/64)]."""
    base = _pow2ceil(2 * K)
    hi = min(B_MAX, N // 64)
    out = []
    for f in (0.25, 0.5, 1.0, 2.0):
        b = int(base * f)
        if B_MIN <= b <= hi and b not in out:
            out.append(b)
    if not out:
        out.append(max(B_MIN, min(hi, base)))
    return out


def probe_signals(N, K, count, seed, device):
    """`count` noiseless K-sparse probe signals (unit magnitude, uniform phase, uniform support)
    synthesised on the device; returns (x (count, N) complex64, list of sorted supports)."""
    import numpy as np
    import torch
    rng = np.random.default_rng(seed)
    xs = torch.empty((count, N), dtype=torch.complex64, device=device)
    supports = []
    for i in range(count):
        f = np.sort(rng.choice(N, size=K, replace=False)).astype(np.int64)
        X = torch.zeros(N, dtype=torch.complex128, device=device)
        X[torch.from_numpy(f).to(device)] = torch.from_numpy(np.exp(2j * np.pi * rng.random(K))).to(device)
        xs[i] = (torch.fft.ifft(X) * N).to(torch.complex64)
        supports.append(f)
    return xs, supports


def saturating_batch(N):
    """Probe batch of about 2^27 samples (8 to 512 signals)."""
    return int(min(512, max(8, (1 << 27) // N)))


def tune_one(N, K, l=16, q=1.0, precision="bf16x3", device=None, batch=None, reps=3, seed=12345):
    """Time every candidate B1 of (N, K) on `batch` probe signals (default: a saturating
    batch); returns a record with the chosen B1 (0 when no candidate recovers every probe,
    i.e. keep the default)."""
    import numpy as np
    import torch
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    if batch is None:
        batch = saturating_batch(N)
    xs, supports = probe_signals(N, K, batch, seed, device)
    stream = torch.cuda.current_stream(xs.device)
    tried = []
    for b in candidates(N, K):
        try:
            p = Plan(N, K, l, q, seed=seed, B1=b, max_batch=batch, precision=precision, device=xs.device)
        except Sfft4Error:
            continue
        out = p._outputs(batch)
        p.execute_batched(xs, out)
        idx, nf = out[0].cpu().numpy(), out[2].cpu().numpy()
        ok = all(np.array_equal(idx[i, :nf[i]], supports[i]) for i in range(batch))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            p.execute_batched(xs, out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps / batch
        tried.append({"B1": b, "ms_per_transform": ms, "exact_support": ok,
                      "samples": p.info["samples_per_transform"], "iterations": p.info["n_iters"]})
        p.close()
    good = [t for t in tried if t["exact_support"]]
    best = min(good, key=lambda t: t["ms_per_transform"]) if good else None
    default = next((t for t in good if t["B1"] == _pow2ceil(2 * K)), None)
    if best is not None and default is not None and best["ms_per_transform"] > 0.97 * default["ms_per_transform"]:
        best = default
    return {"N": N, "K": K, "batch": batch, "B1": best["B1"] if best else 0, "tried": tried}


def _key(dev_name, precision, N, Kc, l, q):
    return f"{dev_name}|{precision}|N={N}|Kc={Kc}|l={l}|q={q}"


def choose_b1(Ns, Ks, l=16, q=1.0, precision="bf16x3", cache_path=None, device=None, batch=None, log=None):
    """First-iteration bucket count for every signal (list aligned with Ns), tuning each
    (N, pow2ceil(K)) class not yet in the cache with the class's largest K."""
    import torch
    device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    dev_name = torch.cuda.get_device_name(device)
    path = cache_path or default_cache_path()
    try:
        cache = json.load(open(path))
    except (OSError, ValueError):
        cache = {}
    classes = {}
    for N, K in zip(Ns, Ks):
        kc = _pow2ceil(int(K))
        classes[(int(N), kc)] = max(classes.get((int(N), kc), 0), int(K))
    t0 = time.time()
    changed = False
    for (N, kc), kmax in sorted(classes.items()):
        key = _key(dev_name, precision, N, kc, l, q)
        if key in cache:
            continue
        rec = tune_one(N, kmax, l, q, precision, device, batch=batch)
        cache[key] = rec
        changed = True
        if log is not None:
            log(key, rec)
    if changed:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, path)
    choose_b1.last_seconds = time.time() - t0
    return [cache[_key(dev_name, precision, int(N), _pow2ceil(int(K)), l, q)]["B1"] for N, K in zip(Ns, Ks)]
