"""Autotuner of the plan per (N, K class): the first-iteration bucket count B1 and the fold's
tile shape (residues per fold CTA, rounds per fold group).

B1 sets the whole static schedule (Section 3.1): more buckets isolate more coefficients per
iteration but widen the window (w ~ 44 B1 samples at delta = 1e-8) and the DFT; fewer buckets
read fewer samples per iteration but need more iterations.  The default is pow2ceil(2K).  For
each (N, pow2ceil(K)) class the tuner times the candidates pow2ceil(2K) x {1/4, 1/2, 1, 2}
(those the planner accepts) on noiseless probe signals of the class's largest K, in batches
large enough to fill the GPU (about 2^27 signal samples per execute, so the time is throughput,
not the latency of one schedule), keeps those that recover every probe's support exactly, and
picks the fastest, keeping the default unless another candidate is at least 3 % faster.
With B1 chosen, the fold's tile shape is tuned the same way, one knob after the other:
residues per fold CTA in {16, 32, 64} (the window width w follows from B and delta, so B1 also
sets w), then the most rounds one fold CTA accumulates in {4, 6, 8}; the defaults (32, 6) stay
unless another value is at least 3 % faster.  The tile shape changes the order of the fold's
sums, so outputs agree with the default's to FP32 rounding.  Choices are cached in a JSON file
keyed by device, precision, N, K class, l and q.

    from paper_2011_05698_gb300 import autotune
    B1s, residues, rounds = autotune.choose(Ns, Ks, l=16, q=1.0, precision="bf16x3")
    plan = BatchPlan(Ns, Ks, 16, 1.0, seed, B1s=B1s, precision="bf16x3",
                     fold_residues=residues, fold_rounds=rounds)
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


RESIDUES = (16, 32, 64)      # residues mod B per fold CTA; default 64
ROUNDS = (2, 3, 4)           # most rounds per fold group; default 3
DEFAULT_SHAPE = (64, 3)
# Rounds per fold group of a batch of uneven signals (the library's default for
# sfft4_plan_batched): measured on the whole 512-signal batch of N = 2^16..2^22, 6 beat 3 and
# 4 by 7-16 %, while the probe batches of a single (N, K) class prefer fewer rounds, so
# choose() keeps 6 for batches and tunes only the residues there.
BATCH_ROUNDS = 6


def _time_plan(N, K, l, q, precision, xs, supports, seed, reps, **kw):
    """(ms per transform, exact support on every probe, plan info) of one plan, or None when
    the planner rejects the options."""
    import numpy as np
    import torch
    batch = xs.shape[0]
    try:
        p = Plan(N, K, l, q, seed=seed, max_batch=batch, precision=precision, device=xs.device, **kw)
    except Sfft4Error:
        return None
    out = p._outputs(batch)
    p.execute_batched(xs, out)
    idx, nf = out[0].cpu().numpy(), out[2].cpu().numpy()
    ok = all(np.array_equal(idx[i, :nf[i]], supports[i]) for i in range(batch))
    stream = torch.cuda.current_stream(xs.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        p.execute_batched(xs, out)
    e1.record(stream)
    torch.cuda.synchronize()
    info = dict(p.info)
    p.close()
    return e0.elapsed_time(e1) / reps / batch, ok, info


def _pick(tried, is_default):
    """The fastest exact candidate, unless the default is within 3 % of it."""
    good = [t for t in tried if t["exact_support"]]
    if not good:
        return None
    best = min(good, key=lambda t: t["ms_per_transform"])
    default = next((t for t in good if is_default(t)), None)
    if default is not None and best["ms_per_transform"] > 0.97 * default["ms_per_transform"]:
        return default
    return best


def tune_one(N, K, l=16, q=1.0, precision="bf16x3", device=None, batch=None, reps=3, seed=12345, shape=True):
    """Time every candidate B1 of (N, K) on `batch` probe signals (default: a saturating
    batch), then (shape=True) the fold tile shapes with the chosen B1; returns a record with
    the chosen B1 (0 when no candidate recovers every probe, i.e. keep the default) and the
    chosen residues per fold CTA and rounds per fold group."""
    import torch
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    if batch is None:
        batch = saturating_batch(N)
    xs, supports = probe_signals(N, K, batch, seed, device)
    tried = []
    for b in candidates(N, K):
        r = _time_plan(N, K, l, q, precision, xs, supports, seed, reps, B1=b)
        if r is None:
            continue
        ms, ok, info = r
        tried.append({"B1": b, "ms_per_transform": ms, "exact_support": ok,
                      "samples": info["samples_per_transform"], "iterations": info["n_iters"]})
    best = _pick(tried, lambda t: t["B1"] == _pow2ceil(2 * K))
    rec = {"N": N, "K": K, "batch": batch, "B1": best["B1"] if best else 0, "tried": tried,
           "fold_residues": DEFAULT_SHAPE[0], "fold_rounds": DEFAULT_SHAPE[1], "tried_shape": []}
    if not shape:
        return rec
    res, rnd = DEFAULT_SHAPE
    for knob, values in (("fold_residues", RESIDUES), ("fold_rounds", ROUNDS)):
        tr = []
        for v in values:
            kw = {"fold_residues": res, "fold_rounds": rnd}
            kw[knob] = v
            r = _time_plan(N, K, l, q, precision, xs, supports, seed, reps, B1=rec["B1"], **kw)
            if r is None:
                continue
            tr.append({**kw, "ms_per_transform": r[0], "exact_support": r[1]})
        pick = _pick(tr, lambda t: t[knob] == DEFAULT_SHAPE[0 if knob == "fold_residues" else 1])
        if pick is not None:
            res, rnd = pick["fold_residues"], pick["fold_rounds"]
        rec["tried_shape"].extend(tr)
    rec["fold_residues"], rec["fold_rounds"] = res, rnd
    return rec


def _key(dev_name, precision, N, Kc, l, q):
    return f"v2|{dev_name}|{precision}|N={N}|Kc={Kc}|l={l}|q={q}"


def _records(Ns, Ks, l, q, precision, cache_path, device, batch, log, shape_of_top=False):
    """The cached (or newly tuned) record of every (N, pow2ceil(K)) class of the batch, tuning
    the B1 of each class not yet in the cache with its largest K, and (shape_of_top) the fold
    tile shape of the class carrying the most samples; returns (records by class, key of a
    signal)."""
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
    weight = {}
    for N, K in zip(Ns, Ks):
        c = (int(N), _pow2ceil(int(K)))
        weight[c] = weight.get(c, 0) + int(N)
    top = max(weight, key=weight.get)
    t0 = time.time()
    changed = False
    for (N, kc), kmax in sorted(classes.items()):
        key = _key(dev_name, precision, N, kc, l, q)
        need_shape = shape_of_top and (N, kc) == top
        if key in cache and (not need_shape or cache[key].get("shape_tuned")):
            continue
        rec = tune_one(N, kmax, l, q, precision, device, batch=batch, shape=need_shape)
        rec["shape_tuned"] = need_shape
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
    _records.last_seconds = time.time() - t0
    return cache, lambda N, K: _key(dev_name, precision, int(N), _pow2ceil(int(K)), l, q)


def choose_b1(Ns, Ks, l=16, q=1.0, precision="bf16x3", cache_path=None, device=None, batch=None, log=None):
    """First-iteration bucket count for every signal (list aligned with Ns)."""
    cache, key = _records(Ns, Ks, l, q, precision, cache_path, device, batch, log)
    choose_b1.last_seconds = _records.last_seconds
    return [cache[key(N, K)]["B1"] for N, K in zip(Ns, Ks)]


def choose(Ns, Ks, l=16, q=1.0, precision="bf16x3", cache_path=None, device=None, batch=None, log=None):
    """(B1 per signal, residues per fold CTA, rounds per fold group) for a batch: the fold's
    tile shape is an option of the whole batch, so the residues are those tuned for the class
    that carries the most samples (signals x N), and the rounds per group BATCH_ROUNDS."""
    cache, key = _records(Ns, Ks, l, q, precision, cache_path, device, batch, log, shape_of_top=True)
    choose.last_seconds = _records.last_seconds
    weight = {}
    for N, K in zip(Ns, Ks):
        weight[key(N, K)] = weight.get(key(N, K), 0) + int(N)
    top = cache[max(weight, key=weight.get)]
    return ([cache[key(N, K)]["B1"] for N, K in zip(Ns, Ks)],
            int(top.get("fold_residues", DEFAULT_SHAPE[0])), BATCH_ROUNDS)
