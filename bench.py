"""Throughput benchmark of the sFFT4.0 hot path on GB300.

A step is one batched sFFT4.0 pass (all iterations: permuted gather + window + fold,
B-point DFT, update, selection, multiscale location, votes, median estimation, merge,
top-K) over a batch of synthetic signals of the metric's configuration: N = 2^22,
K = 1000 unit-magnitude uniform-phase coefficients at uniform random frequencies, time-domain
white noise at 20 dB SNR.  Inputs live in HBM before the timed region; the touched sample
set of a step (several GB) is far larger than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With N > 1 (torchrun, one process per GPU) every rank transforms its
own batch (replicas, weak scaling); rank 0 prints.  --impl reference times the FP64 CPU
oracle on the host cores instead.
"""

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "sFFT4.0 transforms/s N=2^22 K=1000, batched split-precision vs plain FP32"
N_DEF, K_DEF, L_DEF, Q_DEF, SNR_DEF = 2**22, 1000, 16, 1.0, 20.0
WORKLOAD = "precision form: N=2^22 K=1000, unit-magnitude uniform-phase uniform-support spectra, SNR 20 dB"


# --------------------------------------------------------------------------- CPU oracle
def _oracle_one(args):
    """One oracle transform (runs in a spawned worker; imports only the oracle): its time and
    its results (nfound, frequencies, values, votes)."""
    N, K, l, q, seed, snr, signal, plan_seed = args
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import plan as OP, sfft4 as O
    from synth import sparse_signal
    sig = sparse_signal(N, K, seed, snr)
    pseed = seed if plan_seed is None else plan_seed
    t0 = time.perf_counter()
    r = O.run(sig.x.astype(np.complex128), OP.make_plan(N, K, l, q, seed=pseed), signal=signal)
    return time.perf_counter() - t0, int(r["nfound"]), r["f"], r["v"], r["votes"]


def oracle_sample(pool, n, N, K, l, q, snr, seed0, plan_seed=None):
    """n oracle transforms on the pool's workers (one each at a time): signal i synthesised
    from seed seed0 + i and transformed as batch index i of a plan seeded plan_seed (default:
    the signal's own seed).  Returns the oracle's throughput -- the sum over transforms of
    1 / (seconds of its O.run), i.e. the rate of the workers running side by side, signal
    synthesis excluded -- and the per-transform results."""
    res = pool.map(_oracle_one, [(N, K, l, q, seed0 + i, snr, i, plan_seed) for i in range(n)])
    rate = sum(1.0 / max(r[0], 1e-9) for r in res)
    return rate, res


def accuracy_vs_oracle(s4, res, n, snr, seed0, plan_seed, dev):
    """The GPU path's results against the oracle's on the same n signals of the workload (the
    oracle sample of cpu_baseline, run as batch indices 0..n-1 of a plan seeded plan_seed):
    per precision, how many supports and vote lists are identical, and the values' relative
    l2 error where the support is."""
    import numpy as np
    import torch
    from synth import sparse_signal
    xs = torch.from_numpy(np.stack([sparse_signal(N_DEF, K_DEF, seed0 + i, snr).x for i in range(n)])).to(dev)
    out = {"signals": n, "snr_db": snr,
           "bar": "support and votes identical up to decisions within a fragile margin (replay-explained in "
                  "the parity tests); values within 1e-4 relative l2 at 20 dB"}
    for prec in ("bf16x3", "fp32"):
        p = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=plan_seed, max_batch=n, precision=prec)
        idx, val, nf, votes = [t.cpu().numpy() for t in p.execute_batched(xs)]
        p.close()
        sup = vot = 0
        rels = []
        for i, (_, _, f, v, vt) in enumerate(res):
            k = int(nf[i])
            if np.array_equal(idx[i, :k], f):
                sup += 1
                vot += int(np.array_equal(votes[i, :k], vt))
                rels.append(float(np.linalg.norm(val[i, :k] - v) / max(float(np.linalg.norm(v)), 1e-300)))
        out[prec] = {"support_identical": sup, "votes_identical": vot,
                     "value_rel_l2_max": max(rels) if rels else None,
                     "value_rel_l2_median": statistics.median(rels) if rels else None}
    return out


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def make_pool(workers):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(workers)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def reference_arm(args, rank, world):
    """The FP64 oracle on the host cores, each step a bounded sample of the workload."""
    if rank != 0:
        return
    workers = host_cores()
    pool = make_pool(workers)
    for w in range(args.warmup):
        oracle_sample(pool, workers, N_DEF, K_DEF, L_DEF, Q_DEF, args.snr, 10_000 + w * workers)
    rates = []
    for k in range(args.steps):
        rate, _ = oracle_sample(pool, workers, N_DEF, K_DEF, L_DEF, Q_DEF, args.snr, 20_000 + k * workers)
        rates.append(rate)
    pool.close()
    value = statistics.mean(rates)
    tot = workers * args.steps / value
    sample = (f"{workers} transforms per step, one per worker process on {workers} host cores "
              f"({cpu_model()}), FP64 numpy oracle; rate = sum of 1 / (seconds of each O.run), "
              "signal synthesis excluded")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "transforms/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N_DEF, "K": K_DEF, "l": L_DEF, "q": Q_DEF,
                       "snr_db": args.snr, "parallelism": f"{workers} host processes"},
            "cpu_baseline": {"value": value, "unit": "transforms/s", "cores": workers, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.p is not None:
            time.sleep(0.2)
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def fold_source_sha256():
    """sha256 of what sets the fold's DRAM traffic: kernels.cu from its fold section header
    up to the FFT section header and the signal-major launch builder; from plan.cu the round
    segments (build_group), the fold groups, residue slices and copies of each iteration, and
    the lines that set the L2 fetch granularity."""
    csrc = os.path.join(ROOT, "paper_2011_05698_gb300", "csrc")
    src = open(os.path.join(csrc, "kernels.cu")).read()
    a = src.index("// ----------------------------------------------------------------- fold")
    b = src.index("// ----------------------------------------------------------------- FFT")
    c = src.index("int build_signal_major_fold(")
    d = src.index("int launch_fft_multi(")
    plan = open(os.path.join(csrc, "plan.cu")).read()
    e = plan.index("void build_group(")
    f = plan.index("\n}\n", e)
    g = plan.index("// fold groups of up to kFoldRG rounds")
    h = plan.index("p->samples += ih.unique;", g)
    fetch = "".join(ln for ln in plan.splitlines(True) if "L2Fetch" in ln or "l2_fetch_bytes" in ln)
    return hashlib.sha256((src[a:b] + src[c:d] + plan[e:f] + plan[g:h] + fetch).encode()).hexdigest()


def fold_traffic_record():
    """DRAM bytes per fold launch from the committed ncu summary, if the fold kernel's source
    is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "fold_traffic.json")
    try:
        rec = json.load(open(path))
        if rec.get("fold_source_sha256") != fold_source_sha256():
            return None
        return rec
    except (OSError, ValueError):
        return None


def gather_sweep(s4, xs, sm_count, footprints, inflights=(4, 8, 16), fetches=(32, 64, 128),
                 shapes=((256, 2), (256, 4), (256, 8), (512, 1), (512, 2), (512, 4), (1024, 1), (1024, 2)),
                 loads=150_000_000):
    """Random 8-byte loads per second of sfft4_gather_probe_ex over a grid: footprint (rows of
    xs read side by side, nsig x N x 8 bytes), loads in flight per thread, L2 fetch granularity,
    (threads per CTA, CTAs per SM).  Returns the list of points, each with its rate."""
    pts = []
    for nsig in footprints:
        x = xs[:nsig]
        for inf in inflights:
            for fb in fetches:
                for th, cps in shapes:
                    blocks = sm_count * cps
                    iters = max(1, loads // (blocks * th * inf))
                    lps = s4.gather_probe(x, blocks=blocks, iters=iters, threads=th, inflight=inf, l2_fetch_bytes=fb)
                    pts.append({"nsig": nsig, "footprint_mb": nsig * x.shape[1] * 8 / 2**20, "inflight": inf,
                                "l2_fetch_bytes": fb, "threads": th, "ctas_per_sm": cps, "gloads_s": lps / 1e9})
    return pts


def gather_ceiling_form(s4, dev):
    """Sweep of the random-gather probe: footprints from one L2-resident 32 MB signal to 64
    signals (2 GB), 4/8/16 loads in flight per thread, 32/64/128-byte L2 fetches, 256-1024
    threads per CTA and 1-8 CTAs per SM.  Reports every point and the best per footprint."""
    import torch
    from synth.signals import device_signal
    N, S = N_DEF, 64
    xs = torch.empty((S, N), dtype=torch.complex64, device=dev)
    for i in range(S):
        device_signal(N, K_DEF, 5000 + i, None, dev, out=xs[i])
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    pts = gather_sweep(s4, xs, sm, (1, 2, 4, 16, 64))
    best = {}
    for pt in pts:
        b = best.get(pt["nsig"])
        if b is None or pt["gloads_s"] > b["gloads_s"]:
            best[pt["nsig"]] = pt
    return {"form": "gather_ceiling", "N": N, "sm_count": sm, "points": pts,
            "best_per_footprint": [best[k] for k in sorted(best)]}


def device_batch(N, K, S, seed0, snr, device):
    """Seeded synthetic batch synthesised on the device (spectra drawn by synth)."""
    import torch
    from synth.signals import device_signal
    xs = torch.empty((S, N), dtype=torch.complex64, device=device)
    for i in range(S):
        device_signal(N, K, seed0 + i, snr, device, out=xs[i])
    return xs


def uneven_form(s4, args, dev, stream, dist):
    """The uneven batch: 512 signals, N log-uniform over 2^16..2^22, K log-uniform in
    [10, 2000] capped at N/64, SNR uniform in [10, 40] dB; one BatchPlan execute per step,
    replayed as a CUDA graph, BF16x3 DFT, asynchronous (consecutive steps overlap; the
    synchronous form is reported beside it).  Kernel times come from a second, profiled plan."""
    import torch
    from synth.signals import device_signal, signal_seed, uneven_sizes
    nsig, seed = args.uneven_signals, 2026
    Ns, Ks, snrs = uneven_sizes(nsig, seed)
    xs = [device_signal(int(Ns[i]), int(Ks[i]), signal_seed(seed, i), snrs[i], dev)[0] for i in range(nsig)]
    graph = not args.no_graph
    B1s, tune = None, None
    f_res = f_rnd = 0
    if not args.no_autotune:
        import collections
        import tempfile
        from paper_2011_05698_gb300 import autotune
        cache = os.path.join(tempfile.gettempdir(), "sfft4_autotune_bench.json")
        B1s, f_res, f_rnd = autotune.choose(Ns.tolist(), Ks.tolist(), L_DEF, Q_DEF, precision=args.precision,
                                            cache_path=cache, device=dev)
        ratio = collections.Counter()
        for b, k in zip(B1s, Ks.tolist()):
            ratio[f"{b / autotune._pow2ceil(2 * k):g}" if b else "default"] += 1
        tune = {"seconds": autotune.choose.last_seconds, "cache": cache,
                "B1_over_pow2ceil_2K": dict(ratio), "fold_residues": f_res, "fold_rounds": f_rnd}
    bp = s4.BatchPlan(Ns.tolist(), Ks.tolist(), L_DEF, Q_DEF, seed=seed, precision=args.precision, graph=graph,
                      B1s=B1s, fold_residues=f_res, fold_rounds=f_rnd)
    out = bp.outputs()
    outs = [out, bp.outputs(), bp.outputs()]  # one per batch in flight
    ptrs = bp.pointers(xs)
    pipelined = not args.no_async
    counter = [0]

    def step():
        # pipelined: asynchronous executes, three workspaces in turn (the decode chains of
        # two batches overlap each other and the next batch's gathers)
        if pipelined:
            bp.execute(xs, out=outs[counter[0] % len(outs)], ptrs=ptrs, asynchronous=True)
            counter[0] += 1
        else:
            bp.execute(xs, out=out, ptrs=ptrs)

    steps = max(3, min(args.steps, 20))
    el = max_over_ranks(timed(step, steps, args.warmup, stream, dist, finish=bp.wait if pipelined else None),
                        dist, dev)
    world = dist.get_world_size() if dist is not None else 1
    info = dict(bp.info)
    sync = None
    if pipelined:
        es = max_over_ranks(timed(lambda: bp.execute(xs, out=out, ptrs=ptrs), steps, 2, stream, dist), dist, dev)
        sync = {"value": nsig * steps * world / es, "ms_per_step": 1e3 * es / steps,
                "form": "one synchronous execute per step (graph replay)" if graph else "one synchronous execute per step"}
    bp.close()
    # the same launches issued directly (no graph), for comparison
    direct = None
    if graph:
        bd = s4.BatchPlan(Ns.tolist(), Ks.tolist(), L_DEF, Q_DEF, seed=seed, precision=args.precision, B1s=B1s,
                          fold_residues=f_res, fold_rounds=f_rnd)
        outd = bd.outputs()
        ptrd = bd.pointers(xs)
        ed = max_over_ranks(timed(lambda: bd.execute(xs, out=outd, ptrs=ptrd), steps, args.warmup, stream, dist),
                            dist, dev)
        direct = {"value": nsig * steps * world / ed, "ms_per_step": 1e3 * ed / steps}
        bd.close()
    bq = s4.BatchPlan(Ns.tolist(), Ks.tolist(), L_DEF, Q_DEF, seed=seed, precision=args.precision, profile=True,
                      B1s=B1s, fold_residues=f_res, fold_rounds=f_rnd)
    outq = bq.outputs()
    bq.execute(xs, out=outq)
    torch.cuda.synchronize()
    bq.profile(reset=True)
    bq.execute(xs, out=outq)
    prof = bq.profile(reset=True)
    bq.close()
    fold_gbs = 8.0 * prof["fold_samples"] / (prof["fold_ms"] / 1e3) / 1e9 if prof["fold_ms"] > 0 else None
    return {"value": nsig * steps * world / el, "unit": "transforms/s", "ms_per_step": 1e3 * el / steps,
            "steps": steps, "signals": nsig, "precision": args.precision, "graph": graph,
            "samples_per_step": info["samples_per_execute"], "kernels_per_step": info["kernels_per_execute"],
            "graph_launches_per_step": 1 if graph else 0, "levels": info["n_levels"], "classes": info["n_classes"],
            "workload": "512 signals: N=2^n, n uniform on 16..22; K=round(exp U[ln 10, ln 2000]) <= N/64; "
                        "SNR U[10, 40] dB; l=16, q=1",
            "pipelined": pipelined, "synchronous": sync,
            "fold_gbs_useful": fold_gbs, "autotune": tune, "direct_launches": direct,
            "kernel_ms_one_execute": {k: prof[k + "_ms"] for k in ("fold", "fft", "decode", "finalize")}}


def phase_errors(Y, freqs, sigma, N, B, taus):
    """Phase errors |dPhi| (radians) of the levels s = 1..S for every tone alone in its bucket
    neighbourhood: dPhi = wrap(arg(y_s[b] conj(y_0[b])) - 2 pi (u tau_s mod N) / N), u = sigma f
    mod N, b = bucket of u (the location's phase measurement, Section 3.2, Eq. 16-19)."""
    import numpy as np
    L = N // B
    u = (sigma * freqs.astype(np.uint64)) & np.uint64(N - 1)
    b = (((u + np.uint64(L // 2)) // np.uint64(L)) % np.uint64(B)).astype(np.int64)
    occ = np.bincount(b, minlength=B)
    near = occ + np.roll(occ, 1) + np.roll(occ, -1)
    alone = near[b] == 1
    out = []
    for s_ in range(1, len(taus)):
        ideal = ((u[alone] * np.uint64(taus[s_])) & np.uint64(N - 1)).astype(np.float64) / N
        meas = np.angle(Y[s_, b[alone]] * np.conj(Y[0, b[alone]])) / (2 * np.pi)
        d = (meas - ideal + 0.5) % 1.0 - 0.5
        out.append(np.abs(d) * 2 * np.pi)
    return np.concatenate(out) if out else np.zeros(0)


def phase_error_form(s4, args, dev):
    """Monte Carlo of the location's phase error (Section 3.2, Fig. 5): K = 50 tones, SNR in
    {-20, -10, 0, 20, 40, 60, 120} dB, bucket lengths L = N / B from 128 to 8192; iteration-1
    bucket arrays of the library (sfft4_bucketize), 64 signals per point.  Reports quantiles of
    |dPhi| and the bounds they imply: l <= pi / max dPhi (Eq. 18), q >= max dPhi l / pi (Eq. 19),
    with max dPhi the 0.99 quantile."""
    import numpy as np
    from synth.signals import device_signal
    K, trials = 50, 64
    rows = []
    for N, B in ((2**13, 64), (2**17, 64), (2**20, 512), (2**22, 512)):
        p = s4.Plan(N, K, 16, 1.0, seed=99, B1=B)
        it = p.iter_info(1)
        for snr in (-20.0, -10.0, 0.0, 20.0, 40.0, 60.0, 120.0):
            errs = []
            for t in range(trials):
                x, f, _ = device_signal(N, K, 40_000 + t, snr, dev)
                Y = p.bucketize(x, 1, signal=t).cpu().numpy().astype(np.complex128)
                sigma, _ = p.permutation(1, signal=t)
                errs.append(phase_errors(Y, f, np.uint64(sigma), N, B, it["tau"]))
            e = np.concatenate(errs)
            q99 = float(np.quantile(e, 0.99))
            rows.append({"N": N, "B": B, "L": N // B, "snr_db": snr, "samples": int(e.size),
                         "median_rad": float(np.median(e)), "q99_rad": q99,
                         "log10_q99": float(np.log10(max(q99, 1e-300))),
                         "l_upper_bound": float(np.pi / q99) if q99 > 0 else None,
                         "q_lower_bound_at_l16": float(q99 * 16 / np.pi)})
        p.close()
    return {"form": "phase_error", "K": K, "trials": trials, "data": "synthetic", "rows": rows}


def configs_form(s4, args, dev, stream):
    """The small single-signal configurations over 10 seeds each: N = 2^14, K = 16 (l = 4,
    q = 0.5, B1 = 64, noiseless) and N = 2^20, K = 100 (l = 16, q = 1, B1 = 128, 20 dB), plus
    N = 2^22, K = 1000 at 20 dB: plain FP32 form (one execute per signal), batched BF16x3 form
    (the 10 seeds in one execute, and 256 signals per execute for throughput), exact-support
    rate and error against the generator, samples per transform."""
    import numpy as np
    import torch
    from synth.signals import device_signal
    cfgs = [("N=2^14 K=16 l=4 q=0.5 B1=64 noiseless", 2**14, 16, 4, 0.5, 64, None),
            ("N=2^20 K=100 l=16 q=1 B1=128 20 dB", 2**20, 100, 16, 1.0, 128, 20.0),
            ("N=2^22 K=1000 l=16 q=1 20 dB", 2**22, 1000, 16, 1.0, 0, 20.0)]
    out_rows = []
    for name, N, K, l, q, B1, snr in cfgs:
        S = 10
        xs = torch.empty((S, N), dtype=torch.complex64, device=dev)
        truth = [device_signal(N, K, 3000 + i, snr, dev, out=xs[i])[1:] for i in range(S)]
        row = {"config": name, "seeds": S}
        for form, prec in (("plain_fp32", "fp32"), ("batched_bf16x3", "bf16x3")):
            p = s4.Plan(N, K, l, q, seed=21, B1=B1, max_batch=256, precision=prec)
            if form == "plain_fp32":
                res = [p._outputs(1) for _ in range(S)]

                def fn():
                    for i in range(S):
                        p.execute(xs[i], res[i])
                el = timed(fn, 5, 2, stream, None)
                got = [(r[0][0, :int(r[2][0])].cpu().numpy(), r[1][0, :int(r[2][0])].cpu().numpy()) for r in res]
                tps = S * 5 / el
            else:
                o = p._outputs(S)
                el = timed(lambda: p.execute_batched(xs, o), 5, 2, stream, None)
                idx, val, nf = o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy()
                got = [(idx[i, :nf[i]], val[i, :nf[i]]) for i in range(S)]
                tps = S * 5 / el
                big = xs.repeat((256 + S - 1) // S, 1)[:256].contiguous()
                ob = p._outputs(256)
                eb = timed(lambda: p.execute_batched(big, ob), 5, 2, stream, None)
                row["batched_bf16x3_256_per_execute"] = {"transforms_per_s": 256 * 5 / eb}
                del big
            ok, errs = 0, []
            for (fi, vi), (ft, vt) in zip(got, truth):
                ok += int(np.array_equal(fi, ft))
                est = dict(zip(fi.tolist(), vi.tolist()))
                tru = dict(zip(ft.tolist(), vt.tolist()))
                allf = sorted(set(est) | set(tru))
                errs.append(sum(abs(est.get(f, 0) - tru.get(f, 0)) for f in allf) / K)
            row[form] = {"transforms_per_s": tps, "exact_support_rate": ok / S, "l1_error_mean": float(np.mean(errs)),
                         "samples_per_transform": p.info["samples_per_transform"],
                         "samples_frac_of_N": p.info["samples_per_transform"] / N, "iterations": p.info["n_iters"]}
            p.close()
        out_rows.append(row)
    return {"form": "configs", "data": "synthetic", "rows": out_rows}


def sweep_form(s4, args, dev, stream):
    """Large-N sweep: N = 2^26, K = 4000, SNR in {0, 10, 20, 30, 40} dB, l in {4, 8, 16, 32} x
    q in {0.5, 1, 1.5, 2}; per point: runtime of the batched split-precision form (one execute
    of all seeds) and of the plain FP32 form (one execute per signal), samples touched, and
    exact-support success and L1 error of both over the seeds."""
    import numpy as np
    import torch
    from synth.signals import device_signal
    N, K, S = 2**26, 4000, args.sweep_seeds
    xs = torch.empty((S, N), dtype=torch.complex64, device=dev)
    supp = []
    rows = []
    for snr in (0.0, 10.0, 20.0, 30.0, 40.0):
        supp = []
        for i in range(S):
            _, f, v = device_signal(N, K, 9000 + i, snr, dev, out=xs[i])
            supp.append((f, v))
        for l in (4, 8, 16, 32):
            for q in (0.5, 1.0, 1.5, 2.0):
                row = {"snr_db": snr, "l": l, "q": q}
                for form, prec, batched in (("batched_bf16x3", "bf16x3", True), ("plain_fp32", "fp32", False)):
                    p = s4.Plan(N, K, l, q, seed=77, max_batch=S if batched else 1, precision=prec)
                    if batched:
                        out = p._outputs(S)
                        fn = (lambda: p.execute_batched(xs, out))
                    else:
                        out1 = p._outputs(1)
                        res = [p._outputs(1) for _ in range(S)]

                        def fn():
                            for i in range(S):
                                p.execute(xs[i], res[i])
                    el = timed(fn, 3, 1, stream, None)
                    if batched:
                        idx, val, nf = out[0].cpu().numpy(), out[1].cpu().numpy(), out[2].cpu().numpy()
                        got = [(idx[i, :nf[i]], val[i, :nf[i]]) for i in range(S)]
                    else:
                        got = [(r[0][0, :int(r[2][0])].cpu().numpy(), r[1][0, :int(r[2][0])].cpu().numpy()) for r in res]
                        del out1
                    ok, l1 = 0, []
                    for (fi, vi), (ft, vt) in zip(got, supp):
                        ok += int(np.array_equal(fi, ft))
                        allf = np.union1d(fi, ft)
                        est = dict(zip(fi.tolist(), vi.tolist()))
                        tru = dict(zip(ft.tolist(), vt.tolist()))
                        l1.append(sum(abs(est.get(f, 0) - tru.get(f, 0)) for f in allf.tolist()) / K)
                    row[form] = {"ms_per_transform": 1e3 * el / 3 / S, "success": ok / S,
                                 "l1_error_mean": float(np.mean(l1)),
                                 "samples_per_transform": p.info["samples_per_transform"],
                                 "samples_frac_of_N": p.info["samples_per_transform"] / N,
                                 "iterations": p.info["n_iters"]}
                    p.close()
                rows.append(row)
    return {"form": "large_n_sweep", "N": N, "K": K, "seeds": S, "data": "synthetic",
            "workload": "N=2^26 K=4000 unit-magnitude uniform-phase spectra, time-domain noise at the "
                        "stated SNR; plain form: one sfft4_execute per signal (Philox signal 0); "
                        "batched form: one sfft4_execute_batched of all seeds",
            "rows": rows}


# --------------------------------------------------------------------------- ranks
def init_ranks(backend="nccl"):
    """(rank, world, local_rank, dist) from the torchrun environment; dist is the initialised
    torch.distributed module when world > 1, else None."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group(backend)
        dist = tdist
    return rank, world, local, dist


def max_over_ranks(x, dist, device):
    """The maximum of x over all ranks (x itself on one rank)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed0(rank):
    """First signal seed of a rank's batch: replicas transform disjoint synthetic batches."""
    return 1_000_000 * (rank + 1)


def timed(fn, steps, warmup, stream, dist=None, finish=None):
    """Seconds of `steps` calls of fn between CUDA events on `stream` (finish() is issued
    after the last call, before the closing event: it joins work fn left on other streams)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    if finish is not None:
        finish()
    e1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return e0.elapsed_time(e1) / 1e3


# --------------------------------------------------------------------------- main arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--snr", type=float, default=SNR_DEF)
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "bf16x3"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--plain-signals", type=int, default=16)
    ap.add_argument("--uneven-signals", type=int, default=512)
    ap.add_argument("--no-fp32-form", action="store_true")
    ap.add_argument("--fold-order", default="signal_major", choices=["signal_major", "iteration_major"],
                    help="fold order of the headline plan")
    ap.add_argument("--no-async", action="store_true",
                    help="headline steps as synchronous executes (no overlap between batches)")
    ap.add_argument("--form", default="all", choices=["all", "uneven", "sweep", "configs", "phase_error",
                                                      "gather_ceiling"],
                    help="uneven: time only the uneven-batch form; sweep: the large-N SNR x (l, q) "
                         "sweep (N = 2^26, K = 4000, 10 seeds)")
    ap.add_argument("--sweep-seeds", type=int, default=10)
    ap.add_argument("--no-graph", action="store_true", help="uneven form without CUDA-graph replay")
    ap.add_argument("--no-autotune", action="store_true", help="uneven form with the default B1 per signal")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    # the oracle pool starts (spawn) before the first CUDA call
    pool = None
    cpu_workers = host_cores()
    if rank == 0 and not args.no_cpu and args.form == "all":
        pool = make_pool(cpu_workers)

    import torch
    rank, world, local, dist = init_ranks("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2011_05698_gb300 import build
    build.build()
    import paper_2011_05698_gb300 as s4

    if args.form == "phase_error":
        if rank == 0:
            print(json.dumps(phase_error_form(s4, args, dev)), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.form == "gather_ceiling":
        if rank == 0:
            print(json.dumps(gather_ceiling_form(s4, dev)), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.form == "configs":
        if rank == 0:
            print(json.dumps(configs_form(s4, args, dev, torch.cuda.current_stream(dev))), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.form == "sweep":
        if rank == 0:
            print(json.dumps(sweep_form(s4, args, dev, torch.cuda.current_stream(dev))), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    if args.form == "uneven":
        u = uneven_form(s4, args, dev, torch.cuda.current_stream(dev), dist)
        if rank == 0:
            print(json.dumps({"form": "uneven_batch", **u}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return

    S = args.batch
    plan = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=1234, max_batch=S, profile=True,
                   precision=args.precision, fold_order=args.fold_order)
    xs = device_batch(N_DEF, K_DEF, S, rank_seed0(rank), args.snr, dev)
    out = plan._outputs(S)
    outs = [out, plan._outputs(S)]  # one per batch in flight
    stream = torch.cuda.current_stream(dev)
    pipelined = not args.no_async
    counter = [0]

    def step():
        # one batch per step; pipelined: asynchronous executes (two workspaces in turn), so
        # the decode chain of one batch overlaps the gather of the next
        if pipelined:
            plan.execute_batched(xs, outs[counter[0] % len(outs)], asynchronous=True)
            counter[0] += 1
        else:
            plan.execute_batched(xs, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.profile(reset=True)
    with ClockSampler(local) as clk:
        el = timed(step, args.steps, 0, stream, dist, finish=plan.wait if pipelined else None)
    prof = plan.profile(reset=True)
    el = max_over_ranks(el, dist, dev)
    value = S * args.steps * world / el
    ms_per_step = 1e3 * el / args.steps
    # the same batches one synchronous execute at a time (each step's results complete on
    # the caller's stream before the next starts)
    sync_form = None
    if pipelined:
        ksync = max(3, min(args.steps, 30))
        el_s = timed(lambda: plan.execute_batched(xs, out), ksync, 2, stream, dist)
        el_s = max_over_ranks(el_s, dist, dev)
        sync_form = {"value": S * ksync * world / el_s, "ms_per_step": 1e3 * el_s / ksync,
                     "form": "one synchronous execute per step"}
        plan.profile(reset=True)

    # dominant kernel: the permuted gather + window + fold
    peak, peak_kind = measured_peaks()
    fold_s = prof["fold_ms"] / 1e3
    bytes_alg = 8.0 * prof["fold_samples"]
    achieved = bytes_alg / fold_s / 1e9 if fold_s > 0 else 0.0
    tr = fold_traffic_record()
    launches = max(1, prof["fold_launches"])
    traffic = None
    if tr is not None:
        traffic = tr["dram_bytes_per_sample"] * prof["fold_samples"] / launches
    # achievable rate of the gather's access pattern (random 8-byte loads inside each signal
    # of this same batch, footprint far above L2), measured on this device: the best point of
    # a sweep of loads in flight, L2 fetch granularity and CTA shape
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sweep = gather_sweep(s4, xs, sm_count, (S,))
    best_pt = max(sweep, key=lambda q: q["gloads_s"])
    gather_lps = best_pt["gloads_s"] * 1e9
    gather_ceiling = 32.0 * gather_lps / 1e9  # GB/s of 32-byte sectors
    sector_gbs = 4.0 * achieved
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "k_fold (permuted gather + window + fold)",
                "per_unit": "8 B per distinct sample read (complex64)",
                "sector_frac": 4.0 * achieved / peak, "peak_kind": peak_kind,
                "random_gather_ceiling_gbs": gather_ceiling,
                "random_gather_ceiling_point": best_pt,
                "fold_gsamples_s": prof["fold_samples"] / fold_s / 1e9 if fold_s > 0 else None,
                "frac_of_random_gather_ceiling": sector_gbs / gather_ceiling if gather_ceiling > 0 else None,
                "fold_share_of_step": prof["fold_ms"] / (1e3 * el) if el > 0 else None,
                "kernel_ms": {k: prof[k + "_ms"] for k in ("fold", "fft", "decode", "finalize")}}

    # end-to-end through the public API with pinned host buffers: sfft4_execute_batched_host
    # stages each step's batch from host memory (the library's zero-copy kernel), executes it
    # and copies its results back to pinned host outputs; consecutive steps overlap (two
    # workspaces), so one batch crosses the host link while the previous one computes
    e2e = None
    if not args.no_e2e:
        Se = min(S, 64)
        plan_e = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=1234, max_batch=Se, precision=args.precision)
        host_x = [torch.empty((Se, N_DEF), dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        host_x[0].copy_(xs[:Se].cpu())
        host_x[1].copy_(xs[Se:2 * Se].cpu() if S >= 2 * Se else xs[:Se].flip(0).cpu())
        host_o = [plan_e.host_outputs(Se) for _ in range(2)]
        counter = [0]

        def step_e2e():
            b = counter[0] % 2
            plan_e.execute_batched_host(host_x[b], host_o[b])
            counter[0] += 1

        esteps = max(3, min(args.steps, 20))
        for _ in range(2):
            step_e2e()
        plan_e.wait()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(esteps):
            step_e2e()
        plan_e.wait()
        e1.record(stream)
        torch.cuda.synchronize()
        ee = max_over_ranks(e0.elapsed_time(e1) / 1e3, dist, dev)
        h2d = Se * N_DEF * 8
        d2h = sum(t.numel() * t.element_size() for t in host_o[0])
        # the host -> device link alone: the same pinned batch copied with nothing beside it
        dx = torch.empty((Se, N_DEF), dtype=torch.complex64, device=dev)
        copy_stream = torch.cuda.Stream(dev)
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        link_s = []
        for _ in range(3):
            l0.record(copy_stream)
            with torch.cuda.stream(copy_stream):
                dx.copy_(host_x[0], non_blocking=True)
            l1.record(copy_stream)
            l1.synchronize()
            link_s.append(l0.elapsed_time(l1) / 1e3)
        link_gbs = h2d / min(link_s) / 1e9
        # for comparison: the same steps with copy-engine transfers (torch copies on a copy
        # stream, double-buffered) feeding sfft4_execute_batched
        dxs = [dx, torch.empty_like(dx)]
        oute = plan_e._outputs(Se)
        host_o2 = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in oute] for _ in range(2)]
        copied = [torch.cuda.Event() for _ in range(2)]
        free = [torch.cuda.Event() for _ in range(2)]
        for e in free:
            e.record(stream)

        def issue_copy(i):
            b = i % 2
            copy_stream.wait_event(free[b])
            with torch.cuda.stream(copy_stream):
                dxs[b].copy_(host_x[b], non_blocking=True)
            copied[b].record(copy_stream)

        def step_ce(i):
            b = i % 2
            if i == 0:
                issue_copy(0)
            issue_copy(i + 1)
            stream.wait_event(copied[b])
            plan_e.execute_batched(dxs[b], oute)
            free[b].record(stream)
            for h_, d_ in zip(host_o2[b], oute):
                h_.copy_(d_, non_blocking=True)

        for i in range(2):
            step_ce(i)
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for i in range(2, 2 + esteps):
            step_ce(i)
        stream.wait_stream(copy_stream)
        c1.record(stream)
        torch.cuda.synchronize()
        ce = max_over_ranks(c0.elapsed_time(c1) / 1e3, dist, dev)
        e2e = {"value": Se * esteps * world / ee, "unit": "transforms/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "batch": Se, "steps": esteps,
               "h2d_gbs": h2d * esteps / ee / 1e9, "h2d_link_gbs": link_gbs,
               "frac_of_link": h2d * esteps / ee / 1e9 / link_gbs,
               "bound": "host -> device link (every signal's 8 N bytes cross it)",
               "form": "sfft4_execute_batched_host on pinned host batches (library zero-copy staging, "
                       "asynchronous executes in turn, results copied to pinned host outputs), every step",
               "copy_engine_form": {"value": Se * esteps * world / ce, "h2d_gbs": h2d * esteps / ce / 1e9,
                                    "form": "torch pinned copies on a copy stream (double-buffered) + "
                                            "sfft4_execute_batched + results to pinned host"}}
        plan_e.close()
        del dx, dxs, host_x

    # the same batch with the FP32 radix-2 DFT
    fp32_form = None
    if not args.no_fp32_form and args.precision != "fp32":
        plan_f = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=1234, max_batch=S, precision="fp32")
        outf = [plan_f._outputs(S), plan_f._outputs(S)]
        steps_f = max(3, min(args.steps, 50))
        ef = max_over_ranks(timed(lambda: plan_f.execute_batched(xs, outf[0]), steps_f, args.warmup, stream, dist),
                            dist, dev)
        cf = [0]

        def step_f():
            plan_f.execute_batched(xs, outf[cf[0] % 2], asynchronous=True)
            cf[0] += 1

        efp = max_over_ranks(timed(step_f, steps_f, args.warmup, stream, dist, finish=plan_f.wait), dist, dev)
        fp32_form = {"value": S * steps_f * world / ef, "unit": "transforms/s", "steps": steps_f,
                     "form": "batched sfft4_execute_batched, FP32 radix-2 DFT, one synchronous execute per step",
                     "pipelined": {"value": S * steps_f * world / efp, "ms_per_step": 1e3 * efp / steps_f,
                                   "form": "the same batches as asynchronous executes (two workspaces in turn), "
                                           "like the headline"}}
        plan_f.close()

    # crossover context: a dense length-N FFT (cuFFT through torch, outside the library) of
    # the same signals, 32 per call
    dense = None
    chunk = min(S, 32)
    yd = torch.empty((chunk, N_DEF), dtype=torch.complex64, device=dev)

    def step_d():
        for c0 in range(0, S, chunk):
            torch.fft.fft(xs[c0:c0 + chunk], out=yd)

    steps_d = max(3, min(args.steps, 20))
    ed = timed(step_d, steps_d, args.warmup, stream, None)
    dense = {"value": S * steps_d / ed, "unit": "transforms/s", "form": "torch.fft.fft (cuFFT) of the same "
             "complex64 signals, full N-point spectrum, not part of the library"}
    del yd

    uneven = None
    if args.uneven_signals > 0:
        uneven = uneven_form(s4, args, dev, stream, dist)

    # plain form: one signal per execute call, FP32 DFT
    plain = plain_graph = None
    if args.plain_signals > 0:
        plan_p = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=1234, precision="fp32")
        outp = plan_p._outputs(1)
        ns = min(args.plain_signals, S)

        def step_p():
            for i in range(ns):
                plan_p.execute(xs[i], outp)

        pe = timed(step_p, 2, 1, stream, None)
        plain = {"value": ns * 2 / pe, "unit": "transforms/s", "form": "single-signal sfft4_execute, FP32 DFT"}
        plan_p.close()
        # the same with the execute captured once as a CUDA graph and replayed (same buffers)
        plan_g = s4.Plan(N_DEF, K_DEF, L_DEF, Q_DEF, seed=1234, precision="fp32", graph=True)
        outg = plan_g._outputs(1)
        xg = torch.empty(N_DEF, dtype=torch.complex64, device=dev)

        def step_g():
            for i in range(ns):
                xg.copy_(xs[i])
                plan_g.execute(xg, outg)

        pg = timed(step_g, 2, 1, stream, None)
        plain_graph = {"value": ns * 2 / pg, "unit": "transforms/s",
                       "form": "single-signal sfft4_execute replayed as one CUDA graph per call, FP32 DFT "
                               "(includes a 32 MB device copy of each signal into the captured buffer)"}
        plan_g.close()

    cpu = None
    accuracy = None
    if pool is not None:
        n = cpu_workers
        rate, ores = oracle_sample(pool, n, N_DEF, K_DEF, L_DEF, Q_DEF, args.snr, 7_000, plan_seed=1234)
        pool.close()
        try:
            accuracy = accuracy_vs_oracle(s4, ores, n, args.snr, 7_000, 1234, dev)
        except Exception as e:  # a report beside the measurement: never the reason the line is missing
            accuracy = {"error": f"{type(e).__name__}: {e}"}
        cpu = {"value": rate, "unit": "transforms/s", "cores": n, "kind": "oracle", "cpu_model": cpu_model(),
               "sample": f"{n} transforms of the workload, one per spawned process on {n} host cores "
                         "(FP64 numpy oracle); rate = sum of 1 / (seconds of each O.run), signal "
                         "synthesis excluded"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "transforms/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "N": N_DEF, "K": K_DEF, "l": L_DEF, "q": Q_DEF,
                           "snr_db": args.snr, "batch_per_gpu": S, "B1": plan.info["B1"],
                           "iterations": plan.info["n_iters"], "precision": args.precision,
                           "fold_order": args.fold_order,
                           "execute": ("asynchronous, two workspaces in turn (batch k's decode chain "
                                       "overlaps batch k+1's gather)") if pipelined else "synchronous",
                           "samples_per_transform": plan.info["samples_per_transform"],
                           "l2": "inputs larger than L2 (touched samples per step "
                                 f"{S * plan.info['samples_per_transform'] * 32 / 1e9:.1f} GB of 32 B sectors)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "accuracy_vs_oracle": accuracy,
                "gpu_launches": int(prof["fold_launches"] + prof["fft_launches"] + prof["decode_launches"]
                                    + prof["finalize_launches"]),
                "clocks": clk.summary(), "forms": {"batched": {"value": value, "precision": args.precision,
                                                               "pipelined": pipelined},
                                                   "batched_sync": sync_form,
                                                   "batched_fp32": fp32_form, "plain_fp32": plain, "plain_fp32_graph": plain_graph,
                                                   "uneven_batch": uneven, "dense_fft_context": dense}}
        print(json.dumps(line), flush=True)
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
