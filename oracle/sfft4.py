"""sFFT4.0, step by step, in FP64 and exact integers (oracle; test infrastructure only).

Conventions (Section 2.1, Eq. 1-2): X_f = (1/N) sum_n x_n omega_N^{f n},
omega_N = exp(-2 pi i / N), so x_n = sum_f X_f exp(+2 pi i f n / N).

Per iteration m (Section 3.1) with (sigma, a) drawn by Philox:

1. Bucketization (Lemma 1, Eq. 13), gather form of S_tau P_sigma (Eq. 7, reading R2):
   round s reads x'_t = x[(sigma t + o_s) mod N], t = -h..h, with o_s = a + sigma tau_s,
   multiplies by G_t (Q_L, Eq. 10), folds t -> t mod B (U_L, Eq. 11) and takes the
   B-point DFT: yhat_s[b] = sum_j z_s[j] exp(-2 pi i b j / B).
   Then yhat_s[b] = sum_u G'^_{bL-u} X_{sigma^-1 u} exp(2 pi i (sigma^-1 u) o_s / N).
2. Update (Section 3.1, iteration steps 2-3): subtract every found (f, v) from the
   buckets b(u)-1, b(u), b(u)+1 of every round, u = sigma f mod N (reading R13).
3. Large-bucket selection (Section 3, p >= 1 buckets; reading R11): the n_c(m) largest
   |yhat_0|^2 above a significance floor theta, n_c(m) = min(B_m, ceil(c max(K_m, 1)))
   with K_m the schedule's expected sparsity (Section 3.1).
4. Multiscale location (Section 3.2, Eq. 15-19, Fig. 3-4; readings R6-R10) over the
   region [bL - L, bL + L) in exact integer arithmetic on phases held as 2^-32 turns;
   a level votes when the phase and the magnitude of its round agree with round 0
   (Eq. 14-15); accepted when all levels vote and b(u) = b.
5. Median estimation over the rounds (Eq. 14; reading R12) and merge (reading R15).
All iterations of the static schedule run (no data-dependent early exit).
Output: top-K by |v| (reading R16), sorted by frequency.

Every decision also records its margin so tests can tell fragile decisions (where
FP32 and FP64 arithmetic may legitimately disagree) from robust ones.
"""

import math

import numpy as np

from .philox import permutation_draw
from .plan import Q_DEN
from .window import WindowCache

TWO32 = 1 << 32


def bucket_of(u, L, B):
    """Bucket of permuted frequency u: round(u / L) mod B, halves rounded up (Eq. 14, R5)."""
    return ((u + L // 2) // L) % B


def signed_offset(k, N):
    """Representative of k mod N in [-N/2, N/2)."""
    return ((k + N // 2) % N) - N // 2


def circ_dist(a, b):
    """Distance between two phases in 2^-32 turns, on the circle."""
    d = (a - b) % TWO32
    return np.minimum(d, TWO32 - d)


def phase_turns_fixed(c):
    """Phase of c in turns as an integer in [0, 2^32) (2^-32 turns per unit)."""
    ang = np.arctan2(c.imag, c.real) / (2.0 * np.pi)
    return np.round(ang * float(TWO32)).astype(np.int64) % TWO32


def round_offsets(sigma, a, it, N):
    """o_s = a + sigma tau_s mod N for s = 0..S (tau_0 = 0)."""
    return [(a + sigma * t) % N for t in it.tau]


def bucketize(x, N, B, G, h, sigma, offsets):
    """yhat_s = F_B U_L Q_L S P x for each round offset (Lemma 1), shape (R, B), complex128."""
    t = np.arange(-h, h + 1, dtype=np.int64)
    slot = t % B
    Y = np.empty((len(offsets), B), dtype=np.complex128)
    for s, o in enumerate(offsets):
        idx = (sigma * t + o) % N
        y = G * x[idx]
        z = (np.bincount(slot, weights=y.real, minlength=B)
             + 1j * np.bincount(slot, weights=y.imag, minlength=B))
        Y[s] = np.fft.fft(z)
    return Y


def unique_samples(it, N):
    """Number of distinct x positions one iteration reads: |union_s [tau_s - h, tau_s + h]|."""
    iv = sorted((t - it.h, t + it.h) for t in it.tau)
    total, cur_lo, cur_hi = 0, None, None
    for lo, hi in iv:
        if cur_hi is None or lo > cur_hi + 1:
            if cur_hi is not None:
                total += cur_hi - cur_lo + 1
            cur_lo, cur_hi = lo, hi
        else:
            cur_hi = max(cur_hi, hi)
    total += cur_hi - cur_lo + 1
    return min(total, N)


class FoundSet:
    """x^m of Section 3.1: frequencies, values, votes and the iteration of first acceptance."""

    def __init__(self):
        self.f, self.v, self.votes, self.iter = [], [], [], []
        self.index = {}

    def __len__(self):
        return len(self.f)

    def copy(self):
        c = FoundSet()
        c.f, c.v, c.votes, c.iter = list(self.f), list(self.v), list(self.votes), list(self.iter)
        c.index = dict(self.index)
        return c

    def merge(self, f, v, votes, m):
        """x^m = x^{m-1} + x'^m: a repeated frequency adds its value (reading R15)."""
        f = int(f)
        if f in self.index:
            self.v[self.index[f]] += v
        else:
            self.index[f] = len(self.f)
            self.f.append(f)
            self.v.append(complex(v))
            self.votes.append(int(votes))
            self.iter.append(int(m))


def update(Y, found, N, B, L, sigma, offsets, Ghat):
    """yhat' = yhat - yhat_update (Section 3.1 steps 2-3, reading R13); returns a new array."""
    Y = Y.copy()
    if len(found) == 0:
        return Y
    f = np.asarray(found.f, dtype=np.int64)
    v = np.asarray(found.v, dtype=np.complex128)
    u = (sigma * f) % N
    b0 = bucket_of(u, L, B)
    for db in (-1, 0, 1):
        b = (b0 + db) % B
        k = signed_offset(b * L - u, N)
        g = Ghat[np.abs(k)]
        for s, o in enumerate(offsets):
            ph = ((f * o) % N).astype(np.float64) / N
            np.subtract.at(Y[s], b, g * v * np.exp(2j * np.pi * ph))
    return Y


def select(Y0, n_c, theta):
    """Candidate buckets: top n_c by |yhat_0|^2 (ties to the lower b), strictly above theta (R11).

    Returns (sorted bucket indices, margin) where margin is the smallest relative gap
    of a selection decision (n_c-th vs next key, and keys vs theta)."""
    key = Y0.real ** 2 + Y0.imag ** 2
    B = key.shape[0]
    order = np.lexsort((np.arange(B), -key))
    top = order[:n_c]
    keep = top[key[top] > theta]
    gaps = [np.inf]
    if n_c < B:
        k1, k2 = key[order[n_c - 1]], key[order[n_c]]
        gaps.append((k1 - k2) / max(k1, 1e-300))
    if theta > 0:
        gaps.append(float(np.min(np.abs(key[top] - theta))) / theta if top.size else np.inf)
    return np.sort(keep), float(min(gaps))


def locate(Y, bs, it, N, n, l, qn, mag_tol):
    """Multiscale location of the candidate buckets bs (Section 3.2; R6-R10).

    Level s = 1..S-1 (block levels): phi_s = phase(yhat_s[b] conj(yhat_0[b])) ~ u tau_s / N;
    the region [u_min, u_min + Lbar_s) splits into l blocks with centres
    c_j = u_min + (2j+1) Lbar_s / (2l); j* = argmin_j |phi_s - c_j tau_s / N| (circular,
    ties to the lowest j); the new region starts at u_min + floor((j* - q/2) Lbar_s / l).
    Level S (final): the Lbar_S integers u_min + i compete directly.
    The search region of bucket b starts as [bL - L, bL + L) (Lbar_1 = 2L).
    Votes: level s votes when |phi_s - u* tau_s / N| <= H_s and
    | |yhat_s[b]|^2 - |yhat_0[b]|^2 | <= mag_tol |yhat_0[b]|^2.
    Returns dict with u*, votes, ownership and the decision margins (2^-32 turns)."""
    bs = np.asarray(bs, dtype=np.int64)
    S, L, B = it.S, it.L, it.B
    shift = 32 - n
    nc = bs.shape[0]
    Phi = [phase_turns_fixed(Y[s, bs] * np.conj(Y[0, bs])) for s in range(1, S + 1)]
    umin = bs * L - L
    margin = np.full(nc, np.iinfo(np.int64).max, dtype=np.int64)
    jstars = []
    for s in range(1, S):
        Lb, ts = it.Lbar[s - 1], it.tau[s]
        A = ((umin % N) * ts) % N
        j = np.arange(l, dtype=np.int64)
        C = ((2 * j + 1) * Lb * ts) % (2 * l * N)
        E = ((A[:, None] << shift) + (((C << shift) + l) // (2 * l))[None, :]) % TWO32
        d = circ_dist(Phi[s - 1][:, None], E)
        jstar = np.argmin(d, axis=1)
        ds = np.sort(d, axis=1)
        margin = np.minimum(margin, ds[:, 1] - ds[:, 0])
        jstars.append(jstar)
        umin = umin + np.floor_divide((2 * jstar * Q_DEN - qn) * Lb, 2 * l * Q_DEN)
    Lb, ts = it.Lbar[S - 1], it.tau[S]
    i = np.arange(Lb, dtype=np.int64)
    u = (umin[:, None] + i[None, :]) % N
    P = ((u * ts) % N) << shift
    d = circ_dist(Phi[S - 1][:, None], P)
    istar = np.argmin(d, axis=1)
    if Lb > 1:
        ds = np.sort(d, axis=1)
        margin = np.minimum(margin, ds[:, 1] - ds[:, 0])
    ustar = (umin + istar) % N
    votes = np.zeros(nc, dtype=np.int64)
    m0 = np.abs(Y[0, bs]) ** 2
    mag_margin = np.full(nc, np.inf)
    for s in range(1, S + 1):
        ps = ((ustar * it.tau[s]) % N) << shift
        ds = circ_dist(Phi[s - 1], ps)
        dm = np.abs(np.abs(Y[s, bs]) ** 2 - m0)
        votes += (ds <= it.H[s - 1]) & (dm <= mag_tol * m0)
        margin = np.minimum(margin, np.abs(ds - it.H[s - 1]))
        mag_margin = np.minimum(mag_margin, np.abs(dm - mag_tol * m0) / m0)
    own = bucket_of(ustar, L, B) == bs
    return {"ustar": ustar, "votes": votes, "own": own, "margin": margin,
            "mag_margin": mag_margin,
            "Phi": Phi, "jstar": jstars, "istar": istar}


def estimate(Y, bs, ustar, sigma, offsets, it, N, Ghat):
    """Median estimate over rounds (Eq. 14, reading R12).

    v_r = yhat_r[b] exp(-2 pi i (f o_r mod N) / N) / G'^_{bL-u}, f = sigma^-1 u mod N;
    v = median_r Re v_r + i median_r Im v_r (mean of the middle two for even R)."""
    bs = np.asarray(bs, dtype=np.int64)
    sinv = pow(int(sigma), -1, N)
    f = (sinv * ustar) % N
    k = signed_offset(bs * it.L - ustar, N)
    g = Ghat[np.abs(k)]
    vr = np.empty((len(offsets), bs.shape[0]), dtype=np.complex128)
    for r, o in enumerate(offsets):
        ph = ((f * o) % N).astype(np.float64) / N
        vr[r] = Y[r, bs] * np.exp(-2j * np.pi * ph) / g
    v = np.median(vr.real, axis=0) + 1j * np.median(vr.imag, axis=0)
    return f, v, vr


def decode_iteration(Yraw, found, it, plan, sigma, a, theta, Ghat):
    """Steps 2-5 of one iteration on given raw bucket arrays; returns (found', trace).

    Also the replay entry point: tests feed it the bucket arrays the CUDA path
    computed, so both decoders see identical inputs."""
    N, n = plan.N, plan.n
    offsets = round_offsets(sigma, a, it, N)
    Yres = update(Yraw, found, N, it.B, it.L, sigma, offsets, Ghat)
    n_c = it.n_c
    bs, sel_margin = select(Yres[0], n_c, theta)
    need = it.S if plan.min_votes <= 0 else min(plan.min_votes, it.S)
    out = found.copy()
    tr = {"m": it.m, "sigma": sigma, "a": a, "offsets": offsets, "Yres": Yres,
          "cands": bs, "sel_margin": sel_margin, "n_c": n_c}
    if bs.size == 0:
        tr.update(loc=None, accepted=np.zeros(0, bool), f=np.zeros(0, np.int64),
                  v=np.zeros(0, np.complex128))
        return out, tr
    loc = locate(Yres, bs, it, N, n, plan.l, plan.qn, plan.mag_tol)
    acc = (loc["votes"] >= need) & loc["own"]
    f, v, vr = estimate(Yres, bs[acc], loc["ustar"][acc], sigma, offsets, it, N, Ghat)
    for fi, vi, vo in zip(f, v, loc["votes"][acc]):
        out.merge(fi, vi, vo, it.m)
    tr.update(loc=loc, accepted=acc, f=f, v=v, vr=vr)
    return out, tr


def run(x, plan, signal=0, trace=False, stop_after=None):
    """Whole sFFT4.0 of one signal x (complex, length N). Returns a result dict.

    result: f (sorted, <= K), v (complex128), votes, iter, nfound, samples (unique x
    positions read), found (the full FoundSet), traces (per iteration, if trace)."""
    N, K = plan.N, plan.K
    x = np.asarray(x, dtype=np.complex128)
    assert x.shape == (N,)
    wc = WindowCache(N, plan.delta)
    found = FoundSet()
    theta = None
    traces, samples = [], 0
    for it in plan.iters:
        if stop_after is not None and it.m > stop_after:
            break
        sigma, a = permutation_draw(plan.seed, signal, it.m, N)
        G, h, Ghat = wc.get(it.B)
        offsets = round_offsets(sigma, a, it, N)
        Y = bucketize(x, N, it.B, G, h, sigma, offsets)
        samples += unique_samples(it, N)
        if theta is None:
            Y0 = Y[0]
            theta = plan.sig_floor * float(np.max(Y0.real ** 2 + Y0.imag ** 2))
        found, tr = decode_iteration(Y, found, it, plan, sigma, a, theta, Ghat)
        if trace:
            tr["Y"] = Y
            tr["theta"] = theta
            tr["found_after"] = found.copy()
            traces.append(tr)
    res = finalize(found, K)
    res.update(samples=samples, found=found, traces=traces, theta=theta)
    return res


def finalize(found, K):
    """Top-K by |v| (ties to the lower f), then sorted by f (reading R16)."""
    if len(found) == 0:
        return {"f": np.zeros(0, np.int64), "v": np.zeros(0, np.complex128),
                "votes": np.zeros(0, np.int64), "iter": np.zeros(0, np.int64), "nfound": 0}
    f = np.asarray(found.f, dtype=np.int64)
    v = np.asarray(found.v, dtype=np.complex128)
    votes = np.asarray(found.votes, dtype=np.int64)
    its = np.asarray(found.iter, dtype=np.int64)
    order = np.lexsort((f, -np.abs(v)))[:K]
    order = order[np.argsort(f[order], kind="stable")]
    return {"f": f[order], "v": v[order], "votes": votes[order], "iter": its[order],
            "nfound": int(order.size)}
